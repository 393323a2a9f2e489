// Dense-covariance likelihood (LISA_COV_FULL): the complete analysis Sec. III.A names, with six
// flexible noise terms (three diagonal perturbations, three correlation splines z_AE, z_AT, z_ET),
// and the Wishart term of Sec. III.C per bin, -nu [tr(C^-1 P) + ln det C].
//
// In the normalised units of the tables (every template divided by the channel's periodogram
// P_cc, so P-hat_cc = 1 and the off-diagonal P-hat_ab = Re P_ab / sqrt(P_aa P_bb)):
//   D_c = (a_oms^2 Go_c + a_tm^2 Gt_c) 10^{p_c},   H_c = 10^{log10 A + p_h} (f / f_ref)^n Gh_c,
//   C_cc = D_c + H_c,   C_ab = sqrt(D_a D_b) R_ab,
//   R_AE = r_AE, R_AT = r_AT, R_ET = r_AE r_AT + s_AE s_AT r_ET,  r = z / sqrt(1 + z^2),
//   s = 1 / sqrt(1 + z^2).
// Both paths evaluate the term through the diagonal scaling sigma_c = sqrt(C_cc) (exact, and
// every intermediate stays of order one whatever the perturbations do):
//   K_ab = R_ab g_a g_b  (g_c = sqrt(D_c / C_cc), unit diagonal),  Q_cc = 1 / C_cc,
//   Q_ab = P-hat_ab / sqrt(C_aa C_bb),   tr(C^-1 P-hat) = tr(K^-1 Q) = sum adj(K)_ab Q_ab / det K,
//   ln det C = ln det K + sum_c ln C_cc,
// with the 3x3 adjugate and determinant written out.  The constant -sum nu sum_c ln P_cc is
// added by the finalize, as for the diagonal model.
#include "lisa_math.cuh"

namespace lisa {
namespace {
using namespace dm;

constexpr int kFullThreads = 128;

// The per-bin term in FP64 (without the factor nu): tr(C^-1 P-hat) + ln det C from the spline
// values (log10 units for the noise and SGWB splines, plain values for the correlations), the
// bin's table q (x, ell, nu, Go[3], Gt[3], Gh[3]), its cross-spectral entries xc[3], and the
// state's parameters.  Non-finite results (a PSD outside the FP64 range, a singular K) propagate,
// and the finalize turns the state's log L into -inf.
template <bool HAS_H>
__device__ __forceinline__ double full_term64(const double pn[3], double ph, const double zv[3], const double* q,
                                              const double* xc, double ao2, double at2, double lA, double sl) {
    double D[3], Cd[3];
    const double eh = HAS_H ? exp10(lA + ph) * exp2(sl * q[1]) : 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        D[c] = (ao2 * q[3 + c] + at2 * q[6 + c]) * exp10(pn[c]);
        Cd[c] = HAS_H ? D[c] + eh * q[9 + c] : D[c];
    }
    double r[3], sq[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sq[k] = 1.0 / sqrt(1.0 + zv[k] * zv[k]);
        r[k] = zv[k] * sq[k];
    }
    const double R01 = r[0], R02 = r[1], R12 = r[0] * r[1] + sq[0] * sq[1] * r[2];
    double u[3], g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u[c] = 1.0 / sqrt(Cd[c]);
        g[c] = sqrt(D[c]) * u[c];
    }
    const double K01 = R01 * g[0] * g[1], K02 = R02 * g[0] * g[2], K12 = R12 * g[1] * g[2];
    const double A00 = 1.0 - K12 * K12, A11 = 1.0 - K02 * K02, A22 = 1.0 - K01 * K01;
    const double A01 = K02 * K12 - K01, A02 = K01 * K12 - K02, A12 = K01 * K02 - K12;
    const double det = A00 + K01 * A01 + K02 * A02;
    const double tr = (A00 * u[0] * u[0] + A11 * u[1] * u[1] + A22 * u[2] * u[2] +
                       2.0 * (A01 * xc[0] * u[0] * u[1] + A02 * xc[1] * u[0] * u[2] + A12 * xc[2] * u[1] * u[2])) /
                      det;
    return tr + log(det) + log(Cd[0]) + log(Cd[1]) + log(Cd[2]);
}

// ---- plain FP64 path --------------------------------------------------------------------------
template <bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(kThreads)
    full_fp64_kernel(const WorkItem* __restrict__ items, int n_items, const double* __restrict__ rec64,
                     const double* __restrict__ cross64, const double* __restrict__ theta,
                     const int32_t* __restrict__ sstat, const int32_t* __restrict__ nint,
                     const double* __restrict__ srec, int kmax, int nsp, const DatasetDev* __restrict__ ds,
                     double* __restrict__ partial) {
    constexpr int NSP = 3 + (HAS_H ? 1 : 0) + 3;
    constexpr int ZB = 3 + (HAS_H ? 1 : 0);   // first correlation spline
    __shared__ double red[kThreads];
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const int sc = w.sc;
        const int R = kThreads / sc;
        const int ls = tid & (sc - 1);
        const int r = tid / sc;
        const int s = w.s0 + ls;
        const bool active = ls < w.ns && sstat[s] == 0;
        double acc = 0.0;
        if (active) {
            const int lo = (r * w.nb) / R, hi = ((r + 1) * w.nb) / R;
            if (lo < hi) {
                const double* th = theta + (size_t)s * LISA_N_THETA;
                const double ao2 = th[0] * th[0], at2 = th[1] * th[1], lA = th[2], n1 = th[3];
                const double n2 = BROKEN ? th[4] : n1;
                const double* base[NSP];
                int j[NSP], last[NSP];
                double xl[NSP], xr[NSP], ca[NSP], cb[NSP], cc[NSP], cd[NSP];
                const double x0 = __ldg(rec64 + (w.bin0 + lo) * kRec);
                for (int a = 0; a < NSP; ++a) {
                    const int64_t sp = (int64_t)s * nsp + a;
                    base[a] = srec + sp * (int64_t)(kmax + 1) * kSplineRec;
                    last[a] = nint[sp] - 1;
                    j[a] = find_interval<double, kSplineRec, 0>(base[a], nint[sp], x0);
                    const double* z = base[a] + (size_t)j[a] * kSplineRec;
                    xl[a] = z[0]; xr[a] = z[1]; ca[a] = z[2]; cb[a] = z[3]; cc[a] = z[4]; cd[a] = z[5];
                }
                for (int i = lo; i < hi; ++i) {
                    const double* q = rec64 + (w.bin0 + i) * kRec;
                    double qq[kRec];
                    for (int k = 0; k < kRec; ++k) qq[k] = __ldg(q + k);
                    const double x = qq[0];
                    double P[NSP];
                    for (int a = 0; a < NSP; ++a) {
                        while (x >= xr[a] && j[a] < last[a]) {
                            ++j[a];
                            const double* z = base[a] + (size_t)j[a] * kSplineRec;
                            xl[a] = z[0]; xr[a] = z[1]; ca[a] = z[2]; cb[a] = z[3]; cc[a] = z[4]; cd[a] = z[5];
                        }
                        const double t = x - xl[a];
                        P[a] = ca[a] + t * (cb[a] + t * (cc[a] + t * cd[a]));
                    }
                    const double* xc = cross64 + (w.bin0 + i) * kCross;
                    const double xcv[3] = {__ldg(xc), __ldg(xc + 1), __ldg(xc + 2)};
                    const double sl = BROKEN ? (qq[1] < 0.0 ? n1 : n2) : n1;
                    const double pn[3] = {P[0], P[1], P[2]};
                    const double zv[3] = {P[ZB], P[ZB + 1], P[ZB + 2]};
                    acc += qq[2] * full_term64<HAS_H>(pn, HAS_H ? P[3] : 0.0, zv, qq, xcv, ao2, at2, lA, sl);
                }
            }
        }
        red[tid] = acc;
        __syncthreads();
        if (r == 0 && ls < w.ns && sstat[s] == 0) {
            double sum = 0.0;
            for (int q = 0; q < R; ++q) sum += red[ls + q * sc];
            const DatasetDev& D = ds[w.ds];
            partial[D.pbase + (int64_t)(s - D.s0) * D.ntiles + w.tile] = sum;
        }
        __syncthreads();
    }
}

// ---- FP32 bulk path ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned k = 0; k < limit; ++k)
        if (bar_try(bar, parity)) return true;
    return false;
}
// the item's two tables (the pair-block bin table and the cross-spectral table) by two bulk
// copies completing on one mbarrier
__device__ __forceinline__ void stage_item(float* dst, const float* rec32, const float* cross32, const WorkItem& w,
                                           int tile_bins, uint64_t* bar) {
    const unsigned b1 = (unsigned)w.nb * kRec * sizeof(float);
    const unsigned b2 = (unsigned)(w.nb >> 1) * kPairCross * sizeof(float);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(b1 + b2)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(rec32 + (w.bin0 >> 1) * kPairRec), "r"(b1), "r"(smem_u32(bar))
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst + (size_t)tile_bins * kRec)),
        "l"(cross32 + (w.bin0 >> 1) * kPairCross), "r"(b2), "r"(smem_u32(bar))
        : "memory");
}

constexpr float kFullSafe = 120.0f;   // FP32 path: exponents (log2) and PSD scale within 2^+-120

// One thread per state and contiguous bins of the item, one bin at a time.  The current interval of
// each spline (cubic about its midpoint, log2 units, as the setup writes FP32 records) is kept in
// registers, its right end and index in shared memory.  A bin is evaluated in FP32 when every
// interval it uses is well conditioned and every exponent and diagonal entry stays within 2^+-120;
// otherwise ("careful" bins, rare) the spline values are formed in float-float from the records'
// low parts and the term in FP64 by full_term64, the same code as the plain path.
template <bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(kFullThreads, 4)
    full_fp32_kernel(const WorkItem* __restrict__ items, int n_items, const float* __restrict__ rec32,
                     const float* __restrict__ cross32, const float* __restrict__ xlo32,
                     const float* __restrict__ elllo32, const StateParams* __restrict__ prm,
                     const double* __restrict__ theta,
                     const int32_t* __restrict__ sstat, const float* __restrict__ kxr,
                     const float* __restrict__ srec, int kmax, int nsp, const DatasetDev* __restrict__ ds,
                     double* __restrict__ partial, int* __restrict__ err, int tile_bins, unsigned wait_limit) {
    constexpr int NSP = 3 + (HAS_H ? 1 : 0) + 3;
    constexpr int ZB = 3 + (HAS_H ? 1 : 0);
    constexpr float kL2 = 3.32192809488736234787f;   // log2(10): the records' coefficients carry it
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float s_xr[NSP][kFullThreads];
    __shared__ int s_jj[NSP][kFullThreads];
    __shared__ double red[kFullThreads];
    __shared__ int s_fail;   // a bounded wait ran out: stage nothing more (a late copy may still land)
    const int tid = threadIdx.x;
    const size_t stage_floats = (size_t)tile_bins * kRec + (size_t)(tile_bins >> 1) * kPairCross;
    float* sb[2] = {reinterpret_cast<float*>(smem), reinterpret_cast<float*>(smem) + stage_floats};
    if (tid == 0) {
        s_fail = 0;
        bar_init(&bars[0]);
        bar_init(&bars[1]);
        if ((int)blockIdx.x < n_items) stage_item(sb[0], rec32, cross32, items[blockIdx.x], tile_bins, &bars[0]);
    }
    __syncthreads();
    // per spline: the current interval's cubic (xo, c0..c3) and whether it is well conditioned
    float cxo[NSP], c0[NSP], c1[NSP], c2[NSP], c3[NSP];
    unsigned hm = 0;
    int k = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++k) {
        const int b = k & 1;
        const int nxt = it + gridDim.x;
        if (nxt < n_items && tid == 0 && !s_fail)
            stage_item(sb[b ^ 1], rec32, cross32, items[nxt], tile_bins, &bars[b ^ 1]);
        const WorkItem w = items[it];
        const bool ok = bar_wait(&bars[b], (unsigned)(k >> 1) & 1u, wait_limit);
        if (!ok) {
            s_fail = 1;   // read by thread 0 after the next barrier
            atomicOr(err, kErrTimeout);
        }
        const float* tb = sb[b];
        const float* tx = sb[b] + (size_t)tile_bins * kRec;   // cross-spectral pair blocks
        const int sc = w.sc;
        const int R = kFullThreads / sc;
        const int ls = tid & (sc - 1);
        const int r = tid / sc;
        const int s = w.s0 + ls;
        const bool active = ok && ls < w.ns && (sstat[s] & kUserBits) == 0;
        ff accf = {0.f, 0.f};
        double far = 0.0;
        if (active) {
            const int lo = (r * w.nb) / R, hi = ((r + 1) * w.nb) / R;
            if (lo < hi) {
                const StateParams p = prm[s];
                const float ao2 = p.ao2, at2 = p.at2, Af = HAS_H ? p.Af : 0.f;
                const double* th = theta + (size_t)s * LISA_N_THETA;
                auto rec = [&](int a, int j) {
                    return srec + (((int64_t)s * nsp + a) * (int64_t)(kmax + 1) + j) * kSplineRec32;
                };
                auto install = [&](int a, int j) {
                    const float4 A = __ldg(reinterpret_cast<const float4*>(rec(a, j)));
                    const float4 B = __ldg(reinterpret_cast<const float4*>(rec(a, j)) + 1);
                    s_xr[a][tid] = A.x;
                    s_jj[a][tid] = j;
                    cxo[a] = A.y;
                    c0[a] = A.z;
                    c1[a] = A.w;
                    c2[a] = B.x;
                    c3[a] = B.y;
                    hm = B.w <= (float)kRobustT ? (hm & ~(1u << a)) : (hm | (1u << a));
                };
                // intervals at the first bin: the count of right ends <= x in the right-end table
                {
                    const float x = fld(tb, lo, 0);
                    const int kxs = kxr_stride(kmax);
                    hm = 0;
#pragma unroll
                    for (int a = 0; a < NSP; ++a) {
                        const float4* kq = reinterpret_cast<const float4*>(kxr + ((int64_t)s * nsp + a) * kxs);
                        int j = 0;
                        for (int q = 0; q < kxs / 4; ++q) {
                            const float4 v = __ldg(kq + q);
                            j += (v.x <= x) + (v.y <= x) + (v.z <= x) + (v.w <= x);
                        }
                        install(a, min(j, kmax));
                    }
                }
                float xmin = s_xr[0][tid];
#pragma unroll
                for (int a = 1; a < NSP; ++a) xmin = fminf(xmin, s_xr[a][tid]);
                float acc = 0.f;
                int run = 0;
                for (int i = lo; i < hi; ++i) {
                    const float x = fld(tb, i, 0);
                    if (x >= xmin) {
#pragma unroll
                        for (int a = 0; a < NSP; ++a) {
                            if (x >= s_xr[a][tid]) {
                                int j = s_jj[a][tid];
                                do {
                                    ++j;
                                } while (j < kmax && x >= __ldg(rec(a, j)));
                                install(a, j);
                            }
                        }
                        xmin = s_xr[0][tid];
#pragma unroll
                        for (int a = 1; a < NSP; ++a) xmin = fminf(xmin, s_xr[a][tid]);
                    }
                    const float ell = fld(tb, i, 1), nu = fld(tb, i, 2);
                    float pv[NSP];
#pragma unroll
                    for (int a = 0; a < NSP; ++a) {
                        const float t = x - cxo[a];
                        pv[a] = fmaf(fmaf(fmaf(c3[a], t, c2[a]), t, c1[a]), t, c0[a]);
                    }
                    bool careful = hm != 0;
                    float term = 0.f;
                    if (!careful) {
                        float D[3], Cc[3];
                        float eh = 0.f;
                        if (HAS_H) {
                            const float sl = BROKEN ? (ell < 0.f ? p.n1 : p.n2) : p.n1;
                            const float ex = fmaf(sl, ell, pv[3]);
                            careful |= !(fabsf(ex) < kFullSafe);
                            eh = Af * ex2_approx(ex);
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            careful |= !(fabsf(pv[c]) < kFullSafe);
                            D[c] = fmaf(ao2, fld(tb, i, 3 + c), at2 * fld(tb, i, 6 + c)) * ex2_approx(pv[c]);
                            Cc[c] = HAS_H ? fmaf(eh, fld(tb, i, 9 + c), D[c]) : D[c];
                        }
                        const float dmin = fminf(fminf(D[0], D[1]), D[2]);
                        const float cmax = fmaxf(fmaxf(Cc[0], Cc[1]), Cc[2]);
                        careful |= !(dmin > 1e-36f && cmax < 1e36f);
                        if (!careful) {
                            float rr[3], ss[3];
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const float zq = pv[ZB + q];   // z log2(10)
                                const float iq = rsqrtf(fmaf(zq, zq, kL2 * kL2));
                                rr[q] = zq * iq;
                                ss[q] = kL2 * iq;
                            }
                            const float R12 = fmaf(rr[0], rr[1], ss[0] * ss[1] * rr[2]);
                            float u[3], g[3];
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                u[c] = rsqrtf(Cc[c]);
                                g[c] = D[c] * rsqrtf(D[c]) * u[c];
                            }
                            const float K01 = rr[0] * g[0] * g[1], K02 = rr[1] * g[0] * g[2], K12 = R12 * g[1] * g[2];
                            const float A00 = fmaf(-K12, K12, 1.f), A11 = fmaf(-K02, K02, 1.f), A22 = fmaf(-K01, K01, 1.f);
                            const float A01 = fmaf(K02, K12, -K01), A02 = fmaf(K01, K12, -K02), A12 = fmaf(K01, K02, -K12);
                            const float det = fmaf(K02, A02, fmaf(K01, A01, A00));
                            const int pb = (i >> 1) * kPairCross + (i & 1);
                            const float x01 = tx[pb], x02 = tx[pb + 2], x12 = tx[pb + 4];
                            float num = fmaf(A00, u[0] * u[0], fmaf(A11, u[1] * u[1], A22 * (u[2] * u[2])));
                            const float off = fmaf(A01 * x01, u[0] * u[1], fmaf(A02 * x02, u[0] * u[2], A12 * x12 * (u[1] * u[2])));
                            num = fmaf(2.f, off, num);
                            const float prod = det * Cc[0] * Cc[1] * Cc[2];
                            float lg;
                            if (prod > 1e-36f && prod < 1e36f)
                                lg = lg2_approx(prod);
                            else
                                lg = lg2_approx(det) + lg2_approx(Cc[0]) + lg2_approx(Cc[1]) + lg2_approx(Cc[2]);
                            term = nu * (fmaf(num, rcp_approx(det), -3.f) + (float)kLn2 * lg);
                            careful |= !(fabsf(term) < 1e30f) || !(det > 0.f);
                        }
                    }
                    if (careful) {
                        // spline values in float-float from the records (hi + lo parts) and the
                        // FP64 term; its -3 nu goes to the FP64 spill-over like the term itself
                        const double xd = (double)x + (double)__ldg(xlo32 + w.bin0 + i);
                        double pd[NSP];
#pragma unroll
                        for (int a = 0; a < NSP; ++a) {
                            const float* rr = rec(a, s_jj[a][tid]);
                            const float4 A = __ldg(reinterpret_cast<const float4*>(rr));
                            const float4 B = __ldg(reinterpret_cast<const float4*>(rr) + 1);
                            const float4 Cq = __ldg(reinterpret_cast<const float4*>(rr) + 2);
                            const float4 Dq = __ldg(reinterpret_cast<const float4*>(rr) + 3);
                            const ff t = ff_add(ff{(float)xd, (float)(xd - (double)(float)xd)}, ff{-A.y, -Cq.x});
                            ff v = {B.y, Dq.x};
                            v = ff_add(ff_mul(v, t), ff{B.x, Cq.w});
                            v = ff_add(ff_mul(v, t), ff{A.w, Cq.z});
                            v = ff_add(ff_mul(v, t), ff{A.z, Cq.y});
                            pd[a] = ((double)v.hi + (double)v.lo) * (1.0 / kLog2_10);   // log10 units
                        }
                        double qd[kRec];
                        qd[1] = (double)ell + (double)__ldg(elllo32 + w.bin0 + i);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            qd[3 + c] = fld(tb, i, 3 + c);
                            qd[6 + c] = fld(tb, i, 6 + c);
                            qd[9 + c] = fld(tb, i, 9 + c);
                        }
                        const int pb = (i >> 1) * kPairCross + (i & 1);
                        const double xcd[3] = {tx[pb], tx[pb + 2], tx[pb + 4]};
                        const double sl = BROKEN ? (qd[1] < 0.0 ? th[3] : th[4]) : th[3];
                        const double pn[3] = {pd[0], pd[1], pd[2]};
                        const double zv[3] = {pd[ZB], pd[ZB + 1], pd[ZB + 2]};
                        const double t64 = full_term64<HAS_H>(pn, HAS_H ? pd[3] : 0.0, zv, qd, xcd, th[0] * th[0],
                                                              th[1] * th[1], th[2], sl);
                        if (nu != 0.f) far += (double)nu * (t64 - 3.0);
                        term = 0.f;
                    }
                    acc += term;
                    if (++run == 32) {
                        accf = ff_add(accf, ff{acc, 0.f});
                        acc = 0.f;
                        run = 0;
                    }
                }
                accf = ff_add(accf, ff{acc, 0.f});
            }
        }
        red[tid] = ((double)accf.hi + (double)accf.lo) + far;
        __syncthreads();
        if (r == 0 && active) {
            double sum = red[ls];
            for (int q = 1; q < R; ++q) sum += red[ls + q * sc];
            const DatasetDev& D = ds[w.ds];
            partial[D.pbase + (int64_t)(s - D.s0) * D.ntiles + w.tile] = sum;
        }
        __syncthreads();   // the buffer read in this iteration is refilled in the next one
    }
}

template <bool H, bool B>
cudaError_t launch_full(const lisa_data* d, bool fp32, const double* theta, const StateParams* prm,
                        const int32_t* sstat, const int32_t* nint, const float* kxr, const void* srec, int kmax,
                        double* partial, int* err, cudaStream_t sm) {
    if (fp32) {
        auto kern = full_fp32_kernel<H, B>;
        const size_t stage = (size_t)d->tiling.tile_bins * kRec * sizeof(float) +
                             (size_t)(d->tiling.tile_bins >> 1) * kPairCross * sizeof(float);
        const size_t smem = 2 * stage;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFullThreads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        int64_t grid = (int64_t)d->n_sm * per_sm;
        if (grid > d->n_items) grid = d->n_items;
        kern<<<(unsigned)(grid < 1 ? 1 : grid), kFullThreads, smem, sm>>>(
            d->d_items, (int)d->n_items, d->d_rec32, d->d_cross32, d->d_xlo32, d->d_elllo32, prm, theta, sstat, kxr,
            static_cast<const float*>(srec), kmax, d->nsp, d->d_ds, partial, err, d->tiling.tile_bins, d->wait_limit);
        return cudaGetLastError();
    }
    auto kern = full_fp64_kernel<H, B>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)d->n_sm * per_sm;
    if (grid > d->n_items) grid = d->n_items;
    kern<<<(unsigned)(grid < 1 ? 1 : grid), kThreads, 0, sm>>>(d->d_items, (int)d->n_items, d->d_rec64,
                                                                d->d_cross64, theta, sstat, nint,
                                                                static_cast<const double*>(srec), kmax, d->nsp,
                                                                d->d_ds, partial);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_full_cov(const lisa_data* d, bool fp32, const double* theta, const StateParams* prm,
                            const int32_t* sstat, const int32_t* nint, const float* kxr, const void* srec, int kmax,
                            double* partial, int* err, cudaStream_t sm) {
    if (d->sgwb_model == 0)
        return launch_full<false, false>(d, fp32, theta, prm, sstat, nint, kxr, srec, kmax, partial, err, sm);
    if (d->sgwb_model == 1)
        return launch_full<true, false>(d, fp32, theta, prm, sstat, nint, kxr, srec, kmax, partial, err, sm);
    return launch_full<true, true>(d, fp32, theta, prm, sstat, nint, kxr, srec, kmax, partial, err, sm);
}

}  // namespace lisa
