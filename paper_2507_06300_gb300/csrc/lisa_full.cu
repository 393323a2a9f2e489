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
        const WorkItem w = items[LISA_IDX(it, n_items)];
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
                    const double* z = base[a] + (size_t)LISA_IDX(j[a], kmax + 1) * kSplineRec;
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
                            const double* z = base[a] + (size_t)LISA_IDX(j[a], kmax + 1) * kSplineRec;
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

constexpr float kFullLo = 9.094947e-13f;   // 2^-40: FP32 path, D_c above and C_cc below 2^+-40
constexpr float kFullHi = 1.0995116e12f;   // 2^40
constexpr float kFullMinDet = 0.0625f;     // FP32 path: det K at least 1/16

constexpr int kFullChunk = 16;   // bins per thread between two passes over the careful queue

// The FP64 term of one careful bin (queued by the bin loop): the state's intervals at the bin are
// found again in the right-end table, the spline values formed in float-float from the records'
// hi + lo parts, and the term evaluated by full_term64, the same code as the plain path.
template <bool HAS_H, bool BROKEN>
__device__ __noinline__ double full_careful_term(int s, int bin, const float* tb, const float* tx, int i,
                                                 const float* __restrict__ xlo32, const float* __restrict__ elllo32,
                                                 const double* __restrict__ theta, const float* __restrict__ kxr,
                                                 const float* __restrict__ srec, int kmax, int nsp) {
    constexpr int NSP = 3 + (HAS_H ? 1 : 0) + 3;
    constexpr int ZB = 3 + (HAS_H ? 1 : 0);
    const float x = fld(tb, i, 0);
    const int kxs = kxr_stride(kmax);
    double pd[NSP];
#pragma unroll 1
    for (int a = 0; a < NSP; ++a) {
        const int64_t sp = (int64_t)s * nsp + a;
        const float4* kq = reinterpret_cast<const float4*>(kxr + sp * kxs);
        int j = 0;
        for (int q = 0; q < kxs / 4; ++q) {
            const float4 v = __ldg(kq + q);
            j += (v.x <= x) + (v.y <= x) + (v.z <= x) + (v.w <= x);
        }
        const float4* rr = reinterpret_cast<const float4*>(srec + (sp * (int64_t)(kmax + 1) + min(j, kmax)) *
                                                                      kSplineRec32);
        const float4 A = __ldg(rr), B = __ldg(rr + 1), Cq = __ldg(rr + 2), Dq = __ldg(rr + 3);
        const ff t = ff_add(ff{x, __ldg(xlo32 + bin)}, ff{-A.y, -Cq.x});
        ff v = {B.y, Dq.x};
        v = ff_add(ff_mul(v, t), ff{B.x, Cq.w});
        v = ff_add(ff_mul(v, t), ff{A.w, Cq.z});
        v = ff_add(ff_mul(v, t), ff{A.z, Cq.y});
        pd[a] = ((double)v.hi + (double)v.lo) * (1.0 / kLog2_10);   // log10 units
    }
    double qd[kRec];
    qd[1] = (double)fld(tb, i, 1) + (double)__ldg(elllo32 + bin);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        qd[3 + c] = fld(tb, i, 3 + c);
        qd[6 + c] = fld(tb, i, 6 + c);
        qd[9 + c] = fld(tb, i, 9 + c);
    }
    const int pb = (i >> 1) * kPairCross + (i & 1);
    const double xcd[3] = {tx[pb], tx[pb + 2], tx[pb + 4]};
    const double* th = theta + (size_t)s * LISA_N_THETA;
    const double sl = BROKEN ? (qd[1] < 0.0 ? th[3] : th[4]) : th[3];
    const double pn[3] = {pd[0], pd[1], pd[2]};
    const double zv[3] = {pd[ZB], pd[ZB + 1], pd[ZB + 2]};
    return full_term64<HAS_H>(pn, HAS_H ? pd[3] : 0.0, zv, qd, xcd, th[0] * th[0], th[1] * th[1], th[2], sl);
}

// One thread per state and contiguous bins of the item, one bin at a time.  The current interval of
// each spline (cubic about its midpoint, log2 units, as the setup writes FP32 records) is kept in
// registers, its right end and index in shared memory.  On an ill-conditioned interval (prior
// draws with close knots) the spline value is formed in float-float from the record's low parts
// and 2^P as ex2(hi) (1 + lo ln2); the rest of the bin stays in FP32.  The 3x3 algebra is written
// in the factored parameters (g_c^2 = D_c / C_cc, h_c = H_c / C_cc and the correlations' r, s), so
// that det K and the adjugate's diagonal are sums of non-negative products, accurate to a few
// rounding errors whatever the conditioning.  A bin whose diagonal entries leave 2^+-40, whose
// det K is below 1/16 or whose trace cancels by more than a factor 8 ("careful" bins: extreme
// states, rare) is queued in shared memory instead; after every chunk of kFullChunk bins the warp
// evaluates its queued bins in FP64, one bin per lane, so that they cost full lanes rather than a
// divergent branch in the bin loop (and no CTA barrier: the warps of a CTA drift freely within an
// item).  Each warp's queue holds a chunk's worth of bins of its 32 threads and cannot overflow.
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
    __shared__ double s_far[kFullThreads];                 // FP64 sums of the queued bins, per thread
    __shared__ uint32_t s_q[kFullThreads / 32][32 * kFullChunk];   // per-warp careful queue: thread << 16 | bin
    __shared__ int s_nq[kFullThreads / 32];
    __shared__ int s_fail;   // a bounded wait ran out: stage nothing more (a late copy may still land)
    const int tid = threadIdx.x;
    const int wid = tid >> 5, lane = tid & 31;
    const size_t stage_floats = (size_t)tile_bins * kRec + (size_t)(tile_bins >> 1) * kPairCross;
    float* sb[2] = {reinterpret_cast<float*>(smem), reinterpret_cast<float*>(smem) + stage_floats};
    if (tid == 0) {
        s_fail = 0;
        for (int q = 0; q < kFullThreads / 32; ++q) s_nq[q] = 0;
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
        const WorkItem w = items[LISA_IDX(it, n_items)];
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
        const int lo = (r * w.nb) / R, hi = ((r + 1) * w.nb) / R;
        const bool run_bins = active && lo < hi;
        const int nch = ((w.nb + R - 1) / R + kFullChunk - 1) / kFullChunk;   // uniform over the CTA
        s_far[tid] = 0.0;
        ff accf = {0.f, 0.f};
        const StateParams p = prm[run_bins ? s : w.s0];
        const float ao2 = p.ao2, at2 = p.at2, Af = HAS_H ? p.Af : 0.f;
        auto rec = [&](int a, int j) {
            return srec + (((int64_t)s * nsp + a) * (int64_t)(kmax + 1) + LISA_IDX(j, kmax + 1)) * kSplineRec32;
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
        float xmin = 0.f;
        if (run_bins) {
            // intervals at the first bin: the count of right ends <= x in the right-end table
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
            xmin = s_xr[0][tid];
#pragma unroll
            for (int a = 1; a < NSP; ++a) xmin = fminf(xmin, s_xr[a][tid]);
        }
        int* nq = &s_nq[wid];
        for (int ch = 0; ch < nch; ++ch) {
            if (run_bins) {
                float acc = 0.f;
                const int iend = min(hi, lo + (ch + 1) * kFullChunk);
                for (int i = lo + ch * kFullChunk; i < iend; ++i) {
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
                    // the SGWB exponent sl ell + p_h (log2 A is in Af) and, per exponential, a
                    // correction factor 1 + lo ln2 for an exponent known as hi + lo
                    const float sl = BROKEN ? (ell < 0.f ? p.n1 : p.n2) : p.n1;
                    float exh = HAS_H ? fmaf(sl, ell, pv[3]) : 0.f;
                    float ah = Af;
                    float corr[3] = {1.f, 1.f, 1.f}, corrh = 1.f;
                    if (hm) {
                        // an ill-conditioned interval (prior draws with close knots, rare and
                        // divergent): its spline value in float-float from the record's low parts,
                        // and the exponent as an exact hi + lo pair
                        const ff xf = {x, __ldg(xlo32 + w.bin0 + i)};
#pragma unroll
                        for (int a = 0; a < NSP; ++a) {
                            if (!((hm >> a) & 1u)) continue;
                            const float4* rr = reinterpret_cast<const float4*>(rec(a, s_jj[a][tid]));
                            const float4 A = __ldg(rr), B = __ldg(rr + 1), Cq = __ldg(rr + 2), Dq = __ldg(rr + 3);
                            const ff t = ff_add(xf, ff{-A.y, -Cq.x});
                            ff v = {B.y, Dq.x};
                            v = ff_add(ff_mul(v, t), ff{B.x, Cq.w});
                            v = ff_add(ff_mul(v, t), ff{A.w, Cq.z});
                            v = ff_add(ff_mul(v, t), ff{A.z, Cq.y});
                            if (a < 3) {
                                pv[a] = v.hi;
                                corr[a] = fmaf(v.lo, (float)kLn2, 1.f);
                            } else if (HAS_H && a == 3) {
                                const ff sf = BROKEN ? (ell < 0.f ? ff{p.n1, p.n1_lo} : ff{p.n2, p.n2_lo})
                                                     : ff{p.n1, p.n1_lo};
                                const ff ef = {ell, __ldg(elllo32 + w.bin0 + i)};
                                const ff eh = ff_add(ff_add(v, ff_mul(sf, ef)), ff{p.lA_hi, p.lA_lo});
                                exh = eh.hi;
                                corrh = fmaf(eh.lo, (float)kLn2, 1.f);
                                ah = 1.f;               // log2 A is in the exponent
                            } else {
                                pv[a] = v.hi + v.lo;    // a correlation value: plain
                            }
                        }
                    }
                    bool careful = false;
                    float term = 0.f;
                    {
                        float D[3], H[3], Cc[3];
                        const float eh = HAS_H ? ah * ex2_approx(exh) * corrh : 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            D[c] = fmaf(ao2, fld(tb, i, 3 + c), at2 * fld(tb, i, 6 + c)) * (ex2_approx(pv[c]) * corr[c]);
                            H[c] = HAS_H ? eh * fld(tb, i, 9 + c) : 0.f;
                            Cc[c] = HAS_H ? D[c] + H[c] : D[c];
                            // within 2^+-40 every product below stays a normal FP32 number; NaN fails
                            careful |= !(D[c] > kFullLo) || !(Cc[c] < kFullHi);
                        }
                        if (!careful) {
                            // w_c = 1 / C_cc, g_c^2 = D_c / C_cc, h_c = H_c / C_cc (g^2 + h = 1)
                            const float Cp = Cc[0] * Cc[1] * Cc[2];
                            const float W = rcp_approx(Cp);
                            const float w[3] = {W * (Cc[1] * Cc[2]), W * (Cc[0] * Cc[2]), W * (Cc[0] * Cc[1])};
                            float g2[3], h[3];
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                g2[c] = D[c] * w[c];
                                h[c] = HAS_H ? H[c] * w[c] : 0.f;
                            }
                            // r = z / sqrt(1 + z^2), s = 1 / sqrt(1 + z^2) (z in log2(10) units)
                            float rr[3], ss[3];
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const float zq = pv[ZB + q];
                                const float iq = rsqrtf(fmaf(zq, zq, kL2 * kL2));
                                rr[q] = zq * iq;
                                ss[q] = kL2 * iq;
                            }
                            // K = G R G + diag(h) with R = L L^T; the adjugate's diagonal and det K
                            // as sums of non-negative products (no cancellation at any conditioning):
                            // 1 - R01^2 = s0^2, 1 - R02^2 = s1^2, 1 - R12^2 = (s1 s2)^2 + e^2,
                            // det R = (s0 s1 s2)^2
                            const float R12 = fmaf(rr[0], rr[1], ss[0] * ss[1] * rr[2]);
                            const float e = fmaf(rr[0] * rr[2], ss[1], -rr[1] * ss[0]);
                            const float s12 = ss[1] * ss[2];
                            const float m01 = ss[0] * ss[0], m02 = ss[1] * ss[1], m12 = fmaf(s12, s12, e * e);
                            const float sR = ss[0] * s12;
                            float A00, A11, A22, det;
                            if (HAS_H) {
                                A00 = fmaf(g2[1] * g2[2], m12, fmaf(h[1], h[2] + g2[2], h[2] * g2[1]));
                                A11 = fmaf(g2[0] * g2[2], m02, fmaf(h[0], h[2] + g2[2], h[2] * g2[0]));
                                A22 = fmaf(g2[0] * g2[1], m01, fmaf(h[0], h[1] + g2[1], h[1] * g2[0]));
                                const float in = fmaf(g2[1] * g2[2], sR * sR,
                                                      fmaf(h[1], fmaf(g2[2], m02, h[2]), h[2] * g2[1] * m01));
                                det = fmaf(h[0], A00, g2[0] * in);
                            } else {
                                A00 = g2[1] * g2[2] * m12;
                                A11 = g2[0] * g2[2] * m02;
                                A22 = g2[0] * g2[1] * m01;
                                det = g2[0] * g2[1] * g2[2] * (sR * sR);
                            }
                            // off-diagonal adjugate entries times Q_ab = P-hat_ab / sqrt(C_aa C_bb):
                            //   A01 = g0 g1 [s1 (r1 r2 s0 - r0 s1) - h2 r1 R12],
                            //   A02 = g0 g2 [s0 e - h1 r0 R12],  A12 = -g1 g2 [s0 s1 r2 + h0 r0 r1],
                            // with g_a g_b Q_ab = sqrt(D_a D_b) w_a w_b P-hat_ab
                            const int pb = (i >> 1) * kPairCross + (i & 1);
                            const float x01 = tx[pb], x02 = tx[pb + 2], x12 = tx[pb + 4];
                            float b01 = ss[1] * fmaf(rr[1] * rr[2], ss[0], -rr[0] * ss[1]);
                            float b02 = ss[0] * e;
                            float b12 = ss[0] * ss[1] * rr[2];
                            if (HAS_H) {
                                b01 = fmaf(-h[2] * rr[1], R12, b01);
                                b02 = fmaf(-h[1] * rr[0], R12, b02);
                                b12 = fmaf(h[0] * rr[0], rr[1], b12);
                            }
                            const float p01 = D[0] * D[1], p02 = D[0] * D[2], p12 = D[1] * D[2];
                            const float o01 = b01 * x01 * (p01 * rsqrtf(p01)) * (w[0] * w[1]);
                            const float o02 = b02 * x02 * (p02 * rsqrtf(p02)) * (w[0] * w[2]);
                            const float o12 = b12 * x12 * (p12 * rsqrtf(p12)) * (w[1] * w[2]);
                            const float dg = fmaf(A00, w[0], fmaf(A11, w[1], A22 * w[2]));
                            const float num = fmaf(2.f, o01 + o02 - o12, dg);
                            // rounding in the trace grows with its cancellation S / num and with
                            // 1 / det K: beyond these limits (rare) the bin takes the FP64 term
                            const float S = fmaf(2.f, fabsf(o01) + fabsf(o02) + fabsf(o12), dg);
                            careful |= !(det > kFullMinDet) || !(S <= 8.f * fmaxf(num, 3.f * det));
                            // ln det C from one log2 of det K times the product of the C_cc; a warp
                            // vote keeps the two-log form (a product under 1e-36) a real branch
                            const float prod = det * Cp;
                            const bool prod_ok = prod > 1e-36f;
                            float lg;
                            if (__all_sync(__activemask(), prod_ok) || prod_ok)
                                lg = lg2_approx(prod);
                            else
                                lg = lg2_approx(det) + lg2_approx(Cp);
                            term = nu * (fmaf(num, rcp_approx(det), -3.f) + (float)kLn2 * lg);
                            careful |= !(fabsf(term) < 1e30f);
                        }
                    }
                    if (careful) {
                        const int q = atomicAdd(nq, 1);   // < 32 * kFullChunk
                        s_q[wid][q] = ((uint32_t)tid << 16) | (uint32_t)i;
                        term = 0.f;
                    }
                    acc += term;
                }
                accf = ff_add(accf, ff{acc, 0.f});
            }
            // the warp's careful bins of this chunk, one per lane (the warp's lanes share the chunk
            // loop; only this warp's threads own them)
            // (lane 0 reads the count after every lane's appends and broadcasts it: no lane can
            // append for the next chunk before the shuffle, so the count is the same for all)
            __syncwarp();
            const int nqv = __shfl_sync(0xffffffffu, lane == 0 ? *reinterpret_cast<volatile int*>(nq) : 0, 0);
            if (nqv == 0) continue;
            for (int e = lane; e < nqv; e += 32) {
                const uint32_t ent = s_q[wid][e];
                const int owner = (int)(ent >> 16), i = (int)(ent & 0xffffu);
                const int so = w.s0 + (owner & (sc - 1));
                const float nu = fld(tb, i, 2);
                const double t64 = full_careful_term<HAS_H, BROKEN>(so, w.bin0 + i, tb, tx, i, xlo32, elllo32, theta,
                                                                    kxr, srec, kmax, nsp);
                if (nu != 0.f) atomicAdd(&s_far[owner], (double)nu * (t64 - 3.0));
            }
            __syncwarp();
            if (lane == 0) *nq = 0;
            __syncwarp();
        }
        red[tid] = ((double)accf.hi + (double)accf.lo) + s_far[tid];
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

LISA_DEBUG_TU(full)
