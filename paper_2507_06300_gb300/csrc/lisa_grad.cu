// Adjoint of the fused likelihood: log L and d log L / d(theta, knot amplitudes, knot positions)
// for every state.
//
// With S-hat = S / P (the tables are normalised by the periodogram) the per-bin term is
// nu (1/S + ln S) up to constants, so d log L / d S_c = nu (1 - S_c) / S_c^2 =: g_c.  Then, per
// state,
//   d/d a_oms  = 2 a_oms sum_i sum_c g_c G_oms,c E_c          E_c = 10^{P_n,c}
//   d/d a_tm   = 2 a_tm  sum_i sum_c g_c G_tm,c  E_c
//   d/d log10A = ln10 sum_i H_i,      H_i = sum_c g_c E_h G_h,c    (E_h = A (f/f_ref)^n 10^{P_h})
//   d/d n      = ln2  sum_i ell_i H_i (split at f_ref for the broken power law)
// and each spline receives the adjoint signal q(x_i) = d log L / d P(x_i):
//   noise spline c: q = ln10 g_c N_c E_c,   SGWB spline: q = ln10 H_i.
// Because P(x) = a_j + b_j t + c_j t^2 + d_j t^3 (t = x - x_j) on interval j, the gradient
// with respect to that interval's coefficients is the moment vector M_p = sum_{i in j} q_i t_i^p
// (p = 0..3), and the knot position x_j moves t as well: dL/dx_j|direct = -(b M0 + 2c M1 + 3d M2).
// The kernels below recompute the forward pass per bin (nothing per bin is stored), accumulate
// the template sums and the per-interval moments, and an epilogue rebuilds each spline from its
// knots and pushes the moments back through the spline construction (Akima slopes, natural
// cubic system, or linear fallback) to the knot amplitudes and positions.
//
// FP32 mode accumulates the moments about each interval's midpoint x_o (the variable of its
// Horner evaluation, |x - x_o| <= h/2), which keeps the FP32 partial sums small; the epilogue
// converts them exactly (FP64 binomial expansion) to moments about the left knot.
//
// Determinism: a range rho of kAdjBins bins writes the moments of every interval j it touches
// to slot rho + j of its (state, spline) row; the intervals a range touches are monotone in rho,
// so slots never collide, and the epilogue adds them back in a fixed order.
#include "lisa_math.cuh"
#include "lisa_spline_dev.cuh"
#include <type_traits>

namespace lisa {

// Gradient workspace (after 256 bytes): range sums scal | moment slots mom, and for the FP32
// call a flag per state (states whose FP32 sums leave the FP32 range, redone within the call).
struct GradLayout {
    size_t off_scal, off_mom, off_fb, bytes;
};
inline GradLayout grad_layout(const lisa_data* d, int kmax, bool fp32) {
    GradLayout G;
    G.off_scal = 0;
    G.off_mom = align256(sizeof(double) * 6 * (size_t)d->adj_ranges);
    G.off_fb = G.off_mom + align256(sizeof(double) * 4 * (size_t)d->nsp *
                                    ((size_t)d->adj_ranges + (size_t)d->n_states * (size_t)(kmax + 1)));
    G.bytes = G.off_fb + (fp32 ? align256(sizeof(int32_t) * (2 * (size_t)d->n_states + 3)) : 0);
    return G;
}

size_t grad_extra_bytes(const lisa_data* d, int kmax, bool fp32) { return grad_layout(d, kmax, fp32).bytes; }

namespace {
using namespace dm;

constexpr unsigned kFullMask = 0xffffffffu;

// Moment row of (state, spline): 4 doubles per slot, nranges + kmax + 1 slots.
__device__ __forceinline__ double* mom_row(double* mom, int64_t prefix, int s, int a, int nsp, int kmax, int nr) {
    return mom + 4 * ((int64_t)nsp * (prefix + (int64_t)s * (kmax + 1)) + (int64_t)a * (nr + kmax + 1));
}

// The FP32 gradient's flag area fb (int32, zeroed per call): fb[0..S) a flag per state, fb[S]
// the count and fb[S+1..2S] the flagged states (in the order they were flagged), then the item
// counters of the compensated (fb[2S+1]) and fallback (fb[2S+2]) passes.  Flags state s (sums or
// moments beyond the FP32 range) once.
__device__ __forceinline__ void fb_flag(int32_t* fb, int S, int s) {
    if (atomicExch(fb + s, 1) == 0) fb[S + 1 + atomicAdd(fb + S, 1)] = s;
}

// ---- FP32 adjoint: one warp per (dataset, range, up to 32 states) -----------------------------
// The current interval of a spline: right end and index, and -x_o, -x_o's low part and the cubic's
// coefficients duplicated in register pairs for the packed (two bins per instruction) path.
struct AdjIv {
    float xr;
    int j;
    float2 nxo, nxo_lo, c0, c1, c2, c3;
};

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// asynchronous global -> shared copies of one thread (completion by cp.async.wait_group)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kAdjStagePairs = 16;   // pair blocks per staged chunk of the adjoint's table

// EXACT_T: every bin lies inside the knot band and the band satisfies |x_lo| <= 2.9 |x_hi| (same
// sign), so that within any interval |x - x_o| <= 2 |x| and |x_o| <= 2 |x| and the FP32 difference
// x - x_o is exact (Sterbenz); t then needs no two-sum (the same value as the compensated form).
//
// Per bin the forward pass is recomputed and g_c / nu = r (r - 1), r = 1 / S-hat_c, drives the
// template sums and each spline's signal q (the derivative of log L by the spline value; ln10 is
// applied when the moments are stored).  Bins are taken two at a time from the pair-block table,
// whose fields of both bins load as register pairs: a pair whose bins share every spline's
// interval runs on the packed FP32x2 instructions, a pair with a knot between its bins runs as
// two scalar bins.  Chunk sums are kept per lane of the pair (float2) and go to the float-float
// running sums (shared memory) as exact two-sums every 128 bins and at interval ends.
template <int C, bool HAS_H, bool BROKEN, bool EXACT_T>
__global__ void __launch_bounds__(128, 3)
    adjoint_fp32_kernel(const AdjUnit* __restrict__ units, int64_t n_units, const DatasetDev* __restrict__ ds,
                        const float* __restrict__ rec32, const float* __restrict__ xlo32,
                        const double* __restrict__ theta, const int32_t* __restrict__ sstat,
                        const int32_t* __restrict__ nint, const float* __restrict__ srec, int kmax, int nsp,
                        const int64_t* __restrict__ prefix, double* __restrict__ scal, double* __restrict__ mom,
                        int S, int32_t* __restrict__ fb) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    __shared__ float2 s_am[NSP * 4][128];
    __shared__ float2 s_as[6][128];
    // per warp, two staged chunks of the table and of the low parts of x
    __shared__ __align__(16) float s_tab[4][2][kAdjStagePairs * kPairRec];
    __shared__ __align__(16) float2 s_xl[4][2][kAdjStagePairs];
    const int tid = threadIdx.x;
    const int wid = tid >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float2 m1 = dup2(-1.f);
    for (int64_t u = wg; u < n_units; u += nw) {
        const AdjUnit U = units[u];
        const DatasetDev& D = ds[U.ds];
        const int s = U.s0 + lane;
        // the warp's active lanes (the chunk votes below run over them; the unit is warp-uniform)
        const unsigned amask = __ballot_sync(kFullMask, lane < U.ns && (sstat[lane < U.ns ? s : U.s0] & kUserBits) == 0);
        if (!((amask >> lane) & 1u)) continue;
        const double* th = theta + (size_t)s * LISA_N_THETA;
        const float ao2 = (float)(th[0] * th[0]), at2 = (float)(th[1] * th[1]);
        const float Af = HAS_H ? (float)exp10(th[2]) : 0.f;
        const float n1 = (float)th[3], n2 = BROKEN ? (float)th[4] : n1;
        const int64_t b0 = D.bin0 + (int64_t)U.rho * kAdjBins;        // even
        const int nb = (int)min((int64_t)kAdjBins, D.bin0 + D.npad - b0);
        const float* tb = rec32 + (b0 >> 1) * kPairRec;
        const int64_t pre = prefix[s];
        const int32_t* nint_s = nint + (int64_t)s * nsp;
        AdjIv iv[NSP] = {};
        unsigned hm = 0;   // splines whose current interval is ill-conditioned (T > kRobustT)
        bool bad = false;  // a sum beyond the FP32 range: the state goes to the fallback list
        auto base = [&](int a) { return srec + ((int64_t)s * nsp + a) * (int64_t)(kmax + 1) * kSplineRec32; };
        auto load = [&](int a) {
            const float* r = base(a) + (size_t)LISA_IDX(iv[a].j, kmax + 1) * kSplineRec32;
            iv[a].xr = __ldg(r + 0);
            iv[a].nxo = dup2(-__ldg(r + 1));
            iv[a].nxo_lo = dup2(-__ldg(r + 8));
            if (__ldg(r + 7) <= (float)kRobustT) {
                iv[a].c0 = dup2(__ldg(r + 2));
                iv[a].c1 = dup2(__ldg(r + 3));
                iv[a].c2 = dup2(__ldg(r + 4));
                iv[a].c3 = dup2(__ldg(r + 5));
                hm &= ~(1u << a);
            } else {
                // ill-conditioned (routed states): the zero cubic keeps the arithmetic benign, and
                // the thread's bins are masked (nu = 0) while it holds such an interval; the
                // compensated adjoint adds them
                iv[a].c0 = iv[a].c1 = iv[a].c2 = iv[a].c3 = make_float2(0.f, 0.f);
                hm |= 1u << a;
            }
        };
        {
            const float x0 = fld(tb, 0, 0);
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                iv[a].j = find_interval<float, kSplineRec32, 6>(base(a), nint_s[a], x0);
                load(a);
            }
        }
        // accumulators: chunk sums per lane of the bin pair (registers), running sums in
        // float-float (shared)
        float2 cm[NSP][4];
        float2 cs[6];
#pragma unroll
        for (int a = 0; a < NSP; ++a)
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                cm[a][p] = make_float2(0.f, 0.f);
                s_am[4 * a + p][tid] = make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            cs[k] = make_float2(0.f, 0.f);
            s_as[k][tid] = make_float2(0.f, 0.f);
        }
        auto add_run = [&](float2* slot, float2 c) {
            const float2 v = *slot;
            const ff r = ff_add(ff{v.x, v.y}, two_sum(c.x, c.y));
            *slot = make_float2(r.hi, r.lo);
        };
        auto flush_mom = [&](int a) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                add_run(&s_am[4 * a + p][tid], cm[a][p]);
                cm[a][p] = make_float2(0.f, 0.f);
            }
        };
        auto store_mom = [&](int a) {
            flush_mom(a);
            double* row = mom_row(mom, pre, s, a, nsp, kmax, D.nranges) + 4 * (int64_t)LISA_IDX(U.rho + iv[a].j, D.nranges + kmax + 1);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float2 v = s_am[4 * a + p][tid];
                row[p] = kLn10 * ((double)v.x + (double)v.y);   // q carries ln10 only here
                bad |= !isfinite(v.x);
                s_am[4 * a + p][tid] = make_float2(0.f, 0.f);
            }
        };
        auto flush_all = [&]() {
#pragma unroll
            for (int a = 0; a < NSP; ++a) flush_mom(a);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                add_run(&s_as[k][tid], cs[k]);
                cs[k] = make_float2(0.f, 0.f);
            }
        };
        auto advance = [&](int a, float x) {
            while (x >= iv[a].xr && iv[a].j < __ldg(nint_s + a) - 1) {
                store_mom(a);
                ++iv[a].j;
                load(a);
            }
        };
        // one scalar bin (the fields f[0..11] of the table: x, ell, nu, G_oms, G_tm, G_h, and the
        // low part of x), its sums in the first lane of the pair accumulators; the intervals
        // must already hold the bin
        auto bin = [&](const float* f, float x_lo) {
            const float x = f[0], ell = f[1], nu = hm ? 0.f : f[2];
            float P[NSP], tl[NSP];
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                float t;
                if (EXACT_T) {
                    t = (x + iv[a].nxo.x) + (x_lo + iv[a].nxo_lo.x);
                } else {
                    const ff tt = two_sum(x, iv[a].nxo.x);
                    t = tt.hi + (tt.lo + (x_lo + iv[a].nxo_lo.x));
                }
                P[a] = fmaf(fmaf(fmaf(iv[a].c3.x, t, iv[a].c2.x), t, iv[a].c1.x), t, iv[a].c0.x);
                tl[a] = t;
            }
            float eh = 0.f;
            if (HAS_H) {
                const float sl = BROKEN ? (ell < 0.f ? n1 : n2) : n1;
                eh = Af * ex2_approx(fmaf(sl, ell, P[C]));
            }
            float fwd = -(float)C, To = 0.f, Tt = 0.f, Hs = 0.f, prod = 1.f;
            float qn[C], S[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float go = f[3 + c], gt = f[6 + c];
                const float E = ex2_approx(P[c]);
                const float N = fmaf(ao2, go, at2 * gt);
                const float Eh = HAS_H ? eh * f[9 + c] : 0.f;
                const float Sc = HAS_H ? fmaf(E, N, Eh) : E * N;
                const float r = rcp_approx(Sc);
                const float gp = fmaf(r, r, -r);
                const float gE = gp * E;
                fwd += r;
                prod = c == 0 ? Sc : prod * Sc;
                S[c] = Sc;
                To = c == 0 ? gE * go : fmaf(gE, go, To);
                Tt = c == 0 ? gE * gt : fmaf(gE, gt, Tt);
                if (HAS_H) Hs = c == 0 ? gp * Eh : fmaf(gp, Eh, Hs);
                qn[c] = gE * N;
            }
            if (prod > 1e-30f && prod < 1e30f) {
                fwd = fmaf((float)kLn2, lg2_approx(prod), fwd);
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) fwd = fmaf((float)kLn2, lg2_approx(S[c]), fwd);
            }
            cs[0].x = fmaf(nu, fwd, cs[0].x);
            cs[1].x = fmaf(nu, To, cs[1].x);
            cs[2].x = fmaf(nu, Tt, cs[2].x);
            float q[NSP];
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] = nu * qn[c];
            if (HAS_H) {
                const float Hb = nu * Hs;
                cs[3].x += Hb;
                if (BROKEN && ell >= 0.f)
                    cs[5].x = fmaf(ell, Hb, cs[5].x);
                else
                    cs[4].x = fmaf(ell, Hb, cs[4].x);
                q[C] = Hb;
            }
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                const float t = tl[a], qt = q[a] * t, qt2 = qt * t;
                cm[a][0].x += q[a];
                cm[a][1].x += qt;
                cm[a][2].x += qt2;
                cm[a][3].x = fmaf(qt2, t, cm[a][3].x);
            }
        };
        // two bins in the same intervals of every spline, on the packed FP32x2 instructions: the
        // table's fields of both bins F[0..11] and the low parts of their x
        auto pair = [&](const float2* F, float2 xl) {
            const float2 x = F[0], ell = F[1];
            const float2 nu = hm ? make_float2(0.f, 0.f) : F[2];   // bins of ill-conditioned intervals: masked
            float2 P[NSP], tl[NSP];
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                float2 t;
                if (EXACT_T) {
                    t = __fadd2_rn(__fadd2_rn(x, iv[a].nxo), __fadd2_rn(xl, iv[a].nxo_lo));
                } else {
                    // two-sum of x and -x_o per lane: s + e = x - x_o exactly
                    const float2 sm = __fadd2_rn(x, iv[a].nxo);
                    const float2 bb = __ffma2_rn(x, m1, sm);                       // s - x
                    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, sm), m1, x),
                                                __ffma2_rn(bb, m1, iv[a].nxo));     // (x - (s - b)) + (-x_o - b)
                    t = __fadd2_rn(sm, __fadd2_rn(e, __fadd2_rn(xl, iv[a].nxo_lo)));
                }
                P[a] = __ffma2_rn(__ffma2_rn(__ffma2_rn(iv[a].c3, t, iv[a].c2), t, iv[a].c1), t, iv[a].c0);
                tl[a] = t;
            }
            float2 eh = make_float2(0.f, 0.f);
            if (HAS_H) {
                const float2 sl = BROKEN ? make_float2(ell.x < 0.f ? n1 : n2, ell.y < 0.f ? n1 : n2) : dup2(n1);
                const float2 ex = __ffma2_rn(sl, ell, P[C]);
                eh = __fmul2_rn(dup2(Af), make_float2(ex2_approx(ex.x), ex2_approx(ex.y)));
            }
            // with nr = -r: g / nu = r^2 - r = nr^2 + nr, and the forward sum collects nr
            float2 fwn, To, Tt, Hs, prod, qn[C], S[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float2 go = F[3 + c], gt = F[6 + c];
                const float2 E = make_float2(ex2_approx(P[c].x), ex2_approx(P[c].y));
                const float2 N = __ffma2_rn(dup2(ao2), go, __fmul2_rn(dup2(at2), gt));
                const float2 Eh = HAS_H ? __fmul2_rn(eh, F[9 + c]) : make_float2(0.f, 0.f);
                const float2 Sc = HAS_H ? __ffma2_rn(E, N, Eh) : __fmul2_rn(E, N);
                const float2 nr = make_float2(rcp_approx(-Sc.x), rcp_approx(-Sc.y));
                const float2 gp = __ffma2_rn(nr, nr, nr);
                const float2 gE = __fmul2_rn(gp, E);
                S[c] = Sc;
                if (c == 0) {
                    fwn = nr;
                    prod = Sc;
                    To = __fmul2_rn(gE, go);
                    Tt = __fmul2_rn(gE, gt);
                    if (HAS_H) Hs = __fmul2_rn(gp, Eh);
                } else {
                    fwn = __fadd2_rn(fwn, nr);
                    prod = __fmul2_rn(prod, Sc);
                    To = __ffma2_rn(gE, go, To);
                    Tt = __ffma2_rn(gE, gt, Tt);
                    if (HAS_H) Hs = __ffma2_rn(gp, Eh, Hs);
                }
                qn[c] = __fmul2_rn(gE, N);
            }
            // sum_c ln S_c from one log2 of each bin's channel product (per channel outside a safe
            // range, behind a warp vote so that the rare form stays a real branch)
            const bool pok = prod.x > 1e-30f && prod.x < 1e30f && prod.y > 1e-30f && prod.y < 1e30f;
            float2 lg;
            if (__all_sync(__activemask(), pok) || pok) {
                lg = make_float2(lg2_approx(prod.x), lg2_approx(prod.y));
            } else {
                lg = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    lg.x += lg2_approx(S[c].x);
                    lg.y += lg2_approx(S[c].y);
                }
            }
            // forward term: sum_c r + sum_c ln S_c - C
            const float2 fwd = __ffma2_rn(fwn, m1, __ffma2_rn(dup2((float)kLn2), lg, dup2(-(float)C)));
            cs[0] = __ffma2_rn(nu, fwd, cs[0]);
            cs[1] = __ffma2_rn(nu, To, cs[1]);
            cs[2] = __ffma2_rn(nu, Tt, cs[2]);
            float2 q[NSP];
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] = __fmul2_rn(nu, qn[c]);
            if (HAS_H) {
                const float2 Hb = __fmul2_rn(nu, Hs);
                cs[3] = __fadd2_rn(cs[3], Hb);
                if (BROKEN) {
                    // ell at and above the break to n2's sum, below it to n1's
                    const float2 e5 = make_float2(ell.x >= 0.f ? ell.x : 0.f, ell.y >= 0.f ? ell.y : 0.f);
                    const float2 e4 = make_float2(ell.x >= 0.f ? 0.f : ell.x, ell.y >= 0.f ? 0.f : ell.y);
                    cs[4] = __ffma2_rn(e4, Hb, cs[4]);
                    cs[5] = __ffma2_rn(e5, Hb, cs[5]);
                } else {
                    cs[4] = __ffma2_rn(ell, Hb, cs[4]);
                }
                q[C] = Hb;
            }
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                const float2 t = tl[a], qt = __fmul2_rn(q[a], t), qt2 = __fmul2_rn(qt, t);
                cm[a][0] = __fadd2_rn(cm[a][0], q[a]);
                cm[a][1] = __fadd2_rn(cm[a][1], qt);
                cm[a][2] = __fadd2_rn(cm[a][2], qt2);
                cm[a][3] = __ffma2_rn(qt2, t, cm[a][3]);
            }
        };
        // the range's bins two at a time, in chunks of kAdjStagePairs pair blocks that the warp's
        // active lanes stage into shared memory (cp.async, the next chunk in flight while the
        // current one is read): one vote over the lanes per chunk decides whether any spline of any
        // lane can pass a knot inside it (its last bin at or past an interval's right end);
        // knot-free chunks run packed without checks.  The chunk sums go to the running sums every
        // 128 bins.
        const float4* tb4 = reinterpret_cast<const float4*>(tb);
        const float2* xl2 = reinterpret_cast<const float2*>(xlo32 + b0);
        const int rank = __popc(amask & ((1u << lane) - 1u)), nact = __popc(amask);
        const int npair = nb >> 1;
        const int nch = (npair + kAdjStagePairs - 1) / kAdjStagePairs;
        auto stage = [&](int c) {
            const int q0 = c * kAdjStagePairs, nq = min(kAdjStagePairs, npair - q0);
            const float4* src = tb4 + (size_t)q0 * (kPairRec / 4);
            float4* dst = reinterpret_cast<float4*>(s_tab[wid][c & 1]);
            for (int k = rank; k < nq * (kPairRec / 4); k += nact) cp_async16(dst + k, src + k);
            for (int k = rank; k < nq; k += nact) cp_async8(&s_xl[wid][c & 1][k], xl2 + q0 + k);
            cp_async_commit();
        };
        stage(0);
        for (int c = 0; c < nch; ++c) {
            // chunk c + 1 goes into the buffer that chunk c - 1 used (released by the warp sync at
            // the end of the previous iteration)
            if (c + 1 < nch) {
                stage(c + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp(amask);
            const float* T = s_tab[wid][c & 1];
            const float2* XL = s_xl[wid][c & 1];
            const int np = min(kAdjStagePairs, npair - c * kAdjStagePairs);
            const float xlast = T[(np - 1) * kPairRec + 1];   // x of the chunk's last bin
            bool cross = false;
#pragma unroll
            for (int a = 0; a < NSP; ++a) cross |= !(xlast < iv[a].xr);
            if (__any_sync(amask, cross)) {
                for (int ip = 0; ip < np; ++ip) {
                    float4 q4[kPairRec / 4];
#pragma unroll
                    for (int k = 0; k < kPairRec / 4; ++k) q4[k] = reinterpret_cast<const float4*>(T)[ip * (kPairRec / 4) + k];
                    const float2 xl = XL[ip];
                    const float2* F = reinterpret_cast<const float2*>(q4);
                    bool split = false;
#pragma unroll
                    for (int a = 0; a < NSP; ++a) {
                        advance(a, F[0].x);
                        split |= !(F[0].y < iv[a].xr);
                    }
                    if (split) {
                        // a knot between the two bins: each on its own intervals
                        float f0[kRec], f1[kRec];
#pragma unroll
                        for (int k = 0; k < kRec; ++k) {
                            f0[k] = F[k].x;
                            f1[k] = F[k].y;
                        }
                        bin(f0, xl.x);
#pragma unroll
                        for (int a = 0; a < NSP; ++a) advance(a, f1[0]);
                        bin(f1, xl.y);
                    } else {
                        pair(F, xl);
                    }
                }
            } else {
                for (int ip = 0; ip < np; ++ip) {
                    float4 q4[kPairRec / 4];
#pragma unroll
                    for (int k = 0; k < kPairRec / 4; ++k) q4[k] = reinterpret_cast<const float4*>(T)[ip * (kPairRec / 4) + k];
                    pair(reinterpret_cast<const float2*>(q4), XL[ip]);
                }
            }
            if ((c & 3) == 3 || c + 1 == nch) flush_all();
            __syncwarp(amask);   // the buffer is restaged by the next iteration
        }
#pragma unroll
        for (int a = 0; a < NSP; ++a) store_mom(a);
        double* sc = scal + 6 * (pre + U.rho);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 v = s_as[k][tid];
            sc[k] = (double)v.x + (double)v.y;
            bad |= !isfinite(v.x);
        }
        if (bad) fb_flag(fb, S, s);
    }
}

// ---- FP64 adjoint (plain): same decomposition, FP64 throughout ---------------------------------
template <int C, bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(128)
    adjoint_fp64_kernel(const AdjUnit* __restrict__ units, int64_t n_units, const DatasetDev* __restrict__ ds,
                        const double* __restrict__ rec64, const double* __restrict__ theta,
                        const int32_t* __restrict__ sstat, const int32_t* __restrict__ nint,
                        const double* __restrict__ srec, int kmax, int nsp, const int64_t* __restrict__ prefix,
                        double* __restrict__ scal, double* __restrict__ mom) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = wg; u < n_units; u += nw) {
        const AdjUnit U = units[u];
        const DatasetDev& D = ds[U.ds];
        const int s = U.s0 + lane;
        // the warp's active lanes (the chunk votes below run over them; the unit is warp-uniform)
        const unsigned amask = __ballot_sync(kFullMask, lane < U.ns && (sstat[lane < U.ns ? s : U.s0] & kUserBits) == 0);
        if (!((amask >> lane) & 1u)) continue;
        const double* th = theta + (size_t)s * LISA_N_THETA;
        const double ao2 = th[0] * th[0], at2 = th[1] * th[1], lA = th[2], n1 = th[3];
        const double n2 = BROKEN ? th[4] : n1;
        const int64_t b0 = D.bin0 + (int64_t)U.rho * kAdjBins;
        const int nb = (int)min((int64_t)kAdjBins, D.bin0 + D.npad - b0);
        const int64_t pre = prefix[s];
        const double* base[NSP];
        int j[NSP], last[NSP];
        double xl[NSP], xr[NSP], ca[NSP], cb[NSP], cc[NSP], cd[NSP];
        double m[NSP][4];
        const double x0 = rec64[b0 * kRec];
        for (int a = 0; a < NSP; ++a) {
            const int64_t sp = (int64_t)s * nsp + a;
            base[a] = srec + sp * (int64_t)(kmax + 1) * kSplineRec;
            last[a] = nint[sp] - 1;
            j[a] = find_interval<double, kSplineRec, 0>(base[a], nint[sp], x0);
            const double* z = base[a] + (size_t)LISA_IDX(j[a], kmax + 1) * kSplineRec;
            xl[a] = z[0]; xr[a] = z[1]; ca[a] = z[2]; cb[a] = z[3]; cc[a] = z[4]; cd[a] = z[5];
            for (int p = 0; p < 4; ++p) m[a][p] = 0.0;
        }
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < nb; ++i) {
            const double* q = rec64 + (b0 + i) * kRec;
            const double x = q[0], ell = q[1], nu = q[2];
            double P[NSP], t[NSP];
            for (int a = 0; a < NSP; ++a) {
                while (x >= xr[a] && j[a] < last[a]) {
                    double* row = mom_row(mom, pre, s, a, nsp, kmax, D.nranges) + 4 * (int64_t)LISA_IDX(U.rho + j[a], D.nranges + kmax + 1);
                    for (int p = 0; p < 4; ++p) {
                        row[p] = m[a][p];
                        m[a][p] = 0.0;
                    }
                    ++j[a];
                    const double* z = base[a] + (size_t)LISA_IDX(j[a], kmax + 1) * kSplineRec;
                    xl[a] = z[0]; xr[a] = z[1]; ca[a] = z[2]; cb[a] = z[3]; cc[a] = z[4]; cd[a] = z[5];
                }
                t[a] = x - xl[a];
                P[a] = ca[a] + t[a] * (cb[a] + t[a] * (cc[a] + t[a] * cd[a]));
            }
            double eh = 0.0;
            if (HAS_H) {
                const double sl = BROKEN ? (ell < 0.0 ? n1 : n2) : n1;
                eh = exp10(lA + P[C]) * exp2(sl * ell);
            }
            double fwd = 0.0, To = 0.0, Tt = 0.0, H = 0.0, qv[NSP];
            for (int c = 0; c < C; ++c) {
                const double E = exp10(P[c]);
                const double N = ao2 * q[3 + c] + at2 * q[6 + c];
                const double Eh = HAS_H ? eh * q[9 + c] : 0.0;
                const double Sc = E * N + Eh;
                // g = nu (1 - S) / S^2 applied as nu (r - 1) (r E) with r = 1 / S: no intermediate
                // overflows where S^2 would (S beyond 1e154)
                const double r = 1.0 / Sc;
                const double gr = nu * (r - 1.0), rE = r * E;
                fwd += r + log(Sc);
                To += gr * rE * q[3 + c];
                Tt += gr * rE * q[6 + c];
                H += gr * (r * Eh);
                qv[c] = kLn10 * gr * rE * N;
            }
            if (HAS_H) qv[C] = kLn10 * H;
            acc[0] += nu * (fwd - (double)C);
            acc[1] += To;
            acc[2] += Tt;
            acc[3] += H;
            if (BROKEN && ell >= 0.0) acc[5] += ell * H; else acc[4] += ell * H;
            for (int a = 0; a < NSP; ++a) {
                const double qt = qv[a] * t[a];
                m[a][0] += qv[a];
                m[a][1] += qt;
                m[a][2] += qt * t[a];
                m[a][3] += qt * t[a] * t[a];
            }
        }
        for (int a = 0; a < NSP; ++a) {
            double* row = mom_row(mom, pre, s, a, nsp, kmax, D.nranges) + 4 * (int64_t)LISA_IDX(U.rho + j[a], D.nranges + kmax + 1);
            for (int p = 0; p < 4; ++p) row[p] = m[a][p];
        }
        double* sc = scal + 6 * (pre + U.rho);
        for (int k = 0; k < 6; ++k) sc[k] = acc[k];
    }
}

// ---- the FP32 gradient's two per-state passes: one CTA per (state, range) item --------------
// Mode kComp: the bins the FP32 adjoint masked (routed states, whose ill-conditioned intervals
// (conditioning T > kRobustT, prior draws with close knots) it loads as zero cubics). On an
// ill-conditioned interval the spline value is formed in float-float from the records' hi and lo
// parts (2^P as ex2(hi) (1 + lo ln2)) and the moments' products exactly (float-float); the bin's
// other splines take the FP32 adjoint's FP32 Horner and products.  Per-bin terms in FP32; the
// sums are added to the slots the FP32 adjoint wrote.  Only ranges overlapping the state's ill-conditioned x-extent run.
// Mode kFallback: the states the FP32 epilogue flagged (their FP32 sums left the FP32 range), all
// their bins: spline values in float-float from the FP32 records, the PSDs, 1 / S-hat and the
// sums in FP64; the sums overwrite the slots (every interval from the range's first bin to its
// last), in the FP32 adjoint's convention (moments about the records' midpoints, ln10 in q).
// A resident grid runs the (state, range) items of a compact list (kComp: the setup's route
// list; kFallback: the flag area's list), each CTA fetching its next item from a counter.
// The CTA's warps (4 for kComp, 16 for kFallback) split the range's bins, their lanes 32
// consecutive bins at a time; each spline's moments are reduced over the lanes per interval (a fixed butterfly),
// kept per warp and interval in shared memory, and summed over the warps in order.
constexpr int kComp = 0, kFallback = 1;

// 2^k in FP64 for an integer-valued float k (the fallback pass's scales): from the exponent field
// within the normal range, by scalbn beyond it (subnormal, 0, inf).
__device__ __forceinline__ double pow2_fb(float k) {
    if (k >= -1022.f && k <= 1023.f) return __longlong_as_double((long long)((int)k + 1023) << 52);
    return scalbn(1.0, (int)fmaxf(fminf(k, 2100.f), -2100.f));
}


template <int C, bool HAS_H, bool BROKEN, int MODE>
__global__ void __launch_bounds__(MODE == kComp ? 128 : 512)
    adjoint_range_kernel(int S, const int32_t* __restrict__ state_ds, const DatasetDev* __restrict__ ds,
                         const float* __restrict__ rec32, const float* __restrict__ xlo32,
                         const float* __restrict__ elllo32, const double* __restrict__ theta,
                         const int32_t* __restrict__ sstat, const int32_t* __restrict__ list, int R,
                         int32_t* __restrict__ fb, int32_t* __restrict__ next_item,
                         const int32_t* __restrict__ nint, const void* __restrict__ srec_v,
                         const float2* __restrict__ hull, int kmax, int nsp, const int64_t* __restrict__ prefix,
                         double* __restrict__ scal, double* __restrict__ mom) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    // per warp, spline and interval (from the range's first) the 4 moment sums: dynamic shared
    // memory of nwarps * NSP * (kmax + 1) * 4 doubles
    extern __shared__ double s_m[];
    __shared__ double s_t[16][6];
    __shared__ int s_jl[NSP];               // each spline's interval at the range's last bin
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;     // <= 16
    const int nsl = kmax + 1;               // interval slots per spline
    auto sm = [&](int w, int a, int jr, int p) -> double& { return s_m[(((w * NSP) + a) * nsl + jr) * 4 + p]; };
    // the list's (state, range) items, R ranges per state, fetched one at a time by each CTA
    // from the counter (a state's heavy ranges are contiguous in the list); the exits below are
    // CTA-uniform
    __shared__ int s_item;
    const int n_items = list[0] * R;
    for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1);
    __syncthreads();   // also: the previous item's reads of the shared sums are done
    const int it = s_item;
    __syncthreads();   // every thread has read s_item before thread 0 fetches again
    if (it >= n_items) break;
    const int s = LISA_IDX(list[1 + LISA_IDX(it / R, S)], S), rho = it % R;
    if (MODE == kComp && (sstat[s] & (kUserBits | kRouted)) != kRouted) continue;
    const DatasetDev& D = ds[state_ds[s]];
    if (rho >= D.nranges) continue;
    const int64_t b0 = D.bin0 + (int64_t)rho * kAdjBins;
    const int nb = (int)min((int64_t)kAdjBins, D.bin0 + D.npad - b0);
    const float* tb = rec32 + (b0 >> 1) * kPairRec;
    if (MODE == kComp) {
        const float2 hx = hull[s];
        if (fld(tb, nb - 1, 0) < hx.x || fld(tb, 0, 0) >= hx.y) continue;   // no ill-conditioned interval here
    }
    const double* th = theta + (size_t)s * LISA_N_THETA;
    const int64_t pre = prefix[s];
    // the state's parameters as the FP32 adjoint derives them
    const float ao2 = (float)(th[0] * th[0]), at2 = (float)(th[1] * th[1]);
    const float Af = (MODE == kComp && HAS_H) ? (float)exp10(th[2]) : 0.f;
    const float n1 = (float)th[3], n2 = BROKEN ? (float)th[4] : n1;
    // kFallback: the SGWB slopes and log2 A in float-float
    const ff sl1 = ff_from_double(th[3]), sl2 = ff_from_double(BROKEN ? th[4] : th[3]);
    const ff lA2 = ff_from_double(th[2] * kLog2_10);
    // bin i's x as the FP32 adjoint's walk compares it, and the FP32 records
    auto xbin = [&](int i) -> float { return fld(tb, i, 0); };
    auto rec = [&](int a, int j) -> const float* {
        const int64_t sp = (int64_t)s * nsp + a;
        return static_cast<const float*>(srec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(j, kmax + 1)) * kSplineRec32;
    };
    auto right_end = [&](int a, int j) -> float { return __ldg(rec(a, j)); };
    // the interval of spline a holding x, as the walk finds it (the count of right ends <= x,
    // which do not decrease): the lanes load the right ends together; x is warp-uniform and the
    // whole warp calls
    auto locate = [&](int a, float x) {
        const int n = nint[(int64_t)s * nsp + a];
        int c = 0;
        for (int jb = 0; jb < n - 1; jb += 32) {
            const int j = jb + lane;
            c += __popc(__ballot_sync(kFullMask, j < n - 1 && right_end(a, j) <= x));
        }
        return c;
    };
    if (MODE == kComp) {
        // does an ill-conditioned interval hold a bin of this range?  The threads take the
        // (spline, interval) pairs; interval j holds the x with right_end(j - 1) <= x < right_end(j)
        const float xa = xbin(0), xb = xbin(nb - 1);
        bool any = false;
        for (int e = threadIdx.x; e < NSP * nsl; e += blockDim.x) {
            const int a = e / nsl, j = e - a * nsl;
            const int n = nint[(int64_t)s * nsp + a];
            if (j < n && !(__ldg(rec(a, j) + 7) <= (float)kRobustT)) {
                const float lo = j == 0 ? -INFINITY : right_end(a, j - 1);
                const float hi = j == n - 1 ? INFINITY : right_end(a, j);
                any |= lo <= xb && hi > xa;
            }
        }
        if (!__syncthreads_or(any)) continue;   // CTA-uniform
    }
    int j0[NSP], nin[NSP];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        nin[a] = nint[(int64_t)s * nsp + a];
        j0[a] = locate(a, xbin(0));
    }
    for (int e = threadIdx.x; e < nwarps * NSP * nsl * 4; e += blockDim.x) s_m[e] = 0.0;
    if (threadIdx.x < 16 * 6) (&s_t[0][0])[threadIdx.x] = 0.0;
    if (threadIdx.x == 0)
        for (int a = 0; a < NSP; ++a) s_jl[a] = j0[a];
    __syncthreads();
    // this warp's bins and its running intervals
    const int w_lo = (warp * nb) / nwarps, w_hi = ((warp + 1) * nb) / nwarps;
    int cj[NSP];
    double am[NSP][4];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        cj[a] = w_lo < w_hi ? locate(a, xbin(w_lo)) : j0[a];
        for (int p = 0; p < 4; ++p) am[a][p] = 0.0;
    }
    auto wsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
        return v;
    };
    // lane-local running sums of the warp's current intervals (float-float for kComp, FP64 for
    // kFallback; folded into am, over the lanes, only when an interval is left), and (kComp) of
    // the template terms
    ff ls[NSP][4];
    float ltf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // kComp: the template terms (<= 32 per lane)
    double lsd[NSP][4];   // kFallback: the lanes' FP64 running sums, folded the same way
#pragma unroll
    for (int a = 0; a < NSP; ++a)
        for (int p = 0; p < 4; ++p) {
            ls[a][p] = ff{0.f, 0.f};
            lsd[a][p] = 0.0;
        }
    // kComp: float-float sums over the lanes (a fixed butterfly on the FP32 pipe); lane 0 adds
    // the result to its FP64 running sums
    auto wsum_ff = [&](ff v) {
        for (int o = 16; o > 0; o >>= 1)
            v = ff_add(v, ff{__shfl_xor_sync(kFullMask, v.hi, o), __shfl_xor_sync(kFullMask, v.lo, o)});
        return v;
    };
    auto flush = [&](int a) {
        if (MODE == kComp)
            for (int p = 0; p < 4; ++p) {
                const ff w = wsum_ff(ls[a][p]);
                if (lane == 0) am[a][p] += (double)w.hi + (double)w.lo;
                ls[a][p] = ff{0.f, 0.f};
            }
        else
            for (int p = 0; p < 4; ++p) {
                am[a][p] += wsum(lsd[a][p]);
                lsd[a][p] = 0.0;
            }
        if (lane == 0)
            for (int p = 0; p < 4; ++p) sm(warp, a, cj[a] - j0[a], p) = am[a][p];
        for (int p = 0; p < 4; ++p) am[a][p] = 0.0;
    };
    double ts[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    // kComp: the warp's 32-bin groups holding a bin of an ill-conditioned interval (bit g: bins
    // w_lo + 32 g ...), the lanes taking the intervals; the others are skipped (nothing to add)
    unsigned gmask = 0xffffffffu;
    if (MODE == kComp && w_hi - w_lo <= 32 * 32) {
        auto lower = [&](float v) {   // first bin of the warp with x >= v (w_hi if none)
            int lo = w_lo, hi = w_hi;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (xbin(mid) >= v) hi = mid; else lo = mid + 1;
            }
            return lo;
        };
        unsigned m = 0;
#pragma unroll
        for (int a = 0; a < NSP; ++a)
            for (int jb = 0; jb < nin[a]; jb += 32) {
                const int j = jb + lane;
                if (j >= nin[a] || __ldg(rec(a, j) + 7) <= (float)kRobustT) continue;
                // the walk's bins of interval j: right_end(j - 1) <= x < right_end(j)
                const int i_lo = j == 0 ? w_lo : lower(right_end(a, j - 1));
                const int i_hi = j == nin[a] - 1 ? w_hi : lower(right_end(a, j));
                if (i_lo >= i_hi) continue;
                const int g0 = (i_lo - w_lo) >> 5, g1 = (i_hi - 1 - w_lo) >> 5;
                m |= (g1 >= 31 ? 0xffffffffu : ((2u << g1) - 1u)) & ~((1u << g0) - 1u);
            }
        gmask = __reduce_or_sync(kFullMask, m);
    }
    for (int i0 = w_lo; i0 < w_hi; i0 += 32) {
        if (!((gmask >> ((i0 - w_lo) >> 5)) & 1u)) continue;   // warp-uniform
        const int i = i0 + lane;
        const bool valid = i < w_hi;
        const int last_lane = min(31, w_hi - 1 - i0);
        const int ib = valid ? i : i0;
        const float x = xbin(ib);
        int jl[NSP];
        bool hard = false;
#pragma unroll
        for (int a = 0; a < NSP; ++a) {
            int j = cj[a];
            while (j < nin[a] - 1 && x >= right_end(a, j)) ++j;
            jl[a] = j;
            if (MODE == kComp) hard |= !(__ldg(rec(a, j) + 7) <= (float)kRobustT);
        }
        const bool use = valid && (MODE == kFallback || hard);
        if (!__any_sync(kFullMask, use)) {
            // nothing in this group: move the running intervals up (their sums so far first)
#pragma unroll
            for (int a = 0; a < NSP; ++a) {
                const int jlo = __shfl_sync(kFullMask, jl[a], 0);
                if (jlo > cj[a]) {
                    flush(a);
                    cj[a] = jlo;
                }
            }
            continue;
        }
        // the spline signals q (FP32 for kComp, FP64 for kFallback) and t = x - x_o (FP32);
        // kComp: whether each spline's interval is ill-conditioned at this bin
        float qk[NSP], tv[NSP];
        bool hs[NSP];
        double qd[NSP];
        double tc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < NSP; ++a) {
            qk[a] = tv[a] = 0.f;
            qd[a] = 0.0;
            hs[a] = false;
        }
        if (use) {
            if constexpr (MODE == kComp) {
                const float xf = fld(tb, ib, 0), ell = fld(tb, ib, 1), nu = fld(tb, ib, 2);
                const float x_lo = __ldg(xlo32 + b0 + ib);
                // per spline: float-float on an ill-conditioned interval (hs), the FP32 adjoint's
                // FP32 Horner on the compensated t on the others
                float P[NSP], cor[NSP], tl[NSP];
#pragma unroll
                for (int a = 0; a < NSP; ++a) {
                    const float4* rr = reinterpret_cast<const float4*>(rec(a, jl[a]));
                    const float4 A = __ldg(rr), Bq = __ldg(rr + 1), Cq = __ldg(rr + 2);
                    const ff tt = two_sum(xf, -A.y);
                    tl[a] = tt.hi + (tt.lo + (x_lo - Cq.x));   // t = x - x_o as the FP32 adjoint forms it
                    hs[a] = !(Bq.w <= (float)kRobustT);
                    if (hs[a]) {
                        const float4 Dq = __ldg(rr + 3);
                        const ff tf = ff_add(ff{xf, x_lo}, ff{-A.y, -Cq.x});
                        ff v = {Bq.y, Dq.x};
                        v = ff_add(ff_mul(v, tf), ff{Bq.x, Cq.w});
                        v = ff_add(ff_mul(v, tf), ff{A.w, Cq.z});
                        v = ff_add(ff_mul(v, tf), ff{A.z, Cq.y});
                        P[a] = v.hi;
                        cor[a] = fmaf(v.lo, (float)kLn2, 1.f);
                    } else {
                        P[a] = fmaf(fmaf(fmaf(Bq.y, tl[a], Bq.x), tl[a], A.w), tl[a], A.z);
                        cor[a] = 1.f;
                    }
                }
                float eh = 0.f;
                if (HAS_H) {
                    const float sl = BROKEN ? (ell < 0.f ? n1 : n2) : n1;
                    eh = Af * ex2_approx(fmaf(sl, ell, P[C])) * cor[C];
                }
                float lsum = 0.f, rsum = -(float)C, To = 0.f, Tt = 0.f, Hs = 0.f, q[NSP];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float go = fld(tb, ib, 3 + c), gt = fld(tb, ib, 6 + c);
                    const float E = ex2_approx(P[c]) * cor[c];
                    const float N = fmaf(ao2, go, at2 * gt);
                    const float Eh = HAS_H ? eh * fld(tb, ib, 9 + c) : 0.f;
                    const float Sc = HAS_H ? fmaf(E, N, Eh) : E * N;
                    const float r = rcp_approx(Sc);
                    const float gp = fmaf(r, r, -r);
                    const float gE = gp * E;
                    rsum += r;
                    lsum += lg2_approx(Sc);
                    To = fmaf(gE, go, To);
                    Tt = fmaf(gE, gt, Tt);
                    if (HAS_H) Hs = fmaf(gp, Eh, Hs);
                    q[c] = nu * gE * N;
                }
                Hs *= nu;
                if (HAS_H) q[C] = Hs;
                float tf[6] = {nu * fmaf((float)kLn2, lsum, rsum), nu * To, nu * Tt, Hs, 0.f, 0.f};
                if (BROKEN && ell >= 0.f)
                    tf[5] = ell * Hs;
                else
                    tf[4] = ell * Hs;
                for (int k = 0; k < 6; ++k) ltf[k] += tf[k];
#pragma unroll
                for (int a = 0; a < NSP; ++a) {
                    qk[a] = q[a];
                    tv[a] = tl[a];
                }
            } else {
                // exponents in float-float (spline values from the FP32 records' hi + lo); per
                // channel an integer scale k with S-hat = S' 2^k, S' in [0.35, 2.9); S', 1 / S'
                // and log2 S' in FP32; FP64 only for r = 2^-k / S' and the sums
                const float xf = fld(tb, ib, 0), nuf = fld(tb, ib, 2);
                const float x_lo = __ldg(xlo32 + b0 + ib);
                const ff ell = {fld(tb, ib, 1), __ldg(elllo32 + b0 + ib)};
                const double nu = nuf;
                ff Pv[NSP];
#pragma unroll
                for (int a = 0; a < NSP; ++a) {
                    const float4* rr = reinterpret_cast<const float4*>(rec(a, jl[a]));
                    const float4 A = __ldg(rr), Bq = __ldg(rr + 1), Cq = __ldg(rr + 2), Dq = __ldg(rr + 3);
                    const ff tt = two_sum(xf, -A.y);
                    tv[a] = tt.hi + (tt.lo + (x_lo - Cq.x));   // t = x - x_o as the FP32 adjoint
                    const ff tf = ff_add(ff{xf, x_lo}, ff{-A.y, -Cq.x});
                    ff v = {Bq.y, Dq.x};
                    v = ff_add(ff_mul(v, tf), ff{Bq.x, Cq.w});
                    v = ff_add(ff_mul(v, tf), ff{A.w, Cq.z});
                    Pv[a] = ff_add(ff_mul(v, tf), ff{A.z, Cq.y});   // log2 units
                }
                // the SGWB exponent: P_h + slope * log2(f / f_ref) + log2 A
                ff xh = {0.f, 0.f};
                if (HAS_H) xh = ff_add(ff_add(Pv[C], ff_mul((BROKEN && ell.hi >= 0.f) ? sl2 : sl1, ell)), lA2);
                double rs = 0.0, To = 0.0, Tt = 0.0, H = 0.0;
                float ks = 0.f, l2s = 0.f;   // sum of the scales k (integers) and of log2 S'
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float go = fld(tb, ib, 3 + c), gt = fld(tb, ib, 6 + c);
                    const float N = fmaf(ao2, go, at2 * gt);
                    int eN, eG = 0;
                    const float mN = frexpf(N, &eN);   // N = mN 2^eN
                    const float mG = HAS_H ? frexpf(fld(tb, ib, 9 + c), &eG) : 0.f;
                    const float yh = mG > 0.f ? xh.hi + (float)eG : -INFINITY;
                    const float kc = rintf(fmaxf(Pv[c].hi + (float)eN, yh));
                    const ff dN = ff_add(Pv[c], ff{(float)eN - kc, 0.f});
                    const float eNs = ex2_approx(dN.hi + dN.lo) * mN;   // E N / 2^k
                    float eHs = 0.f;                                     // E_h G_h / 2^k
                    if (HAS_H && mG > 0.f) {
                        const ff dH = ff_add(xh, ff{(float)eG - kc, 0.f});
                        eHs = ex2_approx(dH.hi + dH.lo) * mG;
                    }
                    const float Sp = eNs + eHs;
                    const float rp = rcp_approx(Sp);
                    const float rE = eNs * rp;   // E N / S-hat
                    const double r = (double)rp * pow2_fb(-kc);
                    const double gr = nu * (r - 1.0);
                    rs += r;
                    ks += kc;
                    l2s += lg2_approx(Sp);
                    const float rEN = rE * rcp_approx(N);   // E / S-hat
                    To = fma(gr, (double)(rEN * go), To);
                    Tt = fma(gr, (double)(rEN * gt), Tt);
                    if (HAS_H) H = fma(gr, (double)(eHs * rp), H);
                    qd[c] = (kLn10 * gr) * (double)rE;
                }
                const double elld = (double)ell.hi + (double)ell.lo;
                tc[0] = nu * (rs + kLn2 * ((double)ks + (double)l2s) - (double)C);
                tc[1] = To;
                tc[2] = Tt;
                tc[3] = H;
                if (BROKEN && elld >= 0.0)
                    tc[5] = elld * H;
                else
                    tc[4] = elld * H;
                if (HAS_H) qd[C] = kLn10 * H;
            }
        }
        if (MODE == kFallback)
            for (int k = 0; k < 6; ++k) ts[k] += tc[k];
        // moments per interval: the lanes' intervals are non-decreasing, from lane 0's to the last
        // valid lane's
#pragma unroll
        for (int a = 0; a < NSP; ++a) {
            double d[4];
            if (MODE == kComp) {
                // the products q t^p of the FP32 values, exact (float-float) on an ill-conditioned
                // interval, FP32 on the others; while every lane stays in the warp's current
                // interval they go to the lane-local sums
                const float qf = qk[a], t = tv[a], qt = qf * t;
                ff p1 = {qt, 0.f}, p2, p3;
                if (hs[a]) {
                    p1.lo = fmaf(qf, t, -qt);
                    p2 = ff_mul(p1, ff{t, 0.f});
                    p3 = ff_mul(p2, ff{t, 0.f});
                } else {
                    p2 = ff{qt * t, 0.f};
                    p3 = ff{p2.hi * t, 0.f};
                }
                if (__all_sync(kFullMask, !use || jl[a] == cj[a])) {
                    if (use) {
                        ls[a][0] = ff_add(ls[a][0], ff{qf, 0.f});
                        ls[a][1] = ff_add(ls[a][1], p1);
                        ls[a][2] = ff_add(ls[a][2], p2);
                        ls[a][3] = ff_add(ls[a][3], p3);
                    }
                    continue;
                }
                // lanes in several intervals: per interval the float-float sum over its lanes
                const ff dff[4] = {ff{qf, 0.f}, p1, p2, p3};
                const int jlo = __shfl_sync(kFullMask, jl[a], 0);
                const int jhi = __shfl_sync(kFullMask, jl[a], last_lane);
                for (int jj = jlo; jj <= jhi; ++jj) {
                    const bool in = use && jl[a] == jj;
                    ff m[4];
                    for (int p = 0; p < 4; ++p) m[p] = wsum_ff(in ? dff[p] : ff{0.f, 0.f});
                    if (jj > cj[a]) {
                        flush(a);
                        cj[a] = jj;
                    }
                    if (lane == 0)
                        for (int p = 0; p < 4; ++p) am[a][p] += (double)m[p].hi + (double)m[p].lo;
                }
                continue;
            } else {
                const double t = tv[a], qt = qd[a] * t;
                d[0] = qd[a];
                d[1] = qt;
                d[2] = qt * t;
                d[3] = d[2] * t;
                if (__all_sync(kFullMask, !use || jl[a] == cj[a])) {
                    if (use)
                        for (int p = 0; p < 4; ++p) lsd[a][p] += d[p];
                    continue;
                }
            }
            const int jlo = __shfl_sync(kFullMask, jl[a], 0);
            const int jhi = __shfl_sync(kFullMask, jl[a], last_lane);
            for (int jj = jlo; jj <= jhi; ++jj) {
                const bool in = use && jl[a] == jj;
                double m[4];
                for (int p = 0; p < 4; ++p) m[p] = wsum(in ? d[p] : 0.0);
                if (jj > cj[a]) {
                    flush(a);
                    cj[a] = jj;
                }
                for (int p = 0; p < 4; ++p) am[a][p] += m[p];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        if (w_lo < w_hi) {
            flush(a);
            if (lane == 0) atomicMax(&s_jl[a], cj[a]);
        }
    }
    for (int k = 0; k < 6; ++k) {
        const double v = wsum(MODE == kComp ? (double)ltf[k] : ts[k]);
        if (lane == 0) s_t[warp][k] = v;
    }
    __syncthreads();
    // the warps' sums in order, to the slots
    for (int e = threadIdx.x; e < NSP * nsl; e += blockDim.x) {
        const int a = e / nsl, jr = e % nsl;
        const int j = j0[a] + jr;
        if (j > s_jl[a]) continue;
        double v[4];
        for (int p = 0; p < 4; ++p) {
            v[p] = 0.0;
            for (int w = 0; w < nwarps; ++w) v[p] += sm(w, a, jr, p);
        }
        double* row = mom_row(mom, pre, s, a, nsp, kmax, D.nranges) + 4 * (int64_t)LISA_IDX(rho + j, D.nranges + kmax + 1);
        if (MODE == kComp) {
            // the FP32 adjoint's slots carry ln10 (its q's factor)
            if (v[0] != 0.0 || v[1] != 0.0 || v[2] != 0.0 || v[3] != 0.0) {
                bool bad = false;
                for (int p = 0; p < 4; ++p) {
                    row[p] += kLn10 * v[p];
                    bad |= !isfinite(row[p]);
                }
                if (bad) fb_flag(fb, S, s);
            }
        } else {
            for (int p = 0; p < 4; ++p) row[p] = v[p];
        }
    }
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += s_t[w][k];
        if (MODE == kComp) {
            scal[6 * (pre + rho) + k] += v;
            if (!isfinite(scal[6 * (pre + rho) + k])) fb_flag(fb, S, s);
        } else {
            scal[6 * (pre + rho) + k] = v;
        }
    }
    }
}

// ---- epilogue: one warp per state, FP64 ----------------------------------------------------------
constexpr int kEpiRanges = 256;   // adjoint ranges whose bounds the epilogue stages (524,288 bins)

// d s_k / d m_{k+delta}, delta = -2..1, for the Akima slope at knot k (Appendix A rules,
// including the ends), returned in d[0..3] = delta -2, -1, 0, +1.  mm2..mp1 = m_{k-2}..m_{k+1}.
template <class T>
__device__ __forceinline__ void akima_slope_grad(int k, int K, T mm2, T mm1, T m0, T mp1, T sk, T d[4]) {
    d[0] = d[1] = d[2] = d[3] = T(0);
    if (k == 0) {                 // s_0 = (3 m_0 - m_1)/2
        d[2] = T(1.5);
        d[3] = T(-0.5);
        return;
    }
    if (k == K - 1) {             // s_{K-1} = (3 m_{K-2} - m_{K-3})/2
        d[1] = T(1.5);
        d[0] = T(-0.5);
        return;
    }
    auto sgn = [](T v) { return spl::sign_of(v); };
    const T ml = mm1, mr = m0;  // slopes left and right of knot k
    T wl, wr;
    if (k == 1) {
        wl = fabs(mp1 - m0);
        wr = fabs(m0 - mm1);
    } else if (k == K - 2) {
        wl = fabs(m0 - mm1);
        wr = fabs(mm1 - mm2);
    } else {
        wl = fabs(mp1 - m0);
        wr = fabs(mm1 - mm2);
    }
    const T D = wl + wr;
    if (D == T(0)) {
        d[1] = T(0.5);
        d[2] = T(0.5);
        return;
    }
    const T iD = T(1) / D;
    const T dwl = (ml - sk) * iD, dwr = (mr - sk) * iD;   // ds/dwl, ds/dwr
    d[1] += wl * iD;   // ds/dml
    d[2] += wr * iD;   // ds/dmr
    if (k == 1) {
        // wl = |m_{k+1} - m_k|, wr = |m_k - m_{k-1}|
        const T a1 = sgn(mp1 - m0), a2 = sgn(m0 - mm1);
        d[3] += dwl * a1;
        d[2] -= dwl * a1;
        d[2] += dwr * a2;
        d[1] -= dwr * a2;
    } else if (k == K - 2) {
        // wl = |m_k - m_{k-1}|, wr = |m_{k-1} - m_{k-2}|
        const T a1 = sgn(m0 - mm1), a2 = sgn(mm1 - mm2);
        d[2] += dwl * a1;
        d[1] -= dwl * a1;
        d[1] += dwr * a2;
        d[0] -= dwr * a2;
    } else {
        // wl = |m_{k+1} - m_k|, wr = |m_{k-1} - m_{k-2}|
        const T a1 = sgn(mp1 - m0), a2 = sgn(mm1 - mm2);
        d[3] += dwl * a1;
        d[2] -= dwl * a1;
        d[1] += dwr * a2;
        d[0] -= dwr * a2;
    }
}

// One state's reverse map (one warp): log L from the range sums, the template components, and
// per spline the moments gathered over the ranges, re-expanded about the knots (FP32 records:
// they are about the midpoints) and pushed back through the Akima or natural-cubic construction,
// in T (double, or float-float on the FP32 pipe).  Returns true, for the caller to redo the
// state in FP64, where a sum, a moment or a gradient value is not finite (a float-float run
// whose values left the FP32 exponent range); the FP64 run's return value is not used.
// sX, sY: the warp's 64-double scratch rows; sRf, sRl: its kEpiRanges-double range-bound rows.
template <int C, bool HAS_H, bool BROKEN, class T>
__device__ __noinline__ bool epilogue_state(int s, const int32_t* __restrict__ state_ds,
                                            const DatasetDev* __restrict__ ds, const int32_t* __restrict__ sstat,
                                            const double* __restrict__ theta, const int32_t* __restrict__ count,
                                            const double* __restrict__ kx, const double* __restrict__ kw, int kmax,
                                            int kind, int nsp, const int64_t* __restrict__ prefix,
                                            const double* __restrict__ scal, const double* __restrict__ mom,
                                            const float* __restrict__ rec32, const double* __restrict__ rec64,
                                            const void* __restrict__ srec_v, int fp32, double* __restrict__ out_logL,
                                            double* __restrict__ grad, double* sX, double* sY, double* sRf,
                                            double* sRl) {
    constexpr bool kFF = std::is_same<T, spl::F2>::value;
    const int lane = threadIdx.x & 31;
    const int G = LISA_N_THETA + nsp * (2 * kmax + 2);
    double* gs = grad + (size_t)s * G;
    for (int k = lane; k < G; k += 32) gs[k] = 0.0;
    __syncwarp();
    if (sstat[s] & kUserBits) {
        if (lane == 0) out_logL[s] = -INFINITY;
        return false;
    }
    const DatasetDev& D = ds[state_ds[s]];
    const int nr = D.nranges;
    const int64_t pre = prefix[s];
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = lane; r < nr; r += 32)
        for (int k = 0; k < 6; ++k) v[k] += scal[6 * (pre + r) + k];
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 6; ++k) v[k] += __shfl_down_sync(kFullMask, v[k], o);
    for (int k = 0; k < 6; ++k) v[k] = __shfl_sync(kFullMask, v[k], 0);
    double L = -v[0] - D.Cnu + D.K;
    const bool finite = isfinite(L);
    if (kFF) {
        bool sums_ok = finite;
        for (int k = 1; k < 6; ++k) sums_ok &= isfinite(v[k]);
        if (!sums_ok) return true;
    }
    if (lane == 0) out_logL[s] = finite ? L : -INFINITY;
    if (!finite) return false;   // gradient stays zero
    bool bad = false;            // a non-finite moment or gradient value
    // range bounds: in shared memory when they fit, else read per range below
    const bool staged = nr <= kEpiRanges;
    auto range_x = [&](int rho, double& xf, double& xlb) {
        const int64_t b0 = D.bin0 + (int64_t)rho * kAdjBins;
        const int nb = (int)min((int64_t)kAdjBins, D.bin0 + D.npad - b0);
        if (fp32) {
            const float* tb = rec32 + (b0 >> 1) * kPairRec;
            xf = (double)fld(tb, 0, 0);
            xlb = (double)fld(tb, nb - 1, 0);
        } else {
            xf = rec64[b0 * kRec];
            xlb = rec64[(b0 + nb - 1) * kRec];
        }
    };
    if (staged) {
        for (int rho = lane; rho < nr; rho += 32) range_x(rho, sRf[LISA_IDX(rho, kEpiRanges)], sRl[LISA_IDX(rho, kEpiRanges)]);
        __syncwarp();
    }
    const double* th = theta + (size_t)s * LISA_N_THETA;
    if (lane == 0) {
        gs[0] = 2.0 * th[0] * v[1];
        gs[1] = 2.0 * th[1] * v[2];
        if (HAS_H) {
            gs[2] = kLn10 * v[3];
            gs[3] = kLn2 * (BROKEN ? v[4] : v[4] + v[5]);
            gs[4] = BROKEN ? kLn2 * v[5] : 0.0;
        }
    }
    const int per_spline = 2 * kmax + 2;
    for (int a = 0; a < nsp; ++a) {
        const int64_t sp = (int64_t)s * nsp + a;
        spl::WarpSpline<T> W;
        spl::warp_build_spline<T>(W, kx + sp * kmax, kw + sp * (kmax + 2), count[sp], kmax, kind, D.x_lo, D.x_hi,
                               sX, sY);
        if (W.st) continue;
        const int K = W.K;
        const int nint = K - 1;
        const double* row = mom_row(const_cast<double*>(mom), pre, s, a, nsp, kmax, nr);
        // moments of each interval, gathered over the ranges that touched it (fixed order)
        double Md[2][4];   // summed in FP64 (the accumulation over ranges)
        T M[2][4];
        for (int q = 0; q < 2; ++q) {
            const int jj = lane + 32 * q;
            for (int p = 0; p < 4; ++p) {
                Md[q][p] = 0.0;
                M[q][p] = T(0);
            }
            if (jj >= nint) continue;
            double lo_b, hi_b;   // the interval's bounds as the likelihood kernels' walk sees them
            if (fp32) {
                const float* r = static_cast<const float*>(srec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(jj, kmax + 1)) * kSplineRec32;
                lo_b = (double)r[6];
                hi_b = (double)r[0];
            } else {
                const double* r = static_cast<const double*>(srec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(jj, kmax + 1)) * kSplineRec;
                lo_b = r[0];
                hi_b = r[1];
            }
            if (staged) {
                // the ranges that touch the interval are the contiguous span [r0, r1] (bins are
                // sorted): first range whose last bin reaches lo_b, last one that starts below hi_b
                int r0 = 0, r1 = nr - 1;
                if (jj != 0) {
                    int lo = 0, hi = nr;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sRl[mid] >= lo_b) hi = mid; else lo = mid + 1;
                    }
                    r0 = lo;
                }
                if (jj != nint - 1) {
                    int lo = 0, hi = nr;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sRf[mid] < hi_b) lo = mid + 1; else hi = mid;
                    }
                    r1 = lo - 1;
                }
                for (int rho = r0; rho <= r1; ++rho)
                    for (int p = 0; p < 4; ++p) Md[q][p] += row[4 * (int64_t)LISA_IDX(rho + jj, nr + kmax + 1) + p];
            } else {
                for (int rho = 0; rho < nr; ++rho) {
                    double xf, xlb;
                    range_x(rho, xf, xlb);
                    const bool touches = (jj == 0 || xlb >= lo_b) && (jj == nint - 1 || xf < hi_b);
                    if (touches)
                        for (int p = 0; p < 4; ++p) Md[q][p] += row[4 * (int64_t)LISA_IDX(rho + jj, nr + kmax + 1) + p];
                }
            }
            for (int p = 0; p < 4; ++p) {
                bad |= !isfinite(Md[q][p]);
                M[q][p] = T(Md[q][p]);
            }
            if (fp32) {
                // moments about the FP32 midpoint xo -> about the left knot x_j:  t = u + mo
                const float* r = static_cast<const float*>(srec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(jj, kmax + 1)) * kSplineRec32;
                const T mo = spl::from_hilo<T>(r[1], r[8]) - W.x[q];
                const T C0 = M[q][0], C1 = M[q][1], C2 = M[q][2], C3 = M[q][3];
                M[q][0] = C0;
                M[q][1] = C1 + mo * C0;
                M[q][2] = C2 + mo * (T(2) * C1 + mo * C0);
                M[q][3] = C3 + mo * (T(3) * C2 + mo * (T(3) * C1 + mo * C0));
            }
        }
        // ---- reverse through the coefficient map
        T ybar[2], xbar[2], mbar[2], hbar[2], own[2], nxt[2];
        for (int q = 0; q < 2; ++q) {
            const int jj = lane + 32 * q;
            const bool iv = jj < nint;
            const T h = W.h[q], ih = W.ih[q], ih2 = ih * ih;
            const T M0 = M[q][0], M1 = M[q][1], M2 = M[q][2], M3 = M[q][3];
            ybar[q] = iv ? M0 : T(0);
            xbar[q] = iv ? -(W.cb[q] * M0 + T(2) * W.cc[q] * M1 + T(3) * W.cd[q] * M2) : T(0);
            mbar[q] = hbar[q] = own[q] = nxt[q] = T(0);
            if (!iv) continue;
            if (K < 4) {
                mbar[q] = M1;
            } else if (kind == LISA_SPLINE_NATURAL) {
                const T Mj = W.d2[q];
                own[q] = -M1 * h * T(1.0 / 3.0) + T(0.5) * M2 - M3 * ih * T(1.0 / 6.0);   // -> d/dM_j
                nxt[q] = -M1 * h * T(1.0 / 6.0) + M3 * ih * T(1.0 / 6.0);                // -> d/dM_{j+1}
                mbar[q] = M1;
                (void)Mj;
            } else {
                own[q] = M1 - T(2) * M2 * ih + M3 * ih2;               // -> d/ds_j
                nxt[q] = -M2 * ih + M3 * ih2;                         // -> d/ds_{j+1}
                mbar[q] = T(3) * M2 * ih - T(2) * M3 * ih2;
                hbar[q] = -(W.cc[q] * M2 + T(2) * W.cd[q] * M3) * ih;
            }
        }
        if (K >= 4 && kind == LISA_SPLINE_NATURAL) {
            // b = m - h (2 M_j + M_{j+1}) / 6,  d = (M_{j+1} - M_j) / (6 h): h dependence
            T Mn[2];
            spl::shift2(W.d2[0], W.d2[1], 1, Mn[0], Mn[1]);
            for (int q = 0; q < 2; ++q) {
                const int jj = lane + 32 * q;
                if (jj < nint) hbar[q] = -M[q][1] * (T(2) * W.d2[q] + Mn[q]) * T(1.0 / 6.0) - W.cd[q] * M[q][3] * W.ih[q];
            }
            // d/dM_k = own_k + nxt_{k-1}; M_0 and M_{K-1} are fixed
            T nprev[2], Mbar[2];
            spl::shift2(nxt[0], nxt[1], -1, nprev[0], nprev[1]);
            T A[2], B[2], Cc[2], R[2];
            T hm[2];
            spl::shift2(W.h[0], W.h[1], -1, hm[0], hm[1]);
            for (int q = 0; q < 2; ++q) {
                const int k = lane + 32 * q;
                Mbar[q] = (k >= 1 && k <= K - 2) ? own[q] + nprev[q] : T(0);
                if (k >= 1 && k <= K - 2) {
                    A[q] = hm[q];
                    B[q] = T(2) * (hm[q] + W.h[q]);
                    Cc[q] = W.h[q];
                    R[q] = Mbar[q];
                } else {
                    A[q] = T(0);
                    B[q] = T(1);
                    Cc[q] = T(0);
                    R[q] = T(0);
                }
            }
            spl::pcr_solve(A, B, Cc, R, K);   // the system is symmetric: lambda = A^-1 Mbar
            T lam[2], lamn[2], Mnn[2];
            for (int q = 0; q < 2; ++q) lam[q] = R[q] / B[q];
            spl::shift2(lam[0], lam[1], 1, lamn[0], lamn[1]);
            spl::shift2(Mn[0], Mn[1], 1, Mnn[0], Mnn[1]);
            for (int q = 0; q < 2; ++q) {
                const int k = lane + 32 * q;
                const T Mk = W.d2[q];
                // r_k = 6 (m_k - m_{k-1}):  mbar_k += 6 lam_k - 6 lam_{k+1}
                if (k >= 1 && k <= K - 2) mbar[q] += T(6) * lam[q];
                if (k + 1 >= 1 && k + 1 <= K - 2) mbar[q] -= T(6) * lamn[q];
                // row k:   h_{k-1} M_{k-1} + 2 (h_{k-1} + h_k) M_k + h_k M_{k+1}
                //   dh_k from row k: 2 M_k + M_{k+1};  from row k+1: M_k + 2 M_{k+1}
                if (k >= 1 && k <= K - 2) hbar[q] -= lam[q] * (T(2) * Mk + Mn[q]);
                if (k + 1 >= 1 && k + 1 <= K - 2 && k < nint) hbar[q] -= lamn[q] * (Mk + T(2) * Mn[q]);
                (void)Mnn;
            }
        } else if (K >= 4) {
            // Akima: d/ds_k = own_k + nxt_{k-1}, then through the slope rule to the interval slopes
            T nprev[2], sbar[2];
            spl::shift2(nxt[0], nxt[1], -1, nprev[0], nprev[1]);
            T mm1[2], mm2[2], mp1[2];
            spl::shift2(W.m[0], W.m[1], -1, mm1[0], mm1[1]);
            spl::shift2(W.m[0], W.m[1], -2, mm2[0], mm2[1]);
            spl::shift2(W.m[0], W.m[1], 1, mp1[0], mp1[1]);
            T c[4][2];   // contribution of knot k to mbar_{k + delta}, delta = -2..1
            for (int q = 0; q < 2; ++q) {
                const int k = lane + 32 * q;
                sbar[q] = (k < K) ? own[q] + (k >= 1 ? nprev[q] : T(0)) : T(0);
                T dd[4] = {T(0), T(0), T(0), T(0)};
                if (k < K) akima_slope_grad(k, K, mm2[q], mm1[q], W.m[q], mp1[q], W.d2[q], dd);
                for (int t = 0; t < 4; ++t) c[t][q] = sbar[q] * dd[t];
            }
            // mbar_i += c_{i+2}[-2] + c_{i+1}[-1] + c_i[0] + c_{i-1}[+1]
            T f0[2], f1[2], f3[2];
            spl::shift2(c[0][0], c[0][1], 2, f0[0], f0[1]);
            spl::shift2(c[1][0], c[1][1], 1, f1[0], f1[1]);
            spl::shift2(c[3][0], c[3][1], -1, f3[0], f3[1]);
            for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;
                if (i >= nint) continue;
                T add = c[2][q];
                if (i + 2 < K) add += f0[q];
                if (i + 1 < K) add += f1[q];
                if (i >= 1) add += f3[q];
                mbar[q] += add;
            }
        }
        // m_j = (y_{j+1} - y_j) / h_j ;  h_j = x_{j+1} - x_j
        T gmy[2], gmyp[2], ghp[2];
        for (int q = 0; q < 2; ++q) {
            const int jj = lane + 32 * q;
            gmy[q] = (jj < nint) ? mbar[q] * W.ih[q] : T(0);
            if (jj < nint) hbar[q] -= W.m[q] * gmy[q];
            else hbar[q] = T(0);
        }
        spl::shift2(gmy[0], gmy[1], -1, gmyp[0], gmyp[1]);
        spl::shift2(hbar[0], hbar[1], -1, ghp[0], ghp[1]);
        for (int q = 0; q < 2; ++q) {
            const int k = lane + 32 * q;
            if (k >= K) {
                ybar[q] = xbar[q] = T(0);
                continue;
            }
            ybar[q] += -gmy[q] + (k >= 1 ? gmyp[q] : T(0));
            xbar[q] += -hbar[q] + (k >= 1 ? ghp[q] : T(0));
        }
        // scatter: sorted knot k -> caller slots
        double* ga = gs + LISA_N_THETA + a * per_spline;
        const T y0 = spl::bcast(ybar[0], ybar[1], 0);
        const T yK = spl::bcast(ybar[0], ybar[1], K - 1);
        if (lane == 0) {
            ga[0] = spl::to_double(y0);
            ga[kmax + 1] = spl::to_double(yK);
            bad |= !isfinite(ga[0]) || !isfinite(ga[kmax + 1]);
        }
        const int k_in = K - 2;
        for (int half = 0; half < 2; ++half) {
            const int i = lane + 32 * half;          // caller's in-between knot index
            const int r = half ? W.rb : W.ra;        // its sorted position (1..K-2)
            const int rs = (i < k_in) ? r : 0;
            const T gy = spl::shfl(rs < 32 ? ybar[0] : ybar[1], rs & 31);
            const T gx = spl::shfl(rs < 32 ? xbar[0] : xbar[1], rs & 31);
            if (i < k_in) {
                ga[1 + LISA_IDX(i, kmax)] = spl::to_double(gy);
                ga[kmax + 2 + LISA_IDX(i, kmax)] = spl::to_double(gx);
                bad |= !isfinite(ga[1 + i]) || !isfinite(ga[kmax + 2 + i]);
            }
        }
    }
    // (the template components were written by lane 0, which checks them)
    if (lane == 0)
        for (int k = 0; k < LISA_N_THETA; ++k) bad |= !isfinite(gs[k]);
    return __any_sync(kFullMask, bad);
}

// One warp per state.  The FP32 call runs the reverse map in float-float and redoes in FP64 the
// states its adjoint passes flagged (fb[s]: sums beyond the FP32 range, recomputed by the
// fallback pass) and those whose float-float values are not finite; the FP64 call runs FP64.
// 4 CTAs of 128 threads per SM (128 registers) keep 2,432 states resident at once.
template <int C, bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(128, 4)
    adjoint_epilogue_kernel(int S, const int32_t* __restrict__ state_ds, const DatasetDev* __restrict__ ds,
                            const int32_t* __restrict__ sstat, const double* __restrict__ theta,
                            const int32_t* __restrict__ count, const double* __restrict__ kx,
                            const double* __restrict__ kw, int kmax, int kind, int nsp,
                            const int64_t* __restrict__ prefix, const double* __restrict__ scal,
                            const double* __restrict__ mom, const float* __restrict__ rec32,
                            const double* __restrict__ rec64, const void* __restrict__ srec_v, int fp32,
                            double* __restrict__ out_logL, double* __restrict__ grad,
                            const int32_t* __restrict__ fb) {
    __shared__ double sX[4][64];
    __shared__ double sY[4][64];
    // first and last bin's x of each adjoint range of the warp's dataset (the same for all its
    // states and splines), for datasets of up to kEpiRanges ranges
    __shared__ double sRf[4][kEpiRanges], sRl[4][kEpiRanges];
    const int warp = threadIdx.x >> 5;
    const int s = blockIdx.x * 4 + warp;
    if (s >= S) return;
    bool redo = !fp32 || fb[s] != 0;
    if (!redo)
        redo = epilogue_state<C, HAS_H, BROKEN, spl::F2>(s, state_ds, ds, sstat, theta, count, kx, kw, kmax, kind,
                                                         nsp, prefix, scal, mom, rec32, rec64, srec_v, fp32,
                                                         out_logL, grad, sX[warp], sY[warp], sRf[warp], sRl[warp]);
    if (redo)
        epilogue_state<C, HAS_H, BROKEN, double>(s, state_ds, ds, sstat, theta, count, kx, kw, kmax, kind, nsp,
                                                 prefix, scal, mom, rec32, rec64, srec_v, fp32, out_logL, grad,
                                                 sX[warp], sY[warp], sRf[warp], sRl[warp]);
}

// Whether every dataset meets the EXACT_T condition of adjoint_fp32_kernel.
inline bool adj_exact_t(const lisa_data* d) {
    for (const auto& D : d->h_ds) {
        if (D.nbins == 0) continue;
        if (!(D.x_lo <= D.xb_min && D.xb_max <= D.x_hi)) return false;
        const bool neg = D.x_hi < 0.0, pos = D.x_lo > 0.0;
        if (neg && !(-D.x_lo <= 2.9 * -D.x_hi)) return false;
        if (pos && !(D.x_hi <= 2.9 * D.x_lo)) return false;
        if (!neg && !pos) return false;
    }
    return true;
}

// The most adjoint ranges of any dataset (the per-(state, range) grids' second dimension).
inline int adj_max_ranges(const lisa_data* d) {
    int m = 1;
    for (const auto& Dh : d->h_ds) m = std::max(m, (int)Dh.nranges);
    return m;
}

// Dynamic shared memory of adjoint_range_kernel with nwarps warps.
inline size_t range_smem(const lisa_data* d, int kmax, int nwarps) {
    return sizeof(double) * (size_t)nwarps * (size_t)d->nsp * (size_t)(kmax + 1) * 4;
}

// The gradient workspace's arrays for one call (fb: FP32 calls only).
struct GradWs {
    double* scal;
    double* mom;
    int32_t* fb;          // FP32 calls: flags, count and list of the fallback states (fb_flag)
    const float2* hull;   // FP32 calls: the spline buffer's ill-conditioned x-extent per state
    const int32_t* route; // FP32 calls: the spline buffer's route count and list
};

template <int C, bool H, bool B>
cudaError_t launch_adjoint(const lisa_data* d, bool fp32, const lisa_params* params, const lisa_knots* kn,
                           const int32_t* sstat, const int32_t* nint, const void* srec, const GradWs& gw,
                           double* out, double* grad, cudaStream_t sm) {
    double* scal = gw.scal;
    double* mom = gw.mom;
    const int grid = d->n_sm * 8;
    const bool prof = prof_active(d, sm);
    const int S = (int)d->n_states;
    const int R = adj_max_ranges(d);
    prof_mark(d, prof, 0, sm);
    if (fp32 && cudaMemsetAsync(gw.fb, 0, sizeof(int32_t) * (2 * (size_t)S + 3), sm) != cudaSuccess)
        return cudaErrorInvalidValue;
    if (d->n_adj_units > 0) {
        if (fp32 && adj_exact_t(d))
            adjoint_fp32_kernel<C, H, B, true><<<grid, 128, 0, sm>>>(
                d->d_adj_units, d->n_adj_units, d->d_ds, d->d_rec32, d->d_xlo32, params->theta_dev, sstat, nint,
                static_cast<const float*>(srec), kn->kmax, d->nsp, d->d_adj_prefix, scal, mom, S, gw.fb);
        else if (fp32)
            adjoint_fp32_kernel<C, H, B, false><<<grid, 128, 0, sm>>>(
                d->d_adj_units, d->n_adj_units, d->d_ds, d->d_rec32, d->d_xlo32, params->theta_dev, sstat, nint,
                static_cast<const float*>(srec), kn->kmax, d->nsp, d->d_adj_prefix, scal, mom, S, gw.fb);
        prof_mark(d, prof, 1, sm);
        if (fp32) {
            // the bins of ill-conditioned intervals (routed states), masked above: the route
            // list's (state, range) items on a resident grid
            const size_t smc = range_smem(d, kn->kmax, 4);
            if (cudaFuncSetAttribute(adjoint_range_kernel<C, H, B, kComp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smc) != cudaSuccess)
                return cudaErrorInvalidValue;
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_range_kernel<C, H, B, kComp>, 128, smc) !=
                cudaSuccess)
                return cudaErrorInvalidValue;
            adjoint_range_kernel<C, H, B, kComp><<<d->n_sm * std::max(occ, 1), 128, smc, sm>>>(
                S, d->d_state_ds, d->d_ds, d->d_rec32, d->d_xlo32, d->d_elllo32, params->theta_dev, sstat, gw.route,
                R, gw.fb, gw.fb + 2 * S + 1, nint, srec, gw.hull, kn->kmax, d->nsp, d->d_adj_prefix, scal, mom);
            // the states whose FP32 sums left the FP32 range (flagged by both passes above): all
            // their bins again, FP64 sums, on a resident grid of 16-warp CTAs
            const size_t smf = range_smem(d, kn->kmax, 16);
            if (cudaFuncSetAttribute(adjoint_range_kernel<C, H, B, kFallback>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf) != cudaSuccess)
                return cudaErrorInvalidValue;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_range_kernel<C, H, B, kFallback>, 512,
                                                              smf) != cudaSuccess)
                return cudaErrorInvalidValue;
            adjoint_range_kernel<C, H, B, kFallback><<<d->n_sm * std::max(occ, 1), 512, smf, sm>>>(
                S, d->d_state_ds, d->d_ds, d->d_rec32, d->d_xlo32, d->d_elllo32, params->theta_dev, sstat,
                gw.fb + S, R, gw.fb, gw.fb + 2 * S + 2, nint, srec, nullptr, kn->kmax, d->nsp, d->d_adj_prefix, scal,
                mom);
        } else
            adjoint_fp64_kernel<C, H, B><<<grid, 128, 0, sm>>>(d->d_adj_units, d->n_adj_units, d->d_ds, d->d_rec64,
                                                               params->theta_dev, sstat, nint,
                                                               static_cast<const double*>(srec), kn->kmax, d->nsp,
                                                               d->d_adj_prefix, scal, mom);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else {
        prof_mark(d, prof, 1, sm);
    }
    prof_mark(d, prof, 2, sm);
    const unsigned eb = (unsigned)((d->n_states + 3) / 4);
    adjoint_epilogue_kernel<C, H, B><<<eb, 128, 0, sm>>>(
        S, d->d_state_ds, d->d_ds, sstat, params->theta_dev, kn->count_dev, kn->x_dev, kn->w_dev, kn->kmax, kn->kind,
        d->nsp, d->d_adj_prefix, scal, mom, d->d_rec32, d->d_rec64, srec, fp32 ? 1 : 0, out, grad, gw.fb);
    const cudaError_t e = cudaGetLastError();
    prof_mark(d, prof, 3, sm);
    if (prof) d->prof_valid = true;
    return e;
}

template <int C>
cudaError_t dispatch_adjoint(const lisa_data* d, bool fp32, const lisa_params* params, const lisa_knots* kn,
                             const int32_t* sstat, const int32_t* nint, const void* srec, const GradWs& gw,
                             double* out, double* grad, cudaStream_t sm) {
    if (d->sgwb_model == 0)
        return launch_adjoint<C, false, false>(d, fp32, params, kn, sstat, nint, srec, gw, out, grad, sm);
    if (d->sgwb_model == 1)
        return launch_adjoint<C, true, false>(d, fp32, params, kn, sstat, nint, srec, gw, out, grad, sm);
    return launch_adjoint<C, true, true>(d, fp32, params, kn, sstat, nint, srec, gw, out, grad, sm);
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" lisa_status lisa_psd_loglike_grad(const lisa_data* d, const lisa_params* params, const lisa_knots* kn,
                                             const void* buf, size_t buf_bytes, double* out, double* grad,
                                             void* ws, size_t ws_bytes, lisa_precision prec, lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_psd_loglike_grad");
    if (!d || !params || !kn || !buf || !out || !grad || !ws) return LISA_ERR_NULL;
    if (prec != LISA_FP32 && prec != LISA_FP64) return LISA_ERR_VALUE;
    if (d->cov != LISA_COV_DIAGONAL) return LISA_ERR_VALUE;   // the adjoint covers the diagonal model
    if (kn->kmax < 0 || kn->kmax > LISA_MAX_KNOTS || (kn->kind != LISA_SPLINE_AKIMA && kn->kind != LISA_SPLINE_NATURAL))
        return LISA_ERR_VALUE;
    if (params->n_states != d->n_states || kn->n_states != d->n_states || kn->n_splines != d->nsp)
        return LISA_ERR_SHAPE;
    if (d->n_states > 0 && (!params->theta_dev || !kn->count_dev || !kn->w_dev || (kn->kmax > 0 && !kn->x_dev)))
        return LISA_ERR_NULL;
    const SplineLayout L = spline_layout(d->n_states, d->nsp, kn->kmax);
    if (buf_bytes < L.bytes || (reinterpret_cast<uintptr_t>(buf) & 255)) return LISA_ERR_WORKSPACE;
    const bool fp32 = prec == LISA_FP32;
    const GradLayout GL = grad_layout(d, kn->kmax, fp32);
    if (ws_bytes < 256 + GL.bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return LISA_ERR_WORKSPACE;
    if (d->n_states == 0) return LISA_SUCCESS;
    const char* base = static_cast<const char*>(buf);
    const int32_t* sstat = reinterpret_cast<const int32_t*>(base + L.off_status);
    const int32_t* nint = reinterpret_cast<const int32_t*>(base + L.off_nint);
    const void* srec = base + L.off_rec;
    char* w = static_cast<char*>(ws) + 256;
    GradWs gw;
    gw.scal = reinterpret_cast<double*>(w + GL.off_scal);
    gw.mom = reinterpret_cast<double*>(w + GL.off_mom);
    gw.fb = fp32 ? reinterpret_cast<int32_t*>(w + GL.off_fb) : nullptr;
    gw.hull = reinterpret_cast<const float2*>(base + L.off_hull);
    gw.route = reinterpret_cast<const int32_t*>(base + L.off_route);
    cudaStream_t sm = (cudaStream_t)stream;
    cudaError_t e = d->C == 3 ? dispatch_adjoint<3>(d, fp32, params, kn, sstat, nint, srec, gw, out, grad, sm)
                              : dispatch_adjoint<2>(d, fp32, params, kn, sstat, nint, srec, gw, out, grad, sm);
    return e == cudaSuccess ? LISA_SUCCESS : LISA_ERR_CUDA;
}

LISA_DEBUG_TU(grad)
