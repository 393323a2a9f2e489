// Fused likelihood kernels: spline evaluation -> PSD assembly (Eq. splines) -> per-bin
// Wishart terms -> FP64 reduction over bins (Sec. III.C), for every state at once.
//
// FP32 path: the bin records of a work item (a tile of bins of one dataset) are staged into
// shared memory with one bulk asynchronous copy (cp.async.bulk + mbarrier), double-buffered
// across the persistent grid's items, and read by all state lanes of the CTA (broadcast).
// Each thread owns one state and a contiguous run of bins; it keeps the current interval of
// each spline in registers and advances it only when a bin passes the interval's right knot
// (bins are sorted in frequency, so the check is done once per group of bins).
//
// Per bin and state (normalised by the periodogram, so P-hat = 1, S-hat ~ 1):
//   E_c = 2^{P'_n,c(x)},  E_h = A 2^{P'_h(x) + n ell}                  (P' = log2(10) P)
// with each spline interval's cubic expanded about its midpoint (|x - xo| <= h/2 within the
// knots), which keeps the FP32 Horner sums small.
//   S_c = (a_oms^2 G_oms,c + a_tm^2 G_tm,c) E_c + E_h G_h,c
//   term = nu [ sum_c 1/S_c + ln prod_c S_c - C ]
// The reciprocal sum and the log are fused: sum_c 1/S_c = (sum_c prod_{c' != c} S_c') / prod S
// and ln prod S = ln2 lg2(prod S): one MUFU rcp and one MUFU lg2 per state-bin, with a
// per-channel fallback when the product leaves a safe FP32 range.  Terms are summed in FP32 over
// runs of 32 bins and then in FP64; the constant -C sum nu - sum nu ln P is added in FP64 at the
// end.
//
// Bins in a spline interval too ill-conditioned for FP32 (the setup flags such intervals and
// routes their states: large overshoots between close knots, |P| up to tens of decades for prior
// draws) are masked here and evaluated by the compensated kernel, from a per-call work list of
// the tiles they overlap: float-float Horner sums and the per-bin term in the log domain, so any
// exponent range is handled.
#include <cmath>

#include "lisa_math.cuh"

namespace lisa {
namespace {
using namespace dm;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One bulk global->shared copy completing on `bar` (16-byte aligned, size multiple of 16).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Bounded wait: true once the phase with this parity has completed, false after `limit` polls
// (the caller raises the error flag and stops issuing work).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// One spline interval's cubic about its midpoint xo, for the scalar per-bin path.
struct Iv32 {
    float xo, c0, c1, c2, c3;
};

// nu * (sum_c 1/S_c + ln prod_c S_c - C) in FP32: one reciprocal and one lg2 of the product,
// per-channel when the product leaves [1e-30, 1e30].
template <int C>
__device__ __forceinline__ float term_from_S(const float* S, float nu) {
    float prod, num;
    if (C == 3) {
        const float p01 = S[0] * S[1];
        prod = p01 * S[2];
        num = fmaf(S[2], S[0] + S[1], p01);
    } else {
        prod = S[0] * S[1];
        num = S[0] + S[1];
    }
    float v, lg;
    if (prod > 1e-30f && prod < 1e30f && num < 1e30f) {
        v = fmaf(num, rcp_approx(prod), -(float)C);
        lg = lg2_approx(prod);
    } else {
        v = -(float)C;
        lg = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            v += rcp_approx(S[c]);
            lg += lg2_approx(S[c]);
        }
    }
    return nu * fmaf((float)kLn2, lg, v);
}

// One bin, scalar (used next to knots, where the two bins of a pair may sit in different
// intervals).
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ float bin_term32(const float* __restrict__ tb, int i, const Iv32* iv, float ao2,
                                            float at2, float n1, float n2, float Af) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    const float x = fld(tb, i, 0), ell = fld(tb, i, 1), nu = fld(tb, i, 2);
    float p[NSP];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        const float t = x - iv[a].xo;
        p[a] = fmaf(fmaf(fmaf(iv[a].c3, t, iv[a].c2), t, iv[a].c1), t, iv[a].c0);
    }
    float eh = 0.f;
    if (HAS_H) {
        const float sl = BROKEN ? (ell < 0.f ? n1 : n2) : n1;
        eh = Af * ex2_approx(fmaf(sl, ell, p[C]));
    }
    float S[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float nc = fmaf(ao2, fld(tb, i, 3 + c), at2 * fld(tb, i, 6 + c));
        const float e = ex2_approx(p[c]);
        S[c] = HAS_H ? fmaf(e, nc, eh * fld(tb, i, 9 + c)) : e * nc;
    }
    return term_from_S<C>(S, nu);
}

// Safe range of the unguarded pair form.  Above 2^126 the reciprocal of the channel product is
// subnormal and flushed to zero, which would silently drop sum_c 1/S_c: the caller tracks the
// largest log2 of the product and redoes the chunk on the guarded path past this bound.  Below,
// every failure is loud: a product under 2^-126 is flushed to zero (infinite reciprocal, log2 =
// -inf), and an overflowing reciprocal-sum numerator or term is infinite, so the non-finite
// chunk sum that the caller also checks catches them; a normal product has an accurate
// reciprocal and log2.
constexpr float kPairLg2Max = 125.0f;

// 10^v as a float without the FP64 exp10: 2^(v log2 10) split into an exact integer power of
// two and a fractional part in [0, 1) handled by ex2 (one FP64 multiply, ~2 ulp).
__device__ __forceinline__ float exp10_to_float(double v) {
    const double e = v * kLog2_10;
    const double n = floor(e);
    if (n < -149.0) return 0.f;
    if (n > 127.0) return INFINITY;
    const float f = ex2_approx((float)(e - n));
    return n >= -126.0 ? f * __int_as_float(((int)n + 127) << 23) : ldexpf(f, (int)n);
}

// One step of a warp-wide search for the first t in [lo, hi) where a monotone predicate holds
// (hi when it holds nowhere): lane k sampled t = lo + k*step (step = ceil((hi - lo) / 32); lanes
// past hi count as true) and m is the ballot.  The answer lies after the last false sample and
// at or before the first true one, a range of at most step - 1 candidates.
__device__ __forceinline__ void search_narrow(int& lo, int& hi, int step, unsigned m) {
    if (m == 0u) {
        lo += 31 * step + 1;
        return;
    }
    const int k = __ffs(m) - 1;
    if (k == 0) {
        hi = lo;
        return;
    }
    const int first_true = lo + k * step;
    lo += (k - 1) * step + 1;
    hi = min(hi, first_true);
}

// log10 f (FP32) of padded bin b of the pair-block table.
__device__ __forceinline__ float bin_x(const float* __restrict__ rec32, int64_t b) {
    return __ldg(rec32 + (b >> 1) * kPairRec + (b & 1));
}

// Per-state FP32 parameters from theta (FP64), once per call: the per-bin kernels then need no
// FP64 arithmetic.  Non-finite theta propagates (the state's log L becomes -inf).
// One warp per state.  For a state the spline setup routed to the compensated kernel, the warp
// also finds the tiles that overlap the x-extent [h.x, h.y) of its ill-conditioned intervals --
// tile t with first-bin x < h.y and last-bin x >= h.x, a contiguous range because x increases
// with the bin -- appends its entry (RobustEntry) to the work list and records the entry's
// position in rent[s] (-1 for every other state).
__global__ void state_prep_kernel(int S, const double* __restrict__ theta, StateParams* __restrict__ prm,
                                  const int32_t* __restrict__ sstat, const float2* __restrict__ hull,
                                  const int32_t* __restrict__ state_ds, const DatasetDev* __restrict__ ds,
                                  const float* __restrict__ rec32, int tile_bins,
                                  unsigned long long* __restrict__ rcount, RobustEntry* __restrict__ rlist,
                                  int32_t* __restrict__ rent) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s64 = gt >> 5;
    const int lane = threadIdx.x & 31;
    if (s64 >= S) return;   // warp-uniform (blockDim is a multiple of 32)
    const int s = (int)s64;
    if (lane == 0) {
        const double* th = theta + (size_t)s * LISA_N_THETA;
        StateParams p;
        p.ao2 = (float)(th[0] * th[0]);
        p.at2 = (float)(th[1] * th[1]);
        p.Af = exp10_to_float(th[2]);
        const ff lA = ff_from_double(th[2] * kLog2_10);
        const ff n1 = ff_from_double(th[3]);
        const ff n2 = ff_from_double(th[4]);
        p.n1 = n1.hi;
        p.n1_lo = n1.lo;
        p.n2 = n2.hi;
        p.n2_lo = n2.lo;
        p.lA_hi = lA.hi;
        p.lA_lo = lA.lo;
        p.pad0 = p.pad1 = p.pad2 = 0.f;
        prm[s] = p;
        rent[s] = -1;
    }
    if (!(__ldg(sstat + s) & kRouted)) return;   // the same word in every lane
    const DatasetDev& D = ds[__ldg(state_ds + s)];
    const float2 h = __ldg(hull + s);
    const int nt = D.ntiles;
    const int64_t bend = D.bin0 + D.npad;
    // ta = first tile whose last bin has x >= h.x, tb = first tile whose first bin has x >= h.y;
    // the live tiles are [ta, tb).  Both searches run together, 32 samples per round.
    int alo = 0, ahi = nt, blo = 0, bhi = nt;
    while (alo < ahi || blo < bhi) {
        const int sa = (ahi - alo + 31) >> 5, sb = (bhi - blo + 31) >> 5;
        const int tA = alo + lane * sa, tB = blo + lane * sb;
        bool pa = true, pb = true;
        if (alo < ahi && tA < ahi) pa = bin_x(rec32, min(D.bin0 + (int64_t)(tA + 1) * tile_bins, bend) - 1) >= h.x;
        if (blo < bhi && tB < bhi) pb = bin_x(rec32, D.bin0 + (int64_t)tB * tile_bins) >= h.y;
        const unsigned ma = __ballot_sync(0xffffffffu, pa), mb = __ballot_sync(0xffffffffu, pb);
        if (alo < ahi) search_narrow(alo, ahi, sa, ma);
        if (blo < bhi) search_narrow(blo, bhi, sb, mb);
    }
    if (lane == 0 && blo > alo) {
        const unsigned long long old = atomicAdd(rcount, (1ull << 32) | (unsigned long long)(blo - alo));
        RobustEntry e;
        e.s = s;
        e.t0 = alo;
        e.u0 = (uint32_t)(old & 0xffffffffull);
        e.nt = blo - alo;
        e.b0 = D.bin0 + (int64_t)alo * tile_bins;
        e.p0 = (uint32_t)(D.pbase + (int64_t)(s - D.s0) * nt + alo);
        e.nb_last = (int32_t)min((int64_t)tile_bins, D.npad - (int64_t)(blo - 1) * tile_bins);
        rlist[old >> 32] = e;
        rent[s] = (int32_t)(old >> 32);
    }
}

// Current interval of one spline duplicated into register pairs for the packed path.
struct Iv2 {
    float2 nxo, c0, c1, c2, c3;
};

// One bin, scalar, with the intervals held as duplicated pairs (their .x halves).
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ float bin_term32p(const float* __restrict__ tb, int i, const Iv2* iv, float ao2, float at2,
                                             float n1, float n2, float Af) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    Iv32 v[NSP];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        v[a].xo = -iv[a].nxo.x;
        v[a].c0 = iv[a].c0.x;
        v[a].c1 = iv[a].c1.x;
        v[a].c2 = iv[a].c2.x;
        v[a].c3 = iv[a].c3.x;
    }
    return bin_term32<C, HAS_H, BROKEN>(tb, i, v, ao2, at2, n1, n2, Af);
}
// Three-input maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Two consecutive bins (one pair block) with FP32x2 instructions; both bins lie in the current
// intervals.  Returns, for both bins, v = sum_c 1/S_c - C and lg = log2 prod_c S_c (the per-bin
// term is nu (v + ln2 lg)), formed from one reciprocal and one log2 of the channel product
// without a range test, and nu: the caller keeps the running maximum (mx) of log2 prod and
// recomputes the chunk on the guarded scalar path when it passed kPairLg2Max or the chunk sum is
// not finite.
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ void pair_parts32(const float4 q0, const float4* __restrict__ blk, const Iv2* iv,
                                             float2 ao2, float2 at2, float n1, float n2, float2 Af, float& mx,
                                             float2& v_out, float2& lg_out, float2& nu_out) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    const float4 q1 = blk[1], q2 = blk[2], q3 = blk[3], q4 = blk[4], q5 = blk[5];
    const float2 x = make_float2(q0.x, q0.y), ell = make_float2(q0.z, q0.w), nu = make_float2(q1.x, q1.y);
    const float2 go[3] = {make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
    const float2 gt[3] = {make_float2(q3.x, q3.y), make_float2(q3.z, q3.w), make_float2(q4.x, q4.y)};
    const float2 gh[3] = {make_float2(q4.z, q4.w), make_float2(q5.x, q5.y), make_float2(q5.z, q5.w)};
    float2 p[NSP];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        const float2 t = __fadd2_rn(x, iv[a].nxo);
        p[a] = __ffma2_rn(__ffma2_rn(__ffma2_rn(iv[a].c3, t, iv[a].c2), t, iv[a].c1), t, iv[a].c0);
    }
    float2 eh = make_float2(0.f, 0.f);
    if (HAS_H) {
        const float2 sl = BROKEN ? make_float2(ell.x < 0.f ? n1 : n2, ell.y < 0.f ? n1 : n2) : make_float2(n1, n1);
        const float2 ex = __ffma2_rn(sl, ell, p[C]);
        eh = __fmul2_rn(Af, make_float2(ex2_approx(ex.x), ex2_approx(ex.y)));
    }
    float2 S[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float2 nc = __ffma2_rn(ao2, go[c], __fmul2_rn(at2, gt[c]));
        const float2 e = make_float2(ex2_approx(p[c].x), ex2_approx(p[c].y));
        S[c] = HAS_H ? __ffma2_rn(e, nc, __fmul2_rn(eh, gh[c])) : __fmul2_rn(e, nc);
    }
    float2 prod, num;
    if (C == 3) {
        const float2 p01 = __fmul2_rn(S[0], S[1]);
        prod = __fmul2_rn(p01, S[2]);
        num = __ffma2_rn(S[2], __fadd2_rn(S[0], S[1]), p01);
    } else {
        prod = __fmul2_rn(S[0], S[1]);
        num = __fadd2_rn(S[0], S[1]);
    }
    v_out = __ffma2_rn(num, make_float2(rcp_approx(prod.x), rcp_approx(prod.y)), make_float2(-(float)C, -(float)C));
    lg_out = make_float2(lg2_approx(prod.x), lg2_approx(prod.y));
    nu_out = nu;
    mx = fmax3(mx, lg_out.x, lg_out.y);
}

// The per-bin terms nu (v + ln2 lg) of one pair block (the knot path, where the keep factor can
// change from block to block).
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ float2 pair_term32(const float4 q0, const float4* __restrict__ blk, const Iv2* iv,
                                              float2 ao2, float2 at2, float n1, float n2, float2 Af, float& mx) {
    float2 v, lg, nu;
    pair_parts32<C, HAS_H, BROKEN>(q0, blk, iv, ao2, at2, n1, n2, Af, mx, v, lg, nu);
    return __fmul2_rn(nu, __ffma2_rn(make_float2((float)kLn2, (float)kLn2), lg, v));
}

// Work-item pipeline: the bin table of item k is staged into buffer k % kStages by one bulk
// copy completing on full[k % kStages].  Warps do not wait for one another between items: after
// its last read of a buffer each warp adds one to that buffer's counter, and the warp that
// completes the count (the last reader) issues the copy of the item kStages further on into it.
// Items with one state per thread write their partial sums directly; items that split a state's
// bins over several threads (rows) combine the rows in shared memory between two barriers.
constexpr int kStages = 2;
constexpr int kWarps32 = kThreads32 / 32;

template <int C, bool HAS_H, bool BROKEN, int G>
__global__ void __launch_bounds__(kThreads32, G == 8 ? 4 : (G == 4 ? 5 : 6))
    loglike_fp32_kernel(const WorkItem* __restrict__ items, int n_items, const int32_t* __restrict__ cta_first,
                        const float* __restrict__ rec32,
                        const StateParams* __restrict__ prm, const int32_t* __restrict__ sstat,
                        const float* __restrict__ kxr, const float* __restrict__ srec, int kmax, int nsp,
                        const DatasetDev* __restrict__ ds, double* __restrict__ partial, int* __restrict__ err,
                        int tile_bins, unsigned wait_limit, int skip_copies) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    constexpr int U = G / 2;                  // pair blocks per iteration of the knot-free loop
    constexpr int kChunkPairs = 32;           // pair blocks per FP32 partial sum (64 bins)
    constexpr unsigned kLocated = 1u << 31;   // s_hm: this thread's intervals have been located
    constexpr unsigned kSplineBits = (1u << NSP) - 1u;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ unsigned s_done[kStages];
    __shared__ int s_fail;                    // a bounded wait of this CTA ran out: stage nothing more
    __shared__ float2 red[kThreads32];
    // per thread: right end and index of the current interval of each spline, and the bits of
    // the ill-conditioned ones (touched only at knots, so they live here and not in registers)
    __shared__ float s_xr[NSP][kThreads32];
    __shared__ int s_jj[NSP][kThreads32];
    __shared__ unsigned s_hm[kThreads32];     // bit a: spline a ill-conditioned; kLocated: set up
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const size_t stage_floats = (size_t)tile_bins * kRec;
    // the compensated kernel, launched next as a programmatic dependent, may place its CTAs as
    // soon as this grid's CTAs leave SMs (it does not read what this kernel writes)
    asm volatile("griddepcontrol.launch_dependents;");
    s_hm[tid] = 0u;
    // the CTA's items, [cta_first[c], cta_first[c + 1]) of the work list: with many items per
    // CTA a contiguous, cost-balanced block of the (dataset, state chunk, tile)-ordered list
    // (consecutive items are mostly consecutive tiles of the same states, whose intervals carry
    // over); with few, the items a longest-first assignment of the knot-aware costs gave the CTA
    // (without cta_first: every gridDim.x-th item)
    const int step = cta_first ? 1 : (int)gridDim.x;
    const int i_begin = cta_first ? cta_first[blockIdx.x] : (int)blockIdx.x;
    const int i_end = cta_first ? cta_first[blockIdx.x + 1] : n_items;
    auto stage = [&](int q, int item) {   // one bulk copy of item's bin table into buffer q
        const WorkItem w = items[item];
        const unsigned bytes = (unsigned)w.nb * kRec * sizeof(float);
        mbar_expect_tx(&full[q], bytes);
        bulk_copy_g2s(reinterpret_cast<float*>(smem) + q * stage_floats, rec32 + (w.bin0 >> 1) * kPairRec, bytes,
                      &full[q]);
    };
    if (tid == 0) {
        s_fail = 0;
        for (int q = 0; q < kStages; ++q) {
            mbar_init(&full[q], 1);
            s_done[q] = 0u;
        }
        mbar_fence_init();
        // skip_copies (a test of the timeout path only): no copy is issued, so every wait runs
        // out with nothing in flight
        if (!skip_copies)
            for (int q = 0; q < kStages; ++q)
                if (i_begin + q * step < i_end) stage(q, i_begin + q * step);
    }
    __syncthreads();
    // per spline, the current interval's cubic duplicated into register pairs (the scalar path
    // reads the .x halves); xmin = the nearest right knot over the splines.  An ill-conditioned
    // interval (T > kRobustT, routed states only) is loaded as the zero cubic, which keeps its
    // bins' arithmetic benign, and sets its bit in s_hm; keep2 = 0 while any bit is set, 1
    // otherwise, and scales each bin's contribution.  All of it carries over to the next item
    // when that is the next tile of the same state chunk (bins only move right).
    Iv2 iv2[NSP];
    float xmin = INFINITY;
    float2 keep2 = make_float2(1.f, 1.f);
    int k = 0;
    for (int it = i_begin; it < i_end; it += step, ++k) {
        const int b = k % kStages;
        const WorkItem w = items[LISA_IDX(it, n_items)];
        // buffer b's barrier has completed k / kStages phases before this item's
        const bool ok = mbar_wait_bounded(&full[b], (unsigned)(k / kStages) & 1u, wait_limit);
        // a wait that ran out: this thread skips the item (its table may never arrive or be
        // partly written) and raises the flag (finalize turns every log L into NaN and
        // lisa_workspace_status reports LISA_ERR_TIMEOUT); the CTA stages no further copy, since
        // the late one could still be landing in this buffer, and its later waits run out too
        if (!ok) {
            s_fail = 1;
            atomicOr(err, kErrTimeout);
        }
        const float* tb = reinterpret_cast<const float*>(smem) + b * stage_floats;
        const float4* tb4 = reinterpret_cast<const float4*>(tb);
        bool carry = false;
        if (k > 0) {
            const WorkItem pw = items[it - step];
            carry = w.ds == pw.ds && w.s0 == pw.s0 && w.tile == pw.tile + 1;
        }
        const int sc = w.sc;
        const int R = kThreads32 / sc;
        const int ls = tid & (sc - 1);
        const int r = tid / sc;
        const int s = w.s0 + ls;
        // every valid state, routed ones included: the bins of an ill-conditioned interval are
        // masked out here (the compensated kernel adds them), all other bins are summed here
        const bool active = ok && ls < w.ns && (sstat[s] & kUserBits) == 0;
        ff accf = {0.f, 0.f};
        if (active) {
            const int np = w.nb >> 1;                          // pair blocks in the tile
            const int plo = (r * np) / R, phi = ((r + 1) * np) / R;
            if (plo < phi) {
                const float4 q0 = __ldg(reinterpret_cast<const float4*>(prm + s));
                const float ao2 = q0.x, at2 = q0.y, Af = HAS_H ? q0.z : 0.f, n1 = q0.w;
                const float n2 = BROKEN ? __ldg(&prm[s].n2) : n1;
                const float2 ao2_2 = make_float2(ao2, ao2), at2_2 = make_float2(at2, at2), Af2 = make_float2(Af, Af);
                // the records of this state's splines: spline a, interval j at rec(a, j)
                auto rec = [&](int a, int j) {
                    return reinterpret_cast<const float4*>(
                        srec + (((int64_t)s * nsp + a) * (int64_t)(kmax + 1) + LISA_IDX(j, kmax + 1)) * kSplineRec32);
                };
                // installs interval j of spline a from its record (A = xr, xo, c0, c1; B = c2, c3,
                // xl, T)
                auto install = [&](int a, int j, float4 A, float4 B) {
                    s_xr[a][tid] = A.x;
                    s_jj[a][tid] = j;
                    unsigned hm = s_hm[tid];
                    if (B.w <= (float)kRobustT) {
                        iv2[a] = Iv2{make_float2(-A.y, -A.y), make_float2(A.z, A.z), make_float2(A.w, A.w),
                                     make_float2(B.x, B.x), make_float2(B.y, B.y)};
                        hm &= ~(1u << a);
                    } else {
                        const float2 z = make_float2(0.f, 0.f);
                        iv2[a] = Iv2{z, z, z, z, z};
                        hm |= 1u << a;
                    }
                    s_hm[tid] = hm;
                    keep2 = (hm & kSplineBits) ? make_float2(0.f, 0.f) : make_float2(1.f, 1.f);
                };
                // moves spline a to the interval holding x: one dependent load per interval
                // passed (the whole record at once); the last interval's right end is +inf, and
                // the index never leaves the spline's kmax + 1 record slots
                auto advance = [&](int a, float x) {
                    if (x >= s_xr[a][tid]) {
                        int j = s_jj[a][tid];
                        float4 A, B;
                        do {
                            ++j;
                            A = __ldg(rec(a, j));
                            B = __ldg(rec(a, j) + 1);
                        } while (x >= A.x && j < kmax);
                        install(a, j, A, B);
                    }
                };
                auto nearest = [&]() {
                    float m = s_xr[0][tid];
#pragma unroll
                    for (int a = 1; a < NSP; ++a) m = fminf(m, s_xr[a][tid]);
                    return m;
                };
                // the interval of each spline holding x: the count of right ends <= x in the
                // spline's right-end table (independent 16-byte loads), then its record
                auto locate = [&](float x) {
                    s_hm[tid] = kLocated;
                    const int kxs = kxr_stride(kmax);
#pragma unroll
                    for (int a = 0; a < NSP; ++a) {
                        const float4* kq = reinterpret_cast<const float4*>(kxr + ((int64_t)s * nsp + a) * kxs);
                        int j = 0;
#pragma unroll 4
                        for (int q = 0; q < kxs / 4; ++q) {
                            const float4 v = __ldg(kq + q);
                            j += (v.x <= x) + (v.y <= x) + (v.z <= x) + (v.w <= x);
                        }
                        j = min(j, kmax);
                        install(a, j, __ldg(rec(a, j)), __ldg(rec(a, j) + 1));
                    }
                    xmin = nearest();
                };
                // one bin on the scalar path (at knots, and for the guarded redo): advance this
                // thread's intervals if the bin passed a knot, then the guarded term
                auto scalar_bin = [&](int i) {
                    const float x = fld(tb, i, 0);
                    if (x >= xmin) {
#pragma unroll
                        for (int a = 0; a < NSP; ++a) advance(a, x);
                        xmin = nearest();
                    }
                    return keep2.x * bin_term32p<C, HAS_H, BROKEN>(tb, i, iv2, ao2, at2, n1, n2, Af);
                };
                // intervals carry over from this thread's previous item when it held the
                // preceding tile of the same states (a thread whose row was empty there keeps
                // those of an earlier tile, which lie to the left: advancing finds the new ones)
                if (!(carry && (s_hm[tid] & kLocated))) locate(fld(tb, 2 * plo, 0));
                int ip = plo;
                while (ip < phi) {
                    const int pc0 = ip;
                    const int pcend = min(ip + kChunkPairs, phi);
                    const float4* blk = tb4 + LISA_IDX(ip, np) * (kPairRec / 4);
                    float2 acc2 = make_float2(0.f, 0.f);
                    float mx = -INFINITY;
                    // one decision per chunk for the warp: no lane passes a knot inside it (the
                    // common case away from the lowest frequencies) -> no checks at all
                    const float x_last = tb4[(pcend - 1) * (kPairRec / 4)].y;
                    if (!__any_sync(__activemask(), x_last >= xmin)) {
                        // keep2 is constant here: the nu-weighted sums of v and of lg run apart,
                        // ln2 and keep2 applied once for the chunk
                        float2 accv = make_float2(0.f, 0.f), accl = make_float2(0.f, 0.f);
                        for (; ip + U <= pcend; ip += U, blk += U * (kPairRec / 4)) {
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const float4* pb = blk + u * (kPairRec / 4);
                                float2 v, lg, nu;
                                pair_parts32<C, HAS_H, BROKEN>(pb[0], pb, iv2, ao2_2, at2_2, n1, n2, Af2, mx, v, lg,
                                                               nu);
                                accv = __ffma2_rn(nu, v, accv);
                                accl = __ffma2_rn(nu, lg, accl);
                            }
                        }
#pragma unroll 1
                        for (; ip < pcend; ++ip, blk += kPairRec / 4) {
                            float2 v, lg, nu;
                            pair_parts32<C, HAS_H, BROKEN>(blk[0], blk, iv2, ao2_2, at2_2, n1, n2, Af2, mx, v, lg, nu);
                            accv = __ffma2_rn(nu, v, accv);
                            accl = __ffma2_rn(nu, lg, accl);
                        }
                        acc2 = __fmul2_rn(keep2, __ffma2_rn(make_float2((float)kLn2, (float)kLn2), accl, accv));
                    } else {
                        // pair block by pair block: a lane whose block reaches a knot takes its two
                        // bins on the scalar path (advancing its intervals between them), the
                        // others stay packed
#pragma unroll 1
                        for (; ip < pcend; ++ip, blk += kPairRec / 4) {
                            const float4 q0 = blk[0];
                            if (q0.y >= xmin) {
                                acc2.x += scalar_bin(2 * ip);
                                acc2.x += scalar_bin(2 * ip + 1);
                            } else {
                                acc2 = __ffma2_rn(keep2, pair_term32<C, HAS_H, BROKEN>(q0, blk, iv2, ao2_2, at2_2, n1,
                                                                                       n2, Af2, mx),
                                                  acc2);
                            }
                        }
                    }
                    if (!(mx <= kPairLg2Max && fabsf(acc2.x + acc2.y) < INFINITY)) {
                        // a channel product passed the range of the one-reciprocal form (or the
                        // sum overflowed): redo the chunk bin by bin on the guarded path,
                        // intervals re-found at its start
                        locate(fld(tb, 2 * pc0, 0));
                        acc2 = make_float2(0.f, 0.f);
#pragma unroll 1
                        for (int i = 2 * pc0; i < 2 * pcend; ++i) acc2.x += scalar_bin(i);
                    }
                    accf = ff_add(accf, two_sum(acc2.x, acc2.y));
                }
            }
        }
        const DatasetDev& D = ds[w.ds];
        if (R == 1) {
            if (active)
                partial[D.pbase + (int64_t)(s - D.s0) * D.ntiles + LISA_IDX(w.tile, D.ntiles)] =
                    (double)accf.hi + (double)accf.lo;
        } else {
            red[tid] = make_float2(accf.hi, accf.lo);
            __syncthreads();
            if (r == 0 && active) {
                ff sum = {red[ls].x, red[ls].y};
                for (int q = 1; q < R; ++q) sum = ff_add(sum, ff{red[ls + q * sc].x, red[ls + q * sc].y});
                partial[D.pbase + (int64_t)(s - D.s0) * D.ntiles + LISA_IDX(w.tile, D.ntiles)] =
                    (double)sum.hi + (double)sum.lo;
            }
            __syncthreads();   // red is rewritten by the next item
        }
        // release buffer b: the last of the CTA's warps to finish reading it stages item
        // it + kStages * step into it (the count of buffer b reaches kWarps32 * (k / kStages + 1))
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const unsigned done = atomicAdd(&s_done[b], 1u) + 1u;
            if (done == kWarps32 * (unsigned)(k / kStages + 1)) {
                __threadfence_block();
                const int nx = it + kStages * step;
                if (nx < i_end && !skip_copies && !*reinterpret_cast<volatile int*>(&s_fail)) {
                    fence_proxy_async();
                    stage(b, nx);
                }
            }
        }
    }
}


// ---- compensated path: the ill-conditioned intervals of the states the setup routed ------
struct IvR {
    float xr, T;
    ff xo, c[4];
    const float* base;
    int j, last;
};
__device__ __forceinline__ void load_ivr(IvR& v) {
    const float4* r = reinterpret_cast<const float4*>(v.base + (size_t)v.j * kSplineRec32);
    const float4 A = __ldg(r), B = __ldg(r + 1), Cq = __ldg(r + 2), Dq = __ldg(r + 3);
    // A = (xr, xo, c0, c1), B = (c2, c3, xl, T), Cq = (xo_lo, c0_lo, c1_lo, c2_lo), Dq.x = c3_lo
    v.xr = A.x;
    v.T = B.w;
    v.xo = {A.y, Cq.x};
    v.c[0] = {A.z, Cq.y};
    v.c[1] = {A.w, Cq.z};
    v.c[2] = {B.x, Cq.w};
    v.c[3] = {B.y, Dq.x};
}

// log2 of a positive float as an exact float-float pair (exponent, log2 of the mantissa):
// the approximation then only sees arguments in [1, 2), where its absolute error is smallest.
__device__ __forceinline__ ff lg2_split(float v) {
    if (!(v >= 1.17549435e-38f) || !(v < INFINITY)) return ff{lg2_approx(v), 0.f};  // 0, inf, NaN, subnormal
    const int b = __float_as_int(v);
    const float e = (float)(((b >> 23) & 0xff) - 127);
    const float m = __int_as_float((b & 0x007fffff) | 0x3f800000);
    return fast_two_sum(e, lg2_approx(m));
}

// log2 of a positive sum given the log2 of its two parts (either may be -inf).
__device__ __forceinline__ ff log2_sum(ff a, ff b) {
    if (!(b.hi > -INFINITY)) return a;
    if (!(a.hi > -INFINITY)) return b;
    const ff big = a.hi >= b.hi ? a : b;
    const float d = fabsf(a.hi - b.hi);
    const float corr = lg2_approx(1.0f + ex2_approx(-d));
    return ff_add(big, ff{corr, 0.f});
}

// 1/S + ln S from lS = log2 S (float-float).  Inside |lS| < 100 the result is a float-float
// (2^-lS is ex2 of the fractional part scaled by an exact power of two); outside, nu times the
// contribution is added to `far` in FP64 (S beyond the FP32 range: rare, so the FP64 pipe is
// only used there).
__device__ __forceinline__ ff inv_plus_log(ff lS, float nu, double& far) {
    const ff kLn2ff = {0.693147182f, -1.90465421e-09f};
    if (lS.hi > -100.f && lS.hi < 100.f) {
        const float n = rintf(lS.hi);
        const float f = (lS.hi - n) + lS.lo;
        const float inv = ex2_approx(-f) * __int_as_float((127 - (int)n) << 23);
        return ff_add(ff_mul(lS, kLn2ff), ff{inv, 0.f});
    }
    double v;
    if (!(lS.hi > -1.0e6f)) {
        v = INFINITY;                                     // S = 0 (or NaN)
    } else if (!(lS.hi < 1.0e6f)) {
        v = (double)lS.hi * kLn2;                         // S overflows: 1/S = 0
    } else {
        const float n = rintf(lS.hi);
        const float f = (lS.hi - n) + lS.lo;
        v = ldexp((double)ex2_approx(-f), -(int)n) + kLn2 * ((double)lS.hi + (double)lS.lo);
    }
    if (nu != 0.f) far += (double)nu * v;                 // a padding bin (nu = 0) adds nothing
    return ff{0.f, 0.f};
}

// log2 of FP64's overflow threshold: 10^P overflows double precision from P = 1024 in log2 units
constexpr float kP2Overflow = 1024.0f;

// Compensated kernel staging: each warp stages its tile in chunks of kRobChunk bins into its own
// shared-memory slice (the pair-block table by one bulk asynchronous copy, the low parts of x and
// ell by lane loads), then evaluates the chunk from shared memory.  8 warps per CTA: two CTAs
// fill an SM's shared memory (and registers), 16 warps.
constexpr int kRobWarps = 8;
constexpr int kRobChunk = 256;                                    // even
constexpr int kRobChunkF4 = kRobChunk / 2 * (kPairRec / 4);       // float4 of table per chunk
constexpr int kRobSliceF4 = kRobChunkF4 + 2 * kRobChunk / 4;      // + x lo, ell lo
constexpr size_t kRobSmem = (size_t)kRobWarps * kRobSliceF4 * sizeof(float4);

// One bin of a routed state (i: bin within the staged chunk tb, with the low parts of x and ell
// in xs / es), evaluated only if one of its spline intervals is ill-conditioned (the fused kernel
// masks exactly those bins and sums all others): spline values as float-float sums on the
// ill-conditioned intervals, then the moderate-exponent or the log-domain term.
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ void robust_bin(const float* __restrict__ tb, int i, const float* __restrict__ xs,
                                           const float* __restrict__ es, IvR* iv, float ao2, float at2, ff n1,
                                           ff n2, ff lA, ff& acc_ff, double& far) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    const float x_hi = fld(tb, i, 0);
    bool hard = false;
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        while (x_hi >= iv[a].xr && iv[a].j < iv[a].last) {
            ++iv[a].j;
            load_ivr(iv[a]);
        }
        hard |= !(iv[a].T <= (float)kRobustT);
    }
    if (!hard) return;
    const float nu = fld(tb, i, 2);
    const ff x = {x_hi, xs[i]};
    ff P[NSP];
#pragma unroll
    for (int a = 0; a < NSP; ++a) {
        if (!(iv[a].T <= (float)kRobustT)) {
            const ff tt = ff_add(x, ff{-iv[a].xo.hi, -iv[a].xo.lo});
            ff p = iv[a].c[3];
            p = ff_add(ff_mul(p, tt), iv[a].c[2]);
            p = ff_add(ff_mul(p, tt), iv[a].c[1]);
            P[a] = ff_add(ff_mul(p, tt), iv[a].c[0]);
        } else {
            const float tt = x.hi - iv[a].xo.hi;
            P[a] = ff{fmaf(fmaf(fmaf(iv[a].c[3].hi, tt, iv[a].c[2].hi), tt, iv[a].c[1].hi), tt, iv[a].c[0].hi), 0.f};
        }
    }
    // the definition's 10^P as FP64 evaluates it: beyond 2^1024 (P >= 308.25 decades) the PSD is
    // not finite, and the state's log L is -inf in every precision (as in the FP64 path)
    bool over = false;
#pragma unroll
    for (int a = 0; a < NSP; ++a) over |= !(P[a].hi < kP2Overflow);
    if (over) {
        if (nu != 0.f) far = INFINITY;
        return;
    }
    const ff ell = {fld(tb, i, 1), es[i]};
    ff lEh = {-INFINITY, 0.f};
    if (HAS_H) {
        const ff sl = BROKEN ? (ell.hi < 0.f ? n1 : n2) : n1;
        lEh = ff_add(ff_add(P[C], ff_mul(sl, ell)), lA);
    }
    bool moderate = true;
#pragma unroll
    for (int c = 0; c < C; ++c) moderate &= fabsf(P[c].hi) < 60.f;
    if (HAS_H) moderate &= fabsf(P[C].hi) < 60.f && lEh.hi > -120.f && lEh.hi < 60.f;
    if (moderate) {
        // exponents within FP32 range: 2^(hi + lo) = ex2(hi) (1 + lo ln2), accurate to a few ulp
        // because hi is exact; then the ordinary FP32 term
        float S[C];
        const float eh = HAS_H ? ex2_approx(lEh.hi) * fmaf(lEh.lo, (float)kLn2, 1.f) : 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float E = ex2_approx(P[c].hi) * fmaf(P[c].lo, (float)kLn2, 1.f);
            const float N = fmaf(ao2, fld(tb, i, 3 + c), at2 * fld(tb, i, 6 + c));
            S[c] = HAS_H ? fmaf(E, N, eh * fld(tb, i, 9 + c)) : E * N;
        }
        acc_ff = ff_add(acc_ff, ff{term_from_S<C>(S, nu), 0.f});
        return;
    }
    ff term = {-(float)C, 0.f};
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float N = fmaf(ao2, fld(tb, i, 3 + c), at2 * fld(tb, i, 6 + c));
        const ff lN = lg2_split(N);
        const ff lNE = (lN.hi > -INFINITY && lN.hi < INFINITY) ? ff_add(P[c], lN) : lN;
        ff lS = lNE;
        if (HAS_H) {
            const ff lG = lg2_split(fld(tb, i, 9 + c));
            const ff lH = (lG.hi > -INFINITY && lG.hi < INFINITY) ? ff_add(lEh, lG) : lG;
            lS = log2_sum(lNE, lH);
        }
        term = ff_add(term, inv_plus_log(lS, nu, far));
    }
    acc_ff = ff_add(acc_ff, ff_mul(term, ff{nu, 0.f}));
}

// One warp per unit (routed state, tile) of the work list the state-parameter kernel built, on a
// persistent grid, units assigned statically (warp w takes units w, w + warps, ...).  As soon as the warp knows its tile it starts one bulk asynchronous copy of
// the tile's first chunk of the pair-block table into its shared-memory slice; meanwhile it
// locates each spline's interval at the tile's first bin with one ballot over the interval right
// ends (lane k holds interval k) and loads the low parts of x and ell of the chunk (each lane
// reads back only the entries it wrote).  Lane l takes bins l, l + 32, ... of a chunk, so a
// lane's bins come in increasing order and its intervals only move right.  The tile's sum of
// ill-conditioned bins is added to the (state, tile) partial the fused kernel wrote (one warp per
// partial: deterministic).
template <int C, bool HAS_H, bool BROKEN>
__device__ __forceinline__ void robust_units(const unsigned long long* __restrict__ rcount,
                                             const RobustEntry* __restrict__ rlist, int tile_bins,
                                             const float* __restrict__ rec32, const float* __restrict__ xlo32,
                                             const float* __restrict__ elllo32, const StateParams* __restrict__ prm,
                                             const int32_t* __restrict__ nint, const float* __restrict__ srec,
                                             int kmax, int nsp, double* __restrict__ rpart, int* __restrict__ err,
                                             unsigned wait_limit) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
    extern __shared__ float4 rsm[];
    __shared__ __align__(8) uint64_t rbar[kRobWarps];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4* slice = rsm + warp * kRobSliceF4;
    const float* tb = reinterpret_cast<const float*>(slice);
    float* xs = reinterpret_cast<float*>(slice + kRobChunkF4);
    float* es = xs + kRobChunk;
    uint64_t* bar = &rbar[warp];
    const unsigned long long cnt = __ldg(rcount);
    const int n_ent = (int)(cnt >> 32);
    const int64_t units = (int64_t)(cnt & 0xffffffffull);
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (wg >= units) return;   // warp-uniform
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    unsigned phase = 0;
    // a static assignment: handing units out through one global counter was slower here (the
    // requests of all warps serialise on its address)
    for (int64_t u = wg; u < units; u += nw) {
        // the entry holding unit u: the last one whose first unit is <= u
        int lo = 0, hi = n_ent - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)__ldg(&rlist[mid].u0) <= u) lo = mid; else hi = mid - 1;
        }
        const int4 ea = __ldg(reinterpret_cast<const int4*>(rlist + lo));
        const int4 eb = __ldg(reinterpret_cast<const int4*>(rlist + lo) + 1);
        const int s = ea.x;
        const int k_t = (int)(u - (int64_t)(uint32_t)ea.z);   // tile t0 + k_t
        const int64_t b0 = (int64_t)(((uint64_t)(uint32_t)eb.y << 32) | (uint32_t)eb.x) + (int64_t)k_t * tile_bins;
        const int nb = k_t == ea.w - 1 ? eb.w : tile_bins;
        const float* tbase = rec32 + (b0 >> 1) * kPairRec;   // b0 even
        __syncwarp();   // every lane is done with the previous unit's table
        if (lane == 0) {
            const unsigned bytes = (unsigned)min(kRobChunk, nb) * kRec * sizeof(float);   // even bin count
            fence_proxy_async();
            mbar_expect_tx(bar, bytes);
            bulk_copy_g2s(slice, tbase, bytes, bar);
        }
        const float4 q0 = __ldg(reinterpret_cast<const float4*>(prm + s));
        const float4 q1 = __ldg(reinterpret_cast<const float4*>(prm + s) + 1);
        const float4 q2 = __ldg(reinterpret_cast<const float4*>(prm + s) + 2);
        const float ao2 = q0.x, at2 = q0.y;
        const ff n1 = {q0.w, q1.w};
        const ff n2 = BROKEN ? ff{q1.x, q2.x} : n1;
        const ff lA = {q1.y, q1.z};
        // intervals at the tile's first bin: j = number of right ends <= x among intervals
        // 0 .. last-1 (the right ends increase with j)
        const float xf = __ldg(tbase);
        IvR iv[NSP];
        float xr0[NSP];
#pragma unroll
        for (int a = 0; a < NSP; ++a) {
            const int64_t sp = (int64_t)s * nsp + a;
            iv[a].base = srec + sp * (int64_t)(kmax + 1) * kSplineRec32;
            iv[a].last = __ldg(nint + sp) - 1;
            xr0[a] = lane <= kmax ? __ldg(iv[a].base + (size_t)lane * kSplineRec32) : INFINITY;
        }
#pragma unroll
        for (int a = 0; a < NSP; ++a) {
            int j = __popc(__ballot_sync(0xffffffffu, lane < iv[a].last && xr0[a] <= xf));
            if (kmax >= 32) {   // warp-uniform
                const int k = 32 + lane;
                const float xr1 = k <= kmax ? __ldg(iv[a].base + (size_t)k * kSplineRec32) : INFINITY;
                j += __popc(__ballot_sync(0xffffffffu, k < iv[a].last && xr1 <= xf));
            }
            iv[a].j = j;
            load_ivr(iv[a]);
        }
        ff acc_ff = {0.f, 0.f};
        double far = 0.0;
        for (int c0 = 0; c0 < nb; c0 += kRobChunk) {
            const int nbc = min(kRobChunk, nb - c0);
            if (c0 > 0) {
                __syncwarp();   // every lane is done with the previous chunk's table
                if (lane == 0) {
                    const unsigned bytes = (unsigned)nbc * kRec * sizeof(float);
                    fence_proxy_async();
                    mbar_expect_tx(bar, bytes);
                    bulk_copy_g2s(slice, tbase + (c0 >> 1) * kPairRec, bytes, bar);
                }
            }
            float vx[kRobChunk / 32], ve[kRobChunk / 32];
#pragma unroll
            for (int k = 0; k < kRobChunk / 32; ++k) {
                const int q = lane + 32 * k;
                vx[k] = q < nbc ? __ldg(xlo32 + b0 + c0 + q) : 0.f;
                ve[k] = q < nbc ? __ldg(elllo32 + b0 + c0 + q) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kRobChunk / 32; ++k) {
                xs[lane + 32 * k] = vx[k];
                es[lane + 32 * k] = ve[k];
            }
            const bool ok = mbar_wait_bounded(bar, phase, wait_limit);
            if (!__all_sync(0xffffffffu, ok)) {
                // timed out: raise the flag, let the warp's one copy in flight land, then stop
                if (lane == 0) {
                    atomicOr(err, kErrTimeout);
                    mbar_wait_bounded(bar, phase, wait_limit);
                }
                return;
            }
            phase ^= 1;
            for (int i = lane; i < nbc; i += 32)
                robust_bin<C, HAS_H, BROKEN>(tb, i, xs, es, iv, ao2, at2, n1, n2, lA, acc_ff, far);
        }
        // warp sum: float-float tree; the FP64 spill-over only when some lane has one
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            acc_ff = ff_add(acc_ff, ff{__shfl_down_sync(0xffffffffu, acc_ff.hi, o),
                                       __shfl_down_sync(0xffffffffu, acc_ff.lo, o)});
        if (__any_sync(0xffffffffu, far != 0.0))
            for (int o = 16; o > 0; o >>= 1) far += __shfl_down_sync(0xffffffffu, far, o);
        const double acc = ((double)acc_ff.hi + (double)acc_ff.lo) + far;
        if (lane == 0) rpart[u] = acc;
    }
}

template <int C, bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(kRobWarps * 32, 2)
    loglike_robust_kernel(const unsigned long long* __restrict__ rcount, const RobustEntry* __restrict__ rlist,
                          int tile_bins, const float* __restrict__ rec32, const float* __restrict__ xlo32,
                          const float* __restrict__ elllo32, const StateParams* __restrict__ prm,
                          const int32_t* __restrict__ nint, const float* __restrict__ srec, int kmax, int nsp,
                          double* __restrict__ rpart, int* __restrict__ err, unsigned wait_limit) {
    robust_units<C, HAS_H, BROKEN>(rcount, rlist, tile_bins, rec32, xlo32, elllo32, prm, nint, srec, kmax, nsp, rpart,
                                   err, wait_limit);
    // launched as a programmatic dependent of the fused kernel, so that its CTAs can start on SMs
    // the fused kernel's CTAs have left; it reads nothing the fused kernel writes, but it does not
    // complete before the fused kernel has (the finalize kernel after it then sees both)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}


// ---- plain FP64 path: the same decomposition, FP64 throughout, library exp10 / exp2 / log ----

template <int C, bool HAS_H, bool BROKEN>
__global__ void __launch_bounds__(kThreads)
    loglike_fp64_kernel(const WorkItem* __restrict__ items, int n_items, const double* __restrict__ rec64,
                        const double* __restrict__ theta, const int32_t* __restrict__ sstat,
                        const int32_t* __restrict__ nint, const double* __restrict__ srec, int kmax, int nsp,
                        const DatasetDev* __restrict__ ds, double* __restrict__ partial) {
    constexpr int NSP = C + (HAS_H ? 1 : 0);
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
                const double* rb = rec64 + (w.bin0 + lo) * kRec;
                for (int a = 0; a < NSP; ++a) {
                    const int64_t sp = (int64_t)s * nsp + a;
                    base[a] = srec + sp * (int64_t)(kmax + 1) * kSplineRec;
                    last[a] = nint[sp] - 1;
                    j[a] = find_interval<double, kSplineRec, 0>(base[a], nint[sp], __ldg(rb));
                    const double* q = base[a] + (size_t)LISA_IDX(j[a], kmax + 1) * kSplineRec;
                    xl[a] = q[0]; xr[a] = q[1]; ca[a] = q[2]; cb[a] = q[3]; cc[a] = q[4]; cd[a] = q[5];
                }
                for (int i = lo; i < hi; ++i) {
                    const double* q = rec64 + (w.bin0 + i) * kRec;
                    const double x = __ldg(q), ell = __ldg(q + 1), nu = __ldg(q + 2);
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
                    double eh = 0.0;
                    if (HAS_H) {
                        const double sl = BROKEN ? (ell < 0.0 ? n1 : n2) : n1;
                        eh = exp10(lA + P[C]) * exp2(sl * ell);
                    }
                    double term = 0.0;
                    for (int c = 0; c < C; ++c) {
                        const double Sc = (ao2 * __ldg(q + 3 + c) + at2 * __ldg(q + 6 + c)) * exp10(P[c]) +
                                          (HAS_H ? eh * __ldg(q + 9 + c) : 0.0);
                        term += 1.0 / Sc + log(Sc);
                    }
                    acc += nu * term;
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

// Per state (one warp): fixed-order sum of its tiles' partials (lane-strided, then a shuffle
// tree) plus the dataset constants.
__global__ void finalize_kernel(int S, const int32_t* __restrict__ state_ds, const DatasetDev* __restrict__ ds,
                                const int32_t* __restrict__ sstat, const double* __restrict__ partial,
                                const int32_t* __restrict__ rent, const RobustEntry* __restrict__ rlist,
                                const double* __restrict__ rpart, const int* __restrict__ err, int fp32,
                                double* __restrict__ out) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= S) return;   // uniform per warp
    if (sstat[s] & kUserBits) {
        if (lane == 0) out[s] = -INFINITY;
        return;
    }
    const DatasetDev& D = ds[state_ds[s]];
    const double* p = partial + D.pbase + (int64_t)(s - D.s0) * D.ntiles;
    double sum = 0.0;
    for (int t = lane; t < D.ntiles; t += 32) sum += p[t];
    // FP32 mode: the compensated kernel's sums of this state's units, if it has any
    const int e = fp32 ? rent[s] : -1;
    if (e >= 0) {
        const int4 ea = __ldg(reinterpret_cast<const int4*>(rlist + e));   // (s, t0, u0, nt)
        const int64_t u0 = (int64_t)(uint32_t)ea.z;
        for (int u = lane; u < ea.w; u += 32) sum += rpart[u0 + u];
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        double L = fp32 ? (-sum - D.Cnu + D.K) : (-sum + D.K);
        if (!isfinite(L)) L = -INFINITY;
        if (*err) L = NAN;
        out[s] = L;
    }
}

// Model PSD in physical units, FP64: one thread per (state, bin).
template <int C>
__global__ void model_psd_kernel(const int32_t* __restrict__ state_ds, const DatasetDev* __restrict__ ds,
                                 const double* __restrict__ rec64, const double* __restrict__ P, int64_t n_bins,
                                 const double* __restrict__ theta, const int32_t* __restrict__ sstat,
                                 const int32_t* __restrict__ nint, const double* __restrict__ srec, int kmax,
                                 int nsp, int has_h, int broken, double* __restrict__ out) {
    const int s = blockIdx.y;
    const DatasetDev& D = ds[state_ds[s]];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nbins) return;
    double* o = out + D.psd_base + (int64_t)(s - D.s0) * C * D.nbins;
    if (sstat[s] & kUserBits) {
        for (int c = 0; c < C; ++c) o[(int64_t)c * D.nbins + i] = NAN;
        return;
    }
    const int64_t g = D.bin0 + i;            // padded table index
    const int64_t gr = D.rbin0 + i;          // caller's bin index
    const double* q = rec64 + g * kRec;
    const double x = q[0], ell = q[1];
    const double* th = theta + (size_t)s * LISA_N_THETA;
    double Pv[4];
    for (int a = 0; a < C + has_h; ++a) {   // the noise and SGWB splines (not the correlations)
        const int64_t sp = (int64_t)s * nsp + a;
        const double* base = srec + sp * (int64_t)(kmax + 1) * kSplineRec;
        const int j = find_interval<double, kSplineRec, 0>(base, nint[sp], x);
        const double* z = base + (size_t)LISA_IDX(j, kmax + 1) * kSplineRec;
        const double t = x - z[0];
        Pv[a] = z[2] + t * (z[3] + t * (z[4] + t * z[5]));
    }
    double eh = 0.0;
    if (has_h) {
        const double sl = (broken && ell >= 0.0) ? th[4] : th[3];
        eh = exp10(th[2] + Pv[C]) * exp2(sl * ell);
    }
    for (int c = 0; c < C; ++c) {
        const double Sc = (th[0] * th[0] * q[3 + c] + th[1] * th[1] * q[6 + c]) * exp10(Pv[c]) + eh * q[9 + c];
        o[(int64_t)c * D.nbins + i] = Sc * P[(int64_t)c * n_bins + gr];
    }
}

template <class K>
int grid_for(K kernel, const lisa_data* d, size_t smem, int threads) {
    int per_sm = d->tiling.ctas_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int64_t g = (int64_t)d->n_sm * per_sm;
    if (g > d->n_items) g = d->n_items;
    return (int)(g < 1 ? 1 : g);
}

template <int C, bool H, bool B, int G>
cudaError_t launch_fp32_g(const lisa_data* d, const StateParams* prm, const int32_t* sstat, const int32_t* nint,
                          const float* kxr, unsigned long long* rcount, const RobustEntry* rlist, const float* srec,
                          int kmax,
                          double* partial, double* rpart, int* err, cudaStream_t sm, bool prof) {
    auto kern = loglike_fp32_kernel<C, H, B, G>;
    const size_t smem = 2 * (size_t)d->tiling.tile_bins * kRec * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<d->fgrid, kThreads32, smem, sm>>>(d->d_items, (int)d->n_items, d->d_cta_first,
                                              d->d_rec32, prm, sstat, kxr, srec, kmax, d->nsp, d->d_ds, partial, err,
                                              d->tiling.tile_bins, d->wait_limit, d->test_skip_copies);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_mark(d, prof, 1, sm);
    // compensated kernel for the routed states' work list (its warps return at once when the list
    // is empty)
    auto rk = loglike_robust_kernel<C, H, B>;
    e = cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRobSmem);
    if (e != cudaSuccess) return e;
    // launched as a programmatic dependent of the fused kernel (except when each kernel is timed
    // on its own), so that its CTAs take the SMs the fused kernel's last CTAs leave idle
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d->rgrid);
    cfg.blockDim = dim3(kRobWarps * 32);
    cfg.dynamicSmemBytes = kRobSmem;
    cfg.stream = sm;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = prof ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, rk, rcount, rlist, d->tiling.tile_bins, (const float*)d->d_rec32,
                           (const float*)d->d_xlo32, (const float*)d->d_elllo32, prm, nint, srec, kmax, d->nsp, rpart,
                           err, d->wait_limit);
    if (e == cudaSuccess) e = cudaGetLastError();
    prof_mark(d, prof, 2, sm);
    return e;
}

template <int C, bool H, bool B>
int robust_occupancy() {
    auto rk = loglike_robust_kernel<C, H, B>;
    int n = 0;
    if (cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRobSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk, kRobWarps * 32, kRobSmem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <int C, bool H, bool B, int G>
int occupancy_g(const lisa_tiling& t) {
    auto kern = loglike_fp32_kernel<C, H, B, G>;
    const size_t smem = 2 * (size_t)t.tile_bins * kRec * sizeof(float);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads32, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <int C, bool H, bool B>
int occupancy_m(const lisa_tiling& t) {
    switch (t.group) {
        case 2: return occupancy_g<C, H, B, 2>(t);
        case 8: return occupancy_g<C, H, B, 8>(t);
        default: return occupancy_g<C, H, B, 4>(t);
    }
}

template <int C>
int occupancy_c(int sgwb, const lisa_tiling& t) {
    if (sgwb == 0) return occupancy_m<C, false, false>(t);
    if (sgwb == 1) return occupancy_m<C, true, false>(t);
    return occupancy_m<C, true, true>(t);
}

template <int C, bool H, bool B>
cudaError_t launch_fp32(const lisa_data* d, const StateParams* prm, const int32_t* sstat, const int32_t* nint,
                        const float* kxr, unsigned long long* rcount, const RobustEntry* rlist, const float* srec,
                        int kmax, double* partial, double* rpart, int* err, cudaStream_t sm, bool prof) {
    switch (d->tiling.group) {
        case 2: return launch_fp32_g<C, H, B, 2>(d, prm, sstat, nint, kxr, rcount, rlist, srec, kmax, partial, rpart, err, sm,
                                                    prof);
        case 8: return launch_fp32_g<C, H, B, 8>(d, prm, sstat, nint, kxr, rcount, rlist, srec, kmax, partial, rpart, err, sm,
                                                    prof);
        default:
            return launch_fp32_g<C, H, B, 4>(d, prm, sstat, nint, kxr, rcount, rlist, srec, kmax, partial, rpart, err, sm,
                                                    prof);
    }
}

template <int C, bool H, bool B>
cudaError_t launch_fp64(const lisa_data* d, const double* theta, const int32_t* sstat, const int32_t* nint,
                        const double* srec, int kmax, double* partial, cudaStream_t sm, bool prof) {
    auto kern = loglike_fp64_kernel<C, H, B>;
    const int grid = grid_for(kern, d, 0, kThreads);
    kern<<<grid, kThreads, 0, sm>>>(d->d_items, (int)d->n_items, d->d_rec64, theta, sstat, nint, srec, kmax,
                                    d->nsp, d->d_ds, partial);
    const cudaError_t e = cudaGetLastError();
    prof_mark(d, prof, 1, sm);
    prof_mark(d, prof, 2, sm);   // no compensated kernel in FP64 mode
    return e;
}

template <int C>
cudaError_t dispatch_model(const lisa_data* d, bool fp32, const double* theta, const StateParams* prm,
                           const int32_t* sstat, const int32_t* nint, const float* kxr, unsigned long long* rcount,
                           const RobustEntry* rlist, const void* srec, int kmax, double* partial, double* rpart,
                           int* err, cudaStream_t sm, bool prof) {
    const int h = d->sgwb_model;
    if (fp32) {
        const float* r = static_cast<const float*>(srec);
        if (h == 0)
            return launch_fp32<C, false, false>(d, prm, sstat, nint, kxr, rcount, rlist, r, kmax, partial, rpart, err, sm,
                                                 prof);
        if (h == 1)
            return launch_fp32<C, true, false>(d, prm, sstat, nint, kxr, rcount, rlist, r, kmax, partial, rpart, err, sm,
                                                 prof);
        return launch_fp32<C, true, true>(d, prm, sstat, nint, kxr, rcount, rlist, r, kmax, partial, rpart, err, sm,
                                                 prof);
    }
    const double* r = static_cast<const double*>(srec);
    if (h == 0) return launch_fp64<C, false, false>(d, theta, sstat, nint, r, kmax, partial, sm, prof);
    if (h == 1) return launch_fp64<C, true, false>(d, theta, sstat, nint, r, kmax, partial, sm, prof);
    return launch_fp64<C, true, true>(d, theta, sstat, nint, r, kmax, partial, sm, prof);
}

}  // namespace

int fused_ctas_per_sm(const lisa_data* d, const lisa_tiling& t) {
    return d->C == 3 ? occupancy_c<3>(d->sgwb_model, t) : occupancy_c<2>(d->sgwb_model, t);
}

template <int C>
int robust_occupancy_c(int sgwb) {
    if (sgwb == 0) return robust_occupancy<C, false, false>();
    if (sgwb == 1) return robust_occupancy<C, true, false>();
    return robust_occupancy<C, true, true>();
}

int robust_ctas_per_sm(const lisa_data* d) {
    return d->C == 3 ? robust_occupancy_c<3>(d->sgwb_model) : robust_occupancy_c<2>(d->sgwb_model);
}

}  // namespace lisa

using namespace lisa;

extern "C" {

size_t lisa_workspace_bytes(const lisa_data* d, int32_t kmax, lisa_precision p, int32_t with_grad) {
    if (!d || kmax < 0 || kmax > LISA_MAX_KNOTS) return 0;
    size_t b = ws_fwd_bytes(d);
    if (with_grad) b += grad_extra_bytes(d, kmax, p == LISA_FP32);
    return b;
}

lisa_status lisa_psd_loglike(const lisa_data* d, const lisa_params* params, const void* buf, size_t buf_bytes,
                             int32_t kmax, double* out, void* ws, size_t ws_bytes, lisa_precision prec,
                             lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_psd_loglike");
    if (!d || !params || !buf || !out || !ws) return LISA_ERR_NULL;
    if (prec != LISA_FP32 && prec != LISA_FP64) return LISA_ERR_VALUE;
    if (kmax < 0 || kmax > LISA_MAX_KNOTS) return LISA_ERR_VALUE;
    if (params->n_states != d->n_states) return LISA_ERR_SHAPE;
    if (d->n_states > 0 && !params->theta_dev) return LISA_ERR_NULL;
    const bool fp32 = prec == LISA_FP32;
    const SplineLayout L = spline_layout(d->n_states, d->nsp, kmax);
    if (buf_bytes < L.bytes || (reinterpret_cast<uintptr_t>(buf) & 255)) return LISA_ERR_WORKSPACE;
    if (ws_bytes < ws_fwd_bytes(d) || (reinterpret_cast<uintptr_t>(ws) & 255)) return LISA_ERR_WORKSPACE;
    // the compensated kernel's unit counter holds up to 2^32 - 1 (state, tile) units
    if (fp32 && d->n_partials > (int64_t)0xffffffffLL) return LISA_ERR_SHAPE;
    if (d->n_states == 0) return LISA_SUCCESS;
    cudaStream_t sm = (cudaStream_t)stream;
    const char* base = static_cast<const char*>(buf);
    const int32_t* sstat = reinterpret_cast<const int32_t*>(base + L.off_status);
    const int32_t* nint = reinterpret_cast<const int32_t*>(base + L.off_nint);
    const void* srec = base + L.off_rec;
    const float2* hull = reinterpret_cast<const float2*>(base + L.off_hull);
    const float* kxr = reinterpret_cast<const float*>(base + L.off_kxr);
    char* wsb = static_cast<char*>(ws);
    int* err = reinterpret_cast<int*>(wsb);
    unsigned long long* rcount = reinterpret_cast<unsigned long long*>(wsb + kWsCounterOff);
    const WsLayout W = ws_layout(d);
    double* partial = reinterpret_cast<double*>(wsb + W.off_partial);
    StateParams* prm = reinterpret_cast<StateParams*>(wsb + W.off_prm);
    RobustEntry* rlist = reinterpret_cast<RobustEntry*>(wsb + W.off_rlist);
    int32_t* rent = reinterpret_cast<int32_t*>(wsb + W.off_rent);
    double* rpart = reinterpret_cast<double*>(wsb + W.off_rpart);
    // the error flag and the work-list counter
    if (cudaMemsetAsync(wsb, 0, kWsCounterOff + sizeof(unsigned long long), sm) != cudaSuccess)
        return LISA_ERR_CUDA;
    const int S = (int)d->n_states;
    if (fp32) {
        const int64_t threads = 32 * (int64_t)S;
        state_prep_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, sm>>>(
            S, params->theta_dev, prm, sstat, hull, d->d_state_ds, d->d_ds, d->d_rec32, d->tiling.tile_bins, rcount,
            rlist, rent);
        if (cudaGetLastError() != cudaSuccess) return LISA_ERR_CUDA;
    }
    const bool prof = prof_active(d, sm);
    prof_mark(d, prof, 0, sm);
    cudaError_t e = cudaSuccess;
    if (d->cov == LISA_COV_FULL) {
        // one kernel evaluates every bin (ill-conditioned intervals included)
        if (d->n_items > 0)
            e = launch_full_cov(d, fp32, params->theta_dev, prm, sstat, nint, kxr, srec, kmax, partial, err, sm);
        prof_mark(d, prof, 1, sm);
        prof_mark(d, prof, 2, sm);
    } else if (d->n_items > 0)
        e = d->C == 3 ? dispatch_model<3>(d, fp32, params->theta_dev, prm, sstat, nint, kxr, rcount, rlist, srec, kmax,
                                          partial, rpart, err, sm, prof)
                      : dispatch_model<2>(d, fp32, params->theta_dev, prm, sstat, nint, kxr, rcount, rlist, srec, kmax,
                                          partial, rpart, err, sm, prof);
    else {
        prof_mark(d, prof, 1, sm);
        prof_mark(d, prof, 2, sm);
    }
    if (e != cudaSuccess) return LISA_ERR_CUDA;
    finalize_kernel<<<(S + 7) / 8, 256, 0, sm>>>(S, d->d_state_ds, d->d_ds, sstat, partial, rent, rlist, rpart, err,
                                                 fp32 ? 1 : 0, out);
    e = cudaGetLastError();
    prof_mark(d, prof, 3, sm);
    if (prof) d->prof_valid = true;
    return check_cuda(e);
}

lisa_status lisa_workspace_status(const void* ws, lisa_stream_t stream) {
    if (!ws) return LISA_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return LISA_ERR_WORKSPACE;
    cudaStream_t sm = (cudaStream_t)stream;
    int flag = 0;
    if (cudaMemcpyAsync(&flag, ws, sizeof(int), cudaMemcpyDeviceToHost, sm) != cudaSuccess) return LISA_ERR_CUDA;
    if (cudaStreamSynchronize(sm) != cudaSuccess) return LISA_ERR_CUDA;
    return (flag & kErrTimeout) ? LISA_ERR_TIMEOUT : LISA_SUCCESS;
}

lisa_status lisa_data_kernel_ms(const lisa_data* d, float* ms) {
    if (!d || !ms) return LISA_ERR_NULL;
    if (!d->prof_on || !d->prof_valid) return LISA_ERR_VALUE;
    if (cudaEventSynchronize(d->prof_ev[3]) != cudaSuccess) return LISA_ERR_CUDA;
    for (int k = 0; k < 3; ++k)
        if (cudaEventElapsedTime(&ms[k], d->prof_ev[k], d->prof_ev[k + 1]) != cudaSuccess) return LISA_ERR_CUDA;
    return LISA_SUCCESS;
}

lisa_status lisa_model_psd(const lisa_data* d, const lisa_params* params, const void* buf, size_t buf_bytes,
                           int32_t kmax, double* out, lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_model_psd");
    if (!d || !params || !buf || !out) return LISA_ERR_NULL;
    if (kmax < 0 || kmax > LISA_MAX_KNOTS) return LISA_ERR_VALUE;
    if (params->n_states != d->n_states) return LISA_ERR_SHAPE;
    if (d->n_states > 0 && !params->theta_dev) return LISA_ERR_NULL;
    const SplineLayout L = spline_layout(d->n_states, d->nsp, kmax);
    if (buf_bytes < L.bytes || (reinterpret_cast<uintptr_t>(buf) & 255)) return LISA_ERR_WORKSPACE;
    if (d->n_states == 0) return LISA_SUCCESS;
    if (d->n_states > 65535) return LISA_ERR_VALUE;
    int64_t maxN = 0;
    for (const auto& D : d->h_ds) maxN = D.nbins > maxN ? D.nbins : maxN;
    const char* base = static_cast<const char*>(buf);
    const int32_t* sstat = reinterpret_cast<const int32_t*>(base + L.off_status);
    const int32_t* nint = reinterpret_cast<const int32_t*>(base + L.off_nint);
    const double* srec = reinterpret_cast<const double*>(base + L.off_rec);
    dim3 grid((unsigned)((maxN + 255) / 256), (unsigned)d->n_states);
    cudaStream_t sm = (cudaStream_t)stream;
    const int h = d->sgwb_model != 0, br = d->sgwb_model == 2;
    if (d->C == 3)
        model_psd_kernel<3><<<grid, 256, 0, sm>>>(d->d_state_ds, d->d_ds, d->d_rec64, d->d_P, d->n_bins,
                                                  params->theta_dev, sstat, nint, srec, kmax, d->nsp, h, br, out);
    else
        model_psd_kernel<2><<<grid, 256, 0, sm>>>(d->d_state_ds, d->d_ds, d->d_rec64, d->d_P, d->n_bins,
                                                  params->theta_dev, sstat, nint, srec, kmax, d->nsp, h, br, out);
    return check_cuda(cudaGetLastError());
}

}  // extern "C"

// ---- allocation-free variant: scratch in the library's own device image --------------------
// For callers that cannot allocate a workspace (see include/lisa_psd.h).  The array below is
// the workspace of lisa_psd_loglike, fixed in size; host code only ever uses the device address
// obtained from cudaGetSymbolAddress (the symbol itself names a host-side stand-in).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LISA_NOALLOC_SCRATCH_BYTES];

extern "C" lisa_status lisa_psd_loglike_noalloc(const lisa_data* d, const lisa_params* params, const void* buf,
                                                size_t buf_bytes, int32_t kmax, double* out, lisa_precision prec,
                                                lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_psd_loglike_noalloc");
    if (!d || !params || !buf || !out) return LISA_ERR_NULL;
    if (ws_fwd_bytes(d) > (size_t)LISA_NOALLOC_SCRATCH_BYTES) return LISA_ERR_WORKSPACE;
    // the array exists once per device: use the copy on the device that holds the data object
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LISA_ERR_CUDA;
    if (dev != d->device) return LISA_ERR_VALUE;
    // looked up on every call (a query that enqueues nothing), so that a device reset, which
    // reloads the library's device code at a new address, never leaves a stale pointer behind
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return LISA_ERR_CUDA;
    // lisa_psd_loglike clears the error flag on the stream and overwrites the partial sums.
    return lisa_psd_loglike(d, params, buf, buf_bytes, kmax, out, scratch, LISA_NOALLOC_SCRATCH_BYTES, prec,
                            stream);
}

LISA_DEBUG_TU(loglike)
