// Spline setup: one warp per state builds all of the state's perturbation splines
// (Sec. III.A knot scheme, Appendix A Akima, natural cubic as the alternative kind).
//
// Lane layout: a spline has K = k + 2 <= 64 knots; knot j lives in lane j % 32, slot j / 32.
// Neighbouring knots and interval slopes are exchanged with warp shuffles (shift2 below); only
// the sort's permutation goes through shared memory.
#include "lisa_internal.cuh"

namespace lisa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Values of the entries e + d for the entries e = lane (slot 0) and e = lane + 32 (slot 1),
// |d| <= 32.  Entries outside the array come back as unspecified values; callers mask them.
template <class T>
__device__ __forceinline__ void shift2(T v0, T v1, int d, T& o0, T& o1) {
    const int lane = threadIdx.x & 31;
    const int src = (lane + d) & 31;
    T a = __shfl_sync(kFull, v0, src);
    T b = __shfl_sync(kFull, v1, src);
    const int q = (lane + d) >> 5;   // floor((lane + d) / 32)
    o0 = (q == 0) ? a : b;
    o1 = (q == -1) ? a : b;
}

template <class T>
__device__ __forceinline__ T bcast(T v0, T v1, int e) {
    return __shfl_sync(kFull, e < 32 ? v0 : v1, e & 31);
}

// Parallel cyclic reduction of a tridiagonal system held in the two-slot lane layout (rows
// outside [0, K) are identity rows); on return row j reads Rr[j] / B[j] = solution.
template <class T>
__device__ __forceinline__ void pcr_solve(T (&A)[2], T (&B)[2], T (&Cc)[2], T (&Rr)[2], int K) {
    const int lane = threadIdx.x & 31;
    for (int dd = 1; dd < K; dd <<= 1) {
        T Am[2], Bm[2], Cm[2], Rm[2], Ap[2], Bp[2], Cp[2], Rp[2];
        shift2(A[0], A[1], -dd, Am[0], Am[1]);
        shift2(B[0], B[1], -dd, Bm[0], Bm[1]);
        shift2(Cc[0], Cc[1], -dd, Cm[0], Cm[1]);
        shift2(Rr[0], Rr[1], -dd, Rm[0], Rm[1]);
        shift2(A[0], A[1], dd, Ap[0], Ap[1]);
        shift2(B[0], B[1], dd, Bp[0], Bp[1]);
        shift2(Cc[0], Cc[1], dd, Cp[0], Cp[1]);
        shift2(Rr[0], Rr[1], dd, Rp[0], Rp[1]);
        for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            const bool lo_ok = j - dd >= 0 && j - dd < K;
            const bool hi_ok = j + dd < K;
            if (!lo_ok) { Am[q] = T(0); Bm[q] = T(1); Cm[q] = T(0); Rm[q] = T(0); }
            if (!hi_ok) { Ap[q] = T(0); Bp[q] = T(1); Cp[q] = T(0); Rp[q] = T(0); }
            const T al = -A[q] / Bm[q];
            const T ga = -Cc[q] / Bp[q];
            const T nA = al * Am[q];
            const T nC = ga * Cp[q];
            const T nB = B[q] + al * Cm[q] + ga * Ap[q];
            const T nR = Rr[q] + al * Rm[q] + ga * Rp[q];
            A[q] = nA;
            B[q] = nB;
            Cc[q] = nC;
            Rr[q] = nR;
        }
    }
}

// Akima slope at knot j (0-based) from the interval slopes m_{j-2}, m_{j-1}, m_j, m_{j+1}
// (Appendix A), end knots by the SciPy-style rules:  s_0 = (3 m_0 - m_1)/2,
// s_1 = (|m_2 - m_1| m_0 + |m_1 - m_0| m_1) / (|m_2 - m_1| + |m_1 - m_0|),
// s_{K-2} its mirror image, s_{K-1} = (3 m_{K-2} - m_{K-3})/2; an exactly zero weight sum
// takes the mean of the two slopes adjacent to the knot.
template <class T>
__device__ __forceinline__ T akima_slope(int j, int K, T mm2, T mm1, T m0, T mp1, T m_0, T m_1,
                                         T m_Km2, T m_Km3) {
    if (j == 0) return T(0.5) * (T(3) * m_0 - m_1);
    if (j == K - 1) return T(0.5) * (T(3) * m_Km2 - m_Km3);
    T wl, wr, ml, mr;  // weight on the left slope, weight on the right slope
    if (j == 1) {
        wl = fabs(mp1 - m0);       // |m_2 - m_1|
        wr = fabs(m0 - mm1);       // |m_1 - m_0|
    } else if (j == K - 2) {
        wl = fabs(m0 - mm1);       // |m_{K-2} - m_{K-3}|   (mirror of s_1)
        wr = fabs(mm1 - mm2);      // |m_{K-3} - m_{K-4}|
    } else {
        wl = fabs(mp1 - m0);       // w_j     = |m_{j+1} - m_j|
        wr = fabs(mm1 - mm2);      // w_{j-2} = |m_{j-1} - m_{j-2}|
    }
    ml = mm1;
    mr = m0;
    T den = wl + wr;
    if (den == T(0)) return T(0.5) * (ml + mr);
    return (wl * ml + wr * mr) / den;
}

// One warp per state.  The spline is built in FP64 for both output precisions:
//  kF32 = false: FP64 records {xl, xr, a, b, c, d} about the left knot (the plain path);
//  kF32 = true:  FP32 records about the interval midpoint xo, coefficients scaled to log2 units
//                and split into hi + lo floats, plus the interval's conditioning bound T; a state
//                with any T > kRobustT is appended to the route list (compensated kernel).
template <bool kF32>
__global__ void __launch_bounds__(128) spline_setup_kernel(
    const int32_t* __restrict__ count, const double* __restrict__ kx, const double* __restrict__ kw,
    int S, int nsp, int kmax, int kind, const int32_t* __restrict__ state_ds,
    const DatasetDev* __restrict__ ds, int32_t* __restrict__ status_buf, int32_t* __restrict__ nint_buf,
    int32_t* __restrict__ route, void* __restrict__ rec_v, int32_t* __restrict__ status_out) {
    using T = double;
    __shared__ T sX[4][64];
    __shared__ T sY[4][64];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * 4 + warp;
    if (s >= S) return;  // uniform per warp
    const int dsi = state_ds[s];
    const double xlo = ds[dsi].x_lo, xhi = ds[dsi].x_hi;
    const double xbmin = ds[dsi].xb_min, xbmax = ds[dsi].xb_max;
    int st_all = 0;
    bool robust = false;

    for (int a = 0; a < nsp; ++a) {
        const int64_t sp = (int64_t)s * nsp + a;
        const int k = count[sp];
        int st = 0;
        if (k < 0 || k > kmax) st = LISA_STATE_BAD_COUNT;
        double xa = INFINITY, xb = INFINITY, wa = 0.0, wb = 0.0, w0 = 0.0, wn = 0.0;
        int ra = 0, rb = 0;
        if (!st) {
            const double* px = kx + sp * kmax;
            const double* pw = kw + sp * (kmax + 2);
            bool bx = false, bw = false;
            if (lane < k) {
                xa = px[lane];
                wa = pw[1 + lane];
                bx |= !(isfinite(xa) && xa > xlo && xa < xhi);
                bw |= !isfinite(wa);
            }
            if (lane + 32 < k) {
                xb = px[lane + 32];
                wb = pw[1 + lane + 32];
                bx |= !(isfinite(xb) && xb > xlo && xb < xhi);
                bw |= !isfinite(wb);
            }
            w0 = pw[0];
            wn = pw[kmax + 1];
            bw |= !isfinite(w0) || !isfinite(wn);
            if (__any_sync(kFull, bx)) st |= LISA_STATE_BAD_POSITION;
            if (__any_sync(kFull, bw)) st |= LISA_STATE_BAD_AMPLITUDE;
        }
        if (!st) {
            // rank sort (stable), duplicate detection
            bool dup = false;
            for (int i = 0; i < k; ++i) {
                const double xi = bcast(xa, xb, i);
                if (lane < k) {
                    ra += (xi < xa) || (xi == xa && i < lane);
                    dup |= (xi == xa) && (i != lane);
                }
                if (lane + 32 < k) {
                    rb += (xi < xb) || (xi == xb && i < lane + 32);
                    dup |= (xi == xb) && (i != lane + 32);
                }
            }
            if (__any_sync(kFull, dup)) st |= LISA_STATE_DUPLICATE;
        }
        if (!st) {
            if (lane < k) {
                sX[warp][1 + ra] = xa;
                sY[warp][1 + ra] = wa;
            }
            if (lane + 32 < k) {
                sX[warp][1 + rb] = xb;
                sY[warp][1 + rb] = wb;
            }
            if (lane == 0) {
                sX[warp][0] = xlo;
                sY[warp][0] = w0;
                sX[warp][k + 1] = xhi;
                sY[warp][k + 1] = wn;
            }
            __syncwarp();
            const int K = k + 2;
            const int j0 = lane, j1 = lane + 32;
            T x[2], y[2];
            x[0] = j0 < K ? sX[warp][j0] : T(0);
            y[0] = j0 < K ? sY[warp][j0] : T(0);
            x[1] = j1 < K ? sX[warp][j1] : T(0);
            y[1] = j1 < K ? sY[warp][j1] : T(0);
            __syncwarp();  // the next spline reuses sX / sY
            T xn[2], yn[2], h[2], m[2];
            shift2(x[0], x[1], 1, xn[0], xn[1]);
            shift2(y[0], y[1], 1, yn[0], yn[1]);
            for (int q = 0; q < 2; ++q) {
                const int j = lane + 32 * q;
                if (j < K - 1) {
                    h[q] = xn[q] - x[q];
                    m[q] = (yn[q] - y[q]) / h[q];
                } else {
                    h[q] = T(1);
                    m[q] = T(0);
                }
            }
            T ca[2], cb[2], cc[2], cd[2];
            if (K < 4) {
                // Sec. III.A: fewer than two in-between knots -> linear interpolant
                for (int q = 0; q < 2; ++q) {
                    ca[q] = y[q];
                    cb[q] = m[q];
                    cc[q] = T(0);
                    cd[q] = T(0);
                }
            } else if (kind == LISA_SPLINE_NATURAL) {
                // Natural cubic: rows j = 1..K-2:
                //   h_{j-1} M_{j-1} + 2 (h_{j-1} + h_j) M_j + h_j M_{j+1} = 6 (m_j - m_{j-1}),
                // rows 0 and K-1 (and beyond) identity with M = 0.  Parallel cyclic reduction
                // over the warp: log2(64) = 6 steps of shuffles.
                T hm[2], mm[2];
                shift2(h[0], h[1], -1, hm[0], hm[1]);
                shift2(m[0], m[1], -1, mm[0], mm[1]);
                T A[2], B[2], Cc[2], Rr[2];
                for (int q = 0; q < 2; ++q) {
                    const int j = lane + 32 * q;
                    if (j >= 1 && j <= K - 2) {
                        A[q] = hm[q];
                        B[q] = T(2) * (hm[q] + h[q]);
                        Cc[q] = h[q];
                        Rr[q] = T(6) * (m[q] - mm[q]);
                    } else {
                        A[q] = T(0);
                        B[q] = T(1);
                        Cc[q] = T(0);
                        Rr[q] = T(0);
                    }
                }
                pcr_solve(A, B, Cc, Rr, K);
                T M[2], Mn[2];
                for (int q = 0; q < 2; ++q) M[q] = Rr[q] / B[q];
                shift2(M[0], M[1], 1, Mn[0], Mn[1]);
                for (int q = 0; q < 2; ++q) {
                    ca[q] = y[q];
                    cb[q] = m[q] - h[q] * (T(2) * M[q] + Mn[q]) / T(6);
                    cc[q] = T(0.5) * M[q];
                    cd[q] = (Mn[q] - M[q]) / (T(6) * h[q]);
                }
            } else {
                // Akima (Appendix A)
                T mm1[2], mm2[2], mp1[2];
                shift2(m[0], m[1], -1, mm1[0], mm1[1]);
                shift2(m[0], m[1], -2, mm2[0], mm2[1]);
                shift2(m[0], m[1], 1, mp1[0], mp1[1]);
                const T m_0 = bcast(m[0], m[1], 0), m_1 = bcast(m[0], m[1], 1);
                const T m_Km2 = bcast(m[0], m[1], K - 2), m_Km3 = bcast(m[0], m[1], K - 3);
                T sl[2], sn[2];
                for (int q = 0; q < 2; ++q) {
                    const int j = lane + 32 * q;
                    sl[q] = (j < K) ? akima_slope(j, K, mm2[q], mm1[q], m[q], mp1[q], m_0, m_1, m_Km2, m_Km3)
                                    : T(0);
                }
                shift2(sl[0], sl[1], 1, sn[0], sn[1]);
                for (int q = 0; q < 2; ++q) {
                    ca[q] = y[q];
                    cb[q] = sl[q];
                    cc[q] = (T(3) * m[q] - T(2) * sl[q] - sn[q]) / h[q];
                    cd[q] = (sl[q] + sn[q] - T(2) * m[q]) / (h[q] * h[q]);
                }
            }
            for (int q = 0; q < 2; ++q) {
                const int j = lane + 32 * q;
                if (j >= K - 1) continue;
                const bool last = (j + 1 == K - 1);
                if (!kF32) {
                    double* r = static_cast<double*>(rec_v) + (sp * (int64_t)(kmax + 1) + j) * kSplineRec;
                    r[0] = x[q];
                    r[1] = last ? INFINITY : xn[q];
                    r[2] = ca[q];
                    r[3] = cb[q];
                    r[4] = cc[q];
                    r[5] = cd[q];
                    r[6] = 0.0;
                    r[7] = 0.0;
                } else {
                    // re-expand about the midpoint and scale to log2 units
                    const double hm = 0.5 * h[q];
                    const double xo = x[q] + hm;
                    const double c3 = cd[q];
                    const double c2 = cc[q] + 3.0 * hm * cd[q];
                    const double c1 = cb[q] + hm * (2.0 * cc[q] + 3.0 * hm * cd[q]);
                    const double c0 = ca[q] + hm * (cb[q] + hm * (cc[q] + hm * cd[q]));
                    const double cs[4] = {c0 * kLog2_10, c1 * kLog2_10, c2 * kLog2_10, c3 * kLog2_10};
                    const double lo_x = (j == 0) ? fmin(xbmin, x[q]) : x[q];
                    const double hi_x = last ? fmax(xbmax, xn[q]) : xn[q];
                    const double rr = fmax(fabs(lo_x - xo), fabs(hi_x - xo));
                    const double Tc = fabs(cs[0]) + rr * (fabs(cs[1]) + rr * (fabs(cs[2]) + rr * fabs(cs[3])));
                    robust |= !(Tc <= kRobustT);
                    float* r = static_cast<float*>(rec_v) + (sp * (int64_t)(kmax + 1) + j) * kSplineRec32;
                    const float xo_hi = (float)xo;
                    r[0] = last ? INFINITY : (float)xn[q];
                    r[1] = xo_hi;
                    r[6] = (float)x[q];
                    r[7] = (float)Tc;
                    r[8] = (float)(xo - (double)xo_hi);
                    for (int c = 0; c < 4; ++c) {
                        const float hi = (float)cs[c];
                        r[2 + c] = hi;
                        r[9 + c] = (float)(cs[c] - (double)hi);
                    }
                    r[13] = r[14] = r[15] = 0.f;
                }
            }
            if (lane == 0) nint_buf[sp] = K - 1;
        }
        if (st && lane == 0) nint_buf[sp] = 0;
        st_all |= st;
    }
    robust = __any_sync(kFull, robust);
    if (lane == 0) {
        int word = st_all;
        if (kF32 && robust && st_all == 0) {
            word |= kRouted;
            const int slot = atomicAdd(route, 1);
            route[1 + slot] = s;
        }
        status_buf[s] = word;
        if (status_out) status_out[s] = st_all;
    }
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" lisa_status lisa_spline_setup(const lisa_data* d, const lisa_knots* kn, lisa_precision prec,
                                         void* buf, size_t bytes, int32_t* status_out,
                                         lisa_stream_t stream) {
    if (!d || !kn || !buf) return LISA_ERR_NULL;
    if (prec != LISA_FP32 && prec != LISA_FP64) return LISA_ERR_VALUE;
    if (kn->kmax < 0 || kn->kmax > LISA_MAX_KNOTS || (kn->kind != LISA_SPLINE_AKIMA && kn->kind != LISA_SPLINE_NATURAL))
        return LISA_ERR_VALUE;
    if (kn->n_states != d->n_states || kn->n_splines != d->nsp) return LISA_ERR_SHAPE;
    if (!kn->count_dev || !kn->w_dev || (kn->kmax > 0 && !kn->x_dev)) return LISA_ERR_NULL;
    SplineLayout L = spline_layout(d->n_states, d->nsp, kn->kmax);
    if (bytes < L.bytes || (reinterpret_cast<uintptr_t>(buf) & 255) != 0) return LISA_ERR_WORKSPACE;
    if (d->n_states == 0) return LISA_SUCCESS;
    char* base = static_cast<char*>(buf);
    int32_t* status_buf = reinterpret_cast<int32_t*>(base + L.off_status);
    int32_t* nint_buf = reinterpret_cast<int32_t*>(base + L.off_nint);
    int32_t* route = reinterpret_cast<int32_t*>(base + L.off_route);
    const unsigned blocks = (unsigned)((d->n_states + 3) / 4);
    cudaStream_t sm = (cudaStream_t)stream;
    if (cudaMemsetAsync(route, 0, sizeof(int32_t), sm) != cudaSuccess) return LISA_ERR_CUDA;
    if (prec == LISA_FP64)
        spline_setup_kernel<false><<<blocks, 128, 0, sm>>>(kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states,
                                                           d->nsp, kn->kmax, kn->kind, d->d_state_ds, d->d_ds,
                                                           status_buf, nint_buf, route, base + L.off_rec, status_out);
    else
        spline_setup_kernel<true><<<blocks, 128, 0, sm>>>(kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states,
                                                          d->nsp, kn->kmax, kn->kind, d->d_state_ds, d->d_ds,
                                                          status_buf, nint_buf, route, base + L.off_rec, status_out);
    return check_cuda(cudaGetLastError());
}
