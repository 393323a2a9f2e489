// Warp-level construction of one perturbation spline (Sec. III.A knot scheme, Appendix A
// Akima, natural cubic as the alternative kind), shared by the spline setup and the adjoint.
//
// Lane layout: a spline has K = k + 2 <= 64 knots; knot j lives in lane j % 32, slot j / 32.
// Neighbouring knots and interval slopes are exchanged with warp shuffles; only the sort's
// permutation goes through shared memory.
#pragma once

#include "lisa_math.cuh"

namespace lisa {
namespace spl {

constexpr unsigned kFull = 0xffffffffu;

// A float-float value (hi + lo, |lo| <= ulp(hi) / 2, about 48 significant bits) with the
// arithmetic the spline construction needs, so that the FP32 path's setup runs on the FP32 pipe.
// Sums use the accurate float-float addition (both parts two-summed), products and quotients
// one correction step each (Dekker's method); relative error a few times 2^-46 per operation.
struct F2 {
    float hi, lo;
    __device__ F2() : hi(0.f), lo(0.f) {}
    __device__ F2(float h, float l) : hi(h), lo(l) {}
    __device__ F2(int v) : hi((float)v), lo(0.f) {}
    __device__ F2(float v) : hi(v), lo(0.f) {}
    // the nearest float-float to a double (exact for doubles of at most 48 significant bits)
    __device__ explicit F2(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.hi, -a.lo); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    const dm::ff s = dm::two_sum(a.hi, b.hi);
    const dm::ff t = dm::two_sum(a.lo, b.lo);
    dm::ff u = dm::fast_two_sum(s.hi, s.lo + t.hi);
    u = dm::fast_two_sum(u.hi, u.lo + t.lo);
    return F2(u.hi, u.lo);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return a + (-b); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    const dm::ff p = dm::ff_mul(dm::ff{a.hi, a.lo}, dm::ff{b.hi, b.lo});
    return F2(p.hi, p.lo);
}
__device__ __forceinline__ F2 operator/(F2 a, F2 b) {
    const float q1 = a.hi / b.hi;
    const F2 r = a - b * F2(q1);
    const float q2 = r.hi / b.hi;
    const dm::ff q = dm::fast_two_sum(q1, q2);
    return F2(q.hi, q.lo);
}
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ bool operator==(F2 a, F2 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ F2 fabs(F2 a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f) ? -a : a; }
__device__ __forceinline__ double fabs(double v) { return ::fabs(v); }   // (not hidden by the above)

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(F2 v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ double sign_of(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }
__device__ __forceinline__ F2 sign_of(F2 v) {
    const float h = v.hi != 0.f ? v.hi : v.lo;
    return F2(h > 0.f ? 1.f : (h < 0.f ? -1.f : 0.f));
}
// a value given as float hi + lo parts
template <class T>
__device__ __forceinline__ T from_hilo(float hi, float lo);
template <>
__device__ __forceinline__ double from_hilo<double>(float hi, float lo) { return (double)hi + (double)lo; }
template <>
__device__ __forceinline__ F2 from_hilo<F2>(float hi, float lo) {
    const dm::ff v = dm::two_sum(hi, lo);
    return F2(v.hi, v.lo);
}

__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(kFull, v, src); }
__device__ __forceinline__ F2 shfl(F2 v, int src) {
    return F2(__shfl_sync(kFull, v.hi, src), __shfl_sync(kFull, v.lo, src));
}

// Values of the entries e + d for the entries e = lane (slot 0) and e = lane + 32 (slot 1),
// |d| <= 32.  Entries outside the array come back as unspecified values; callers mask them.
template <class T>
__device__ __forceinline__ void shift2(T v0, T v1, int d, T& o0, T& o1) {
    const int lane = threadIdx.x & 31;
    const int src = (lane + d) & 31;
    T a = shfl(v0, src);
    T b = shfl(v1, src);
    const int q = (lane + d) >> 5;   // floor((lane + d) / 32)
    o0 = (q == 0) ? a : b;
    o1 = (q == -1) ? a : b;
}

template <class T>
__device__ __forceinline__ T bcast(T v0, T v1, int e) {
    return shfl(e < 32 ? v0 : v1, e & 31);
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

// One spline, built by a whole warp in T (double, or F2 float-float for the FP32 path's records).
// Per lane, slot q holds knot j = lane + 32 q:
//   x, y     sorted knot positions and amplitudes (j < K)
//   h, m     width and slope of interval j (j < K - 1); ih = 1 / h
//   d2       Akima slope s_j (kind 0, K >= 4) or natural-cubic second derivative M_j (kind 1)
//   ca..cd   coefficients of interval j about x_j (log10 units)
// ra, rb are the sorted positions (1-based, edges excluded) of in-between knots lane, lane+32.
template <class T>
struct WarpSpline {
    int K, st;
    int ra, rb;
    T x[2], y[2], h[2], ih[2], m[2], d2[2];
    T ca[2], cb[2], cc[2], cd[2];
};

// Validates the knots of one spline (status bits as in lisa_psd.h) and builds it.  px/pw point
// at the spline's kmax positions and kmax + 2 amplitudes; sX/sY are 64-entry shared scratch
// owned by the warp.  Returns with W.st != 0 (and nothing else defined) for invalid knots.  The
// knots' validation and sort, and the interval widths and amplitude steps (differences of the
// FP64 inputs, exact for close knots), are taken in FP64; the rest of the construction in T.
template <class T>
__device__ __forceinline__ void warp_build_spline(WarpSpline<T>& W, const double* __restrict__ px,
                                                  const double* __restrict__ pw, int k, int kmax, int kind,
                                                  double xlo, double xhi, double* sX, double* sY) {
    const int lane = threadIdx.x & 31;
    int st = 0;
    if (k < 0 || k > kmax) st = LISA_STATE_BAD_COUNT;
    double xa = INFINITY, xb = INFINITY, wa = 0.0, wb = 0.0, w0 = 0.0, wn = 0.0;
    int ra = 0, rb = 0;
    if (!st) {
        bool bx = false, bw = false;
        if (lane < k) {
            xa = px[LISA_IDX(lane, kmax)];
            wa = pw[1 + LISA_IDX(lane, kmax)];
            bx |= !(isfinite(xa) && xa > xlo && xa < xhi);
            bw |= !isfinite(wa);
        }
        if (lane + 32 < k) {
            xb = px[LISA_IDX(lane + 32, kmax)];
            wb = pw[1 + LISA_IDX(lane + 32, kmax)];
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
        // rank sort (stable) with duplicate detection, on integer keys that order like the
        // (finite) doubles, so the comparisons run on the integer pipes
        auto key = [](double v) {
            const long long b = __double_as_longlong(v);
            return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
        };
        const long long ka = key(xa), kb = key(xb);
        bool dup = false;
        for (int i = 0; i < k; ++i) {
            const long long ki = __shfl_sync(kFull, i < 32 ? ka : kb, i & 31);
            if (lane < k) {
                ra += (ki < ka) || (ki == ka && i < lane);
                dup |= (ki == ka) && (i != lane);
            }
            if (lane + 32 < k) {
                rb += (ki < kb) || (ki == kb && i < lane + 32);
                dup |= (ki == kb) && (i != lane + 32);
            }
        }
        if (__any_sync(kFull, dup)) st |= LISA_STATE_DUPLICATE;
    }
    W.st = st;
    if (st) return;
    W.ra = 1 + ra;
    W.rb = 1 + rb;
    // scratch rows of 64 doubles: knots 0 .. k + 1 <= kmax + 1
    if (lane < k) {
        sX[LISA_IDX(1 + ra, 64)] = xa;
        sY[LISA_IDX(1 + ra, 64)] = wa;
    }
    if (lane + 32 < k) {
        sX[LISA_IDX(1 + rb, 64)] = xb;
        sY[LISA_IDX(1 + rb, 64)] = wb;
    }
    if (lane == 0) {
        sX[0] = xlo;
        sY[0] = w0;
        sX[LISA_IDX(k + 1, 64)] = xhi;
        sY[LISA_IDX(k + 1, 64)] = wn;
    }
    __syncwarp();
    const int K = k + 2;
    W.K = K;
    const int j0 = lane, j1 = lane + 32;
    T* x = W.x;
    T* y = W.y;
    double xd[2], yd[2];
    xd[0] = j0 < K ? sX[j0] : 0.0;
    yd[0] = j0 < K ? sY[j0] : 0.0;
    xd[1] = j1 < K ? sX[j1] : 0.0;
    yd[1] = j1 < K ? sY[j1] : 0.0;
    __syncwarp();  // the caller may reuse sX / sY
    double xn[2], yn[2];
    T* h = W.h;
    T* m = W.m;
    shift2(xd[0], xd[1], 1, xn[0], xn[1]);
    shift2(yd[0], yd[1], 1, yn[0], yn[1]);
    T* ih = W.ih;
    for (int q = 0; q < 2; ++q) {
        x[q] = T(xd[q]);
        y[q] = T(yd[q]);
    }
    h[1] = ih[1] = T(1);
    m[1] = T(0);
    for (int q = 0; q < (K > 32 ? 2 : 1); ++q) {
        const int j = lane + 32 * q;
        if (j < K - 1) {
            h[q] = T(xn[q] - xd[q]);
            ih[q] = T(1) / h[q];
            m[q] = T(yn[q] - yd[q]) * ih[q];
        } else {
            h[q] = ih[q] = T(1);
            m[q] = T(0);
        }
    }
    T* ca = W.ca;
    T* cb = W.cb;
    T* cc = W.cc;
    T* cd = W.cd;
    W.d2[0] = W.d2[1] = T(0);
    W.ca[1] = W.cb[1] = W.cc[1] = W.cd[1] = T(0);
    const int nq = K > 32 ? 2 : 1;   // the second lane slot is only used by splines with K > 32
    if (K < 4) {
        // Sec. III.A: fewer than two in-between knots -> linear interpolant
        for (int q = 0; q < nq; ++q) {
            ca[q] = y[q];
            cb[q] = m[q];
            cc[q] = T(0);
            cd[q] = T(0);
        }
    } else if (kind == LISA_SPLINE_NATURAL) {
        // Natural cubic: rows j = 1..K-2:
        //   h_{j-1} M_{j-1} + 2 (h_{j-1} + h_j) M_j + h_j M_{j+1} = 6 (m_j - m_{j-1}),
        // rows 0 and K-1 (and beyond) identity with M = 0; parallel cyclic reduction.
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
        T Mn[2];
        for (int q = 0; q < nq; ++q) W.d2[q] = Rr[q] / B[q];
        shift2(W.d2[0], W.d2[1], 1, Mn[0], Mn[1]);
        for (int q = 0; q < nq; ++q) {
            const T M = W.d2[q];
            ca[q] = y[q];
            cb[q] = m[q] - h[q] * (T(2) * M + Mn[q]) * T(1.0 / 6.0);
            cc[q] = T(0.5) * M;
            cd[q] = (Mn[q] - M) * ih[q] * T(1.0 / 6.0);
        }
    } else {
        // Akima (Appendix A)
        T mm1[2], mm2[2], mp1[2];
        shift2(m[0], m[1], -1, mm1[0], mm1[1]);
        shift2(m[0], m[1], -2, mm2[0], mm2[1]);
        shift2(m[0], m[1], 1, mp1[0], mp1[1]);
        const T m_0 = bcast(m[0], m[1], 0), m_1 = bcast(m[0], m[1], 1);
        const T m_Km2 = bcast(m[0], m[1], K - 2), m_Km3 = bcast(m[0], m[1], K - 3);
        T sn[2];
        for (int q = 0; q < nq; ++q) {
            const int j = lane + 32 * q;
            W.d2[q] = (j < K) ? akima_slope(j, K, mm2[q], mm1[q], m[q], mp1[q], m_0, m_1, m_Km2, m_Km3) : T(0);
        }
        shift2(W.d2[0], W.d2[1], 1, sn[0], sn[1]);
        for (int q = 0; q < nq; ++q) {
            const T sl = W.d2[q];
            ca[q] = y[q];
            cb[q] = sl;
            cc[q] = (T(3) * m[q] - T(2) * sl - sn[q]) * ih[q];
            cd[q] = (sl + sn[q] - T(2) * m[q]) * (ih[q] * ih[q]);
        }
    }
}

}  // namespace spl
}  // namespace lisa
