// Spline setup: one CTA per state, one warp per perturbation spline
// (Sec. III.A knot scheme, Appendix A Akima, natural cubic as the alternative kind) with the
// warp-level construction of lisa_spline_dev.cuh and writes the interval records.
#include "lisa_spline_dev.cuh"

#include <type_traits>

namespace lisa {
namespace {

// One CTA per state, one warp per spline.
//  kF32 = false: built in FP64; FP64 records {xl, xr, a, b, c, d} about the left knot (the plain
//                path);
//  kF32 = true:  built in float-float on the FP32 pipe (FP64 only for the inputs' validation,
//                sort and differences); FP32 records about the interval midpoint xo,
//                coefficients scaled to log2 units as hi floats, plus the interval's
//                conditioning bound T; a state with any T > kRobustT is appended to the route
//                list (compensated kernel).  The lo floats of the coefficients (float-float value
//                - hi) complete every record: the compensated kernels and the gradient's
//                fallback pass evaluate the spline from hi + lo.
// 7 CTAs per SM (at most 72 registers) keep 1,064 states resident at once.
// kMaxSp: splines per state the launch allows (4 for the diagonal covariance, 8 for the full one,
// which has seven); do_route = 0 leaves the routing bit unset (the full-covariance FP32 kernel
// evaluates ill-conditioned intervals itself).
template <bool kF32, int kMaxSp>
__global__ void __launch_bounds__(32 * kMaxSp, kMaxSp == 4 ? 7 : 3) spline_setup_kernel(
    const int32_t* __restrict__ count, const double* __restrict__ kx, const double* __restrict__ kw,
    int S, int nsp, int kmax, int kind, const int32_t* __restrict__ state_ds,
    const DatasetDev* __restrict__ ds, int32_t* __restrict__ status_buf, int32_t* __restrict__ nint_buf,
    int32_t* __restrict__ route, void* __restrict__ rec_v, float2* __restrict__ hull,
    float* __restrict__ kxr, int32_t* __restrict__ status_out, int do_route) {
    using T = double;
    __shared__ T sX[kMaxSp][64];
    __shared__ T sY[kMaxSp][64];
    __shared__ int sSt[kMaxSp], sRob[kMaxSp];
    __shared__ float sHlo[kMaxSp], sHhi[kMaxSp];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x;
    const int dsi = state_ds[s];
    const double xlo = ds[dsi].x_lo, xhi = ds[dsi].x_hi;
    const float xbmin_f = (float)ds[dsi].xb_min, xbmax_f = (float)ds[dsi].xb_max;
    int st_all = 0;
    bool robust = false;
    float hlo = INFINITY, hhi = -INFINITY;   // x-extent of this spline's ill-conditioned intervals

    {
        const int a = warp;   // blockDim.x = 32 * nsp
        const int64_t sp = (int64_t)s * nsp + a;
        // the FP32 path's records are built in float-float (FP32 pipe), the FP64 path's in FP64
        using BT = typename std::conditional<kF32, spl::F2, double>::type;
        spl::WarpSpline<BT> W;
        spl::warp_build_spline<BT>(W, kx + sp * kmax, kw + sp * (kmax + 2), count[sp], kmax, kind, xlo, xhi, sX[warp],
                                   sY[warp]);
        const int st = W.st;
        if (!st) {
            const int K = W.K;
            BT xn[2];
            spl::shift2(W.x[0], W.x[1], 1, xn[0], xn[1]);
            for (int q = 0; q < (K > 32 ? 2 : 1); ++q) {   // warp-uniform
                const int j = lane + 32 * q;
                const bool valid = j < K - 1;
                const bool last = (j + 1 == K - 1);
                const BT* x = W.x;
                const BT *ca = W.ca, *cb = W.cb, *cc = W.cc, *cd = W.cd, *h = W.h;
                if constexpr (!kF32) {
                    if (!valid) continue;
                    double* r = static_cast<double*>(rec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(j, kmax + 1)) * kSplineRec;
                    r[0] = x[q];
                    r[1] = last ? INFINITY : xn[q];
                    r[2] = ca[q];
                    r[3] = cb[q];
                    r[4] = cc[q];
                    r[5] = cd[q];
                    r[6] = 0.0;
                    r[7] = 0.0;
                } else {
                    // re-expand about the midpoint and scale to log2 units in float-float (every
                    // lane computes, lanes past the last interval on finite placeholder values,
                    // and only valid lanes write); hi parts are the records' FP32 coefficients,
                    // lo parts their remainders
                    using spl::F2;
                    const F2 hm = h[q] * F2(0.5f);
                    const F2 xo = x[q] + hm;
                    const F2 h3d = F2(3) * hm * cd[q];
                    const F2 c3 = cd[q];
                    const F2 c2 = cc[q] + h3d;
                    const F2 c1 = cb[q] + hm * (F2(2) * cc[q] + h3d);
                    const F2 c0 = ca[q] + hm * (cb[q] + hm * (cc[q] + hm * cd[q]));
                    const F2 L2(kLog2_10);
                    const F2 cs[4] = {c0 * L2, c1 * L2, c2 * L2, c3 * L2};
                    float chi[4];
                    for (int c = 0; c < 4; ++c) chi[c] = cs[c].hi;
                    const float xo_hi = xo.hi;
                    const float xl_f = x[q].hi, xr_f = xn[q].hi;
                    // the conditioning bound only steers the routing: FP32 is precise enough (and
                    // keeps these steps off the FP64 pipe, which bounds this kernel)
                    const float lo_x = (j == 0) ? fminf(xbmin_f, xl_f) : xl_f;
                    const float hi_x = last ? fmaxf(xbmax_f, xr_f) : xr_f;
                    const float rr = fmaxf(fabsf(lo_x - xo_hi), fabsf(hi_x - xo_hi));
                    const float Tc = fabsf(chi[0]) + rr * (fabsf(chi[1]) + rr * (fabsf(chi[2]) + rr * fabsf(chi[3])));
                    const bool hard = valid && !(Tc <= (float)kRobustT);
                    if (hard) {
                        robust = true;
                        hlo = fminf(hlo, j == 0 ? -INFINITY : xl_f);
                        hhi = fmaxf(hhi, last ? INFINITY : xr_f);
                    }
                    if (!valid) continue;
                    float* r = static_cast<float*>(rec_v) + (sp * (int64_t)(kmax + 1) + LISA_IDX(j, kmax + 1)) * kSplineRec32;
                    r[0] = last ? INFINITY : xr_f;
                    kxr[sp * kxr_stride(kmax) + LISA_IDX(j, kxr_stride(kmax))] = r[0];
                    r[1] = xo_hi;
                    r[6] = xl_f;
                    r[7] = Tc;
                    r[8] = xo.lo;
                    for (int c = 0; c < 4; ++c) {
                        r[2 + c] = chi[c];
                        r[9 + c] = cs[c].lo;
                    }
                    r[13] = r[14] = r[15] = 0.f;
                }
            }
            if (lane == 0) nint_buf[sp] = K - 1;
        }
        if (st && lane == 0) nint_buf[sp] = 0;
        if (kF32) {
            // right-end table past the last interval (all of it for an invalid spline): +inf
            const int first_pad = st ? 0 : W.K - 1;
            for (int j = lane; j < kxr_stride(kmax); j += 32)
                if (j >= first_pad) kxr[sp * kxr_stride(kmax) + j] = INFINITY;
        }
        st_all |= st;
    }
    robust = __any_sync(spl::kFull, robust);
    for (int o = 16; o > 0; o >>= 1) {
        hlo = fminf(hlo, __shfl_xor_sync(spl::kFull, hlo, o));
        hhi = fmaxf(hhi, __shfl_xor_sync(spl::kFull, hhi, o));
    }
    if (lane == 0) {
        sSt[warp] = st_all;
        sRob[warp] = robust ? 1 : 0;
        sHlo[warp] = hlo;
        sHhi[warp] = hhi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        robust = false;
        st_all = 0;
        hlo = INFINITY;
        hhi = -INFINITY;
        for (int a = 0; a < nsp; ++a) {
            st_all |= sSt[a];
            robust |= sRob[a] != 0;
            hlo = fminf(hlo, sHlo[a]);
            hhi = fmaxf(hhi, sHhi[a]);
        }
        if (kF32) hull[s] = make_float2(hlo, hhi);
        int word = st_all;
        if (kF32 && do_route && robust && st_all == 0) {
            word |= kRouted;
            const int slot = atomicAdd(route, 1);
            route[1 + LISA_IDX(slot, S)] = s;
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
    lisa::NvtxRange nvtx_range("lisa_spline_setup");
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
    const unsigned blocks = (unsigned)d->n_states;
    const unsigned threads = 32u * (unsigned)d->nsp;
    cudaStream_t sm = (cudaStream_t)stream;
    if (cudaMemsetAsync(route, 0, sizeof(int32_t), sm) != cudaSuccess) return LISA_ERR_CUDA;
    const int do_route = d->cov == LISA_COV_DIAGONAL;
    float2* hull = reinterpret_cast<float2*>(base + L.off_hull);
    float* kxr = reinterpret_cast<float*>(base + L.off_kxr);
    void* rec = base + L.off_rec;
    if (d->nsp <= 4) {
        if (prec == LISA_FP64)
            spline_setup_kernel<false, 4><<<blocks, threads, 0, sm>>>(
                kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states, d->nsp, kn->kmax, kn->kind, d->d_state_ds,
                d->d_ds, status_buf, nint_buf, route, rec, hull, kxr, status_out, do_route);
        else
            spline_setup_kernel<true, 4><<<blocks, threads, 0, sm>>>(
                kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states, d->nsp, kn->kmax, kn->kind, d->d_state_ds,
                d->d_ds, status_buf, nint_buf, route, rec, hull, kxr, status_out, do_route);
    } else {
        if (prec == LISA_FP64)
            spline_setup_kernel<false, 8><<<blocks, threads, 0, sm>>>(
                kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states, d->nsp, kn->kmax, kn->kind, d->d_state_ds,
                d->d_ds, status_buf, nint_buf, route, rec, hull, kxr, status_out, do_route);
        else
            spline_setup_kernel<true, 8><<<blocks, threads, 0, sm>>>(
                kn->count_dev, kn->x_dev, kn->w_dev, (int)d->n_states, d->nsp, kn->kmax, kn->kind, d->d_state_ds,
                d->d_ds, status_buf, nint_buf, route, rec, hull, kxr, status_out, do_route);
    }
    return check_cuda(cudaGetLastError());
}

LISA_DEBUG_TU(spline)
