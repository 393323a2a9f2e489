// Data preparation (Sec. III.C): synthetic frequency-domain data and the averaged periodogram,
// the inputs of lisa_data_create.  Both are streaming kernels bound by HBM bandwidth.
#include <cmath>

#include "lisa_internal.cuh"

namespace lisa {
namespace {

// d = sqrt(S / 2) (z0 + i z1), grid-stride over (channel, sample), 16-byte loads and stores.
__global__ void fd_synth_kernel(const double* __restrict__ S, const double2* __restrict__ z, int64_t n,
                                double2* __restrict__ d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double a = sqrt(0.5 * __ldg(S + i));
        const double2 v = __ldg(z + i);
        d[i] = make_double2(a * v.x, a * v.y);
    }
}

// Averaged periodogram: a group of G lanes per bin (G divides 32), lanes striding over the bin's
// samples with 16-byte loads; the group's partial sums are combined by a butterfly of shuffles (a
// fixed order for a given G).  GB300's FP64 pipe, not HBM, bounds this kernel: per complex sample
// the work is two FP64 FMAs, and each bin adds log2(G) shuffle-adds per channel plus an epilogue
// (a division, the bin centre) that occupy FP64 issue slots for the whole warp.  G = 4 keeps the
// useful share of those slots near 85 % for 64-sample bins while each group still reads 64
// contiguous bytes.
template <int C, int G>
__global__ void avg_periodogram_kernel(const double2* __restrict__ d, int64_t n_freq, double f0, double df,
                                       const int64_t* __restrict__ off, int64_t n_bins, double* __restrict__ P,
                                       double* __restrict__ f_out, double* __restrict__ nu_out, int n_ch) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t n_iter = (n_bins + ng - 1) / ng;   // the same trip count for every lane
    for (int64_t it = 0; it < n_iter; ++it) {
        const int64_t i = g0 + it * ng;
        const bool live = i < n_bins;
        int64_t b0 = 0, b1 = 0;
        if (live) {
            b0 = min(max(__ldg(off + i), (int64_t)0), n_freq);
            b1 = min(max(__ldg(off + i + 1), b0), n_freq);
        }
        double acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
#pragma unroll 4
        for (int64_t k = b0 + lane; k < b1; k += G) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (c < n_ch) {
                    const double2 v = __ldg(d + (int64_t)c * n_freq + k);
                    acc[c] = fma(v.x, v.x, fma(v.y, v.y, acc[c]));
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
        if (live && lane == 0) {
            const int64_t n = b1 - b0;
#pragma unroll
            for (int c = 0; c < C; ++c)
                if (c < n_ch) P[(int64_t)c * n_bins + i] = n > 0 ? acc[c] / (double)n : NAN;
            f_out[i] = f0 + df * (0.5 * (double)(b0 + b1 - 1));
            nu_out[i] = (double)n;
        }
    }
}

template <int C, int G>
cudaError_t launch_avg(const double2* d, int64_t n_freq, double f0, double df, const int64_t* off, int64_t n_bins,
                       double* P, double* f, double* nu, int n_ch, cudaStream_t sm) {
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    const int64_t want = (n_bins * G + threads - 1) / threads;
    const int64_t cap = (int64_t)n_sm * 8;   // persistent: 8 blocks of 256 threads per SM
    const unsigned grid = (unsigned)(want < cap ? (want < 1 ? 1 : want) : cap);
    avg_periodogram_kernel<C, G><<<grid, threads, 0, sm>>>(d, n_freq, f0, df, off, n_bins, P, f, nu, n_ch);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" lisa_status lisa_fd_synthesize(const double* psd, const double* normal, int32_t n_channels, int64_t n_freq,
                                          double* d, lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_fd_synthesize");
    if (n_channels < 1 || n_freq < 0) return LISA_ERR_VALUE;
    if (n_freq == 0) return LISA_SUCCESS;
    if (!psd || !normal || !d) return LISA_ERR_NULL;
    if ((reinterpret_cast<uintptr_t>(normal) | reinterpret_cast<uintptr_t>(d)) & 15) return LISA_ERR_VALUE;
    const int64_t n = (int64_t)n_channels * n_freq;
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, cap = (int64_t)n_sm * 8;
    fd_synth_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(
        psd, reinterpret_cast<const double2*>(normal), n, reinterpret_cast<double2*>(d));
    return check_cuda(cudaGetLastError());
}

extern "C" lisa_status lisa_averaged_periodogram(const double* d, int32_t n_channels, int64_t n_freq, double f0,
                                                 double df, const int64_t* off, int64_t n_bins, double* P, double* f,
                                                 double* nu, lisa_stream_t stream) {
    lisa::NvtxRange nvtx_range("lisa_averaged_periodogram");
    if (n_channels < 1 || n_channels > 3 || n_freq < 0 || n_bins < 0 || !(df > 0.0) || !std::isfinite(f0))
        return LISA_ERR_VALUE;
    if (n_bins == 0) return LISA_SUCCESS;
    if (!d || !off || !P || !f || !nu) return LISA_ERR_NULL;
    if (reinterpret_cast<uintptr_t>(d) & 15) return LISA_ERR_VALUE;
    const double2* dd = reinterpret_cast<const double2*>(d);
    cudaStream_t sm = (cudaStream_t)stream;
    // lanes per bin from the mean bin width: 8 lanes for bins of hundreds of samples, 4 for tens,
    // one thread for bins of a few samples
    const double width = (double)n_freq / (double)n_bins;
    cudaError_t e;
    if (width >= 256.0)
        e = launch_avg<3, 8>(dd, n_freq, f0, df, off, n_bins, P, f, nu, n_channels, sm);
    else if (width >= 12.0)
        e = launch_avg<3, 4>(dd, n_freq, f0, df, off, n_bins, P, f, nu, n_channels, sm);
    else
        e = launch_avg<3, 1>(dd, n_freq, f0, df, off, n_bins, P, f, nu, n_channels, sm);
    return check_cuda(e);
}

LISA_DEBUG_TU(prep)
