// Pipe-rate measurement (lisa_peaks.h): one kernel per instruction kind, each thread running
// kChains independent dependency chains of that instruction so that the pipe, not latency,
// limits the rate.  The chains are fixed-point iterations whose values stay finite.
#include "lisa_internal.cuh"
#include "lisa_peaks.h"

namespace lisa {
namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kBlocksPerSm = 8;

template <int OP>
__global__ void __launch_bounds__(kBlock) pipe_rate_kernel(int iters, float a, float b, float* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (OP == LISA_PIPE_DFMA) {
        double v[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) v[u] = 0.25 + 0.01 * u + 1e-6 * (g & 1023);
        const double ad = a, bd = b;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kChains; ++u) v[u] = fma(v[u], ad, bd);
        }
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < kChains; ++u) s += v[u];
        out[g] = (float)s;
        return;
    }
    if (OP == LISA_PIPE_MIX) {
        // the fused FP32 likelihood's instruction mix per pair block (two bins of one state, A,E,T
        // with a power-law SGWB): 37 packed FP32 operations, 8 ex2, 2 rcp, 2 lg2, here as
        // independent chains so that only the pipes, not latency, set the rate
        float2 v[kChains];
        float m[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) {
            v[u] = make_float2(0.25f + 0.01f * u, 0.5f + 1e-6f * (g & 1023));
            m[u] = 0.3f + 0.02f * u;
        }
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int u = 0; u < kChains; ++u) v[u] = __ffma2_rn(v[u], a2, b2);
#pragma unroll
            for (int u = 0; u < 5; ++u) v[u] = __ffma2_rn(v[u], a2, b2);
#pragma unroll
            for (int u = 0; u < kChains; ++u) {
                float y;
                const float x = -m[u];   // x <- 2^-x converges to 0.6412
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
                m[u] = y;
            }
            // two reciprocals and two log2s, each folded back into its chain so that nothing is
            // optimised away (x <- 1/x damped, x <- log2(x + 1.5) stay in (0, 2))
            float y0, y1, y2, y3;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(m[0]));
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(m[1]));
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y2) : "f"(m[2] + 1.5f));
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y3) : "f"(m[3] + 1.5f));
            m[0] = fmaf(y0, 0.5f, 0.5f);
            m[1] = fmaf(y1, 0.5f, 0.5f);
            m[2] = y2;
            m[3] = y3;
        }
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < kChains; ++u) s += v[u].x + v[u].y + m[u];
        out[g] = s;
        return;
    }
    if (OP == LISA_PIPE_FFMA2) {
        float2 v[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) v[u] = make_float2(0.25f + 0.01f * u, 0.5f + 1e-6f * (g & 1023));
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kChains; ++u) v[u] = __ffma2_rn(v[u], a2, b2);
        }
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < kChains; ++u) s += v[u].x + v[u].y;
        out[g] = s;
        return;
    }
    float v[kChains];
#pragma unroll
    for (int u = 0; u < kChains; ++u) v[u] = 0.25f + 0.01f * u + 1e-6f * (g & 1023);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kChains; ++u) {
            if (OP == LISA_PIPE_EX2) {
                const float m = -v[u];   // x <- 2^-x converges to 0.6412, staying finite
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(v[u]) : "f"(m));
            } else if (OP == LISA_PIPE_RCP) {
                // x <- 1/x + 1 converges to the golden ratio; the add keeps the compiler from
                // cancelling consecutive reciprocals and costs an FMA-pipe slot, not a MUFU one
                float y;
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v[u]));
                v[u] = y + 1.0f;
            } else if (OP == LISA_PIPE_LG2_EX2) {
                float l;
                asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(v[u]));
                const float m = -l;      // x <- 1/x through its logarithm: alternates, stays finite
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(v[u]) : "f"(m));
            } else {
                v[u] = fmaf(v[u], a, b);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < kChains; ++u) s += v[u];
    out[g] = s;
}

template <int OP>
lisa_status time_op(int iters, int reps, int n_sm, float* buf, cudaStream_t sm, double* rate) {
    if (OP == LISA_PIPE_DFMA) iters = iters / 8 > 2 ? iters / 8 : 2;   // the FP64 pipe is slow
    const unsigned blocks = (unsigned)(n_sm * kBlocksPerSm);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LISA_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LISA_ERR_CUDA;
    }
    lisa_status st = LISA_SUCCESS;
    pipe_rate_kernel<OP><<<blocks, kBlock, 0, sm>>>(iters, 0.999f, 0.001f, buf);
    float best = 0.f;
    for (int r = 0; r < reps && st == LISA_SUCCESS; ++r) {
        cudaEventRecord(e0, sm);
        pipe_rate_kernel<OP><<<blocks, kBlock, 0, sm>>>(iters, 0.999f, 0.001f, buf);
        cudaEventRecord(e1, sm);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = LISA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    if (st == LISA_SUCCESS) st = check_cuda(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LISA_SUCCESS) return st;
    // lane operations per chain step (a packed FMA, or lg2 + ex2, counts two); the mix counts
    // state-bins: one iteration of a thread is one pair block, two state-bins
    const double per_step = (OP == LISA_PIPE_LG2_EX2 || OP == LISA_PIPE_FFMA2) ? 2.0 : 1.0;
    const double ops = OP == LISA_PIPE_MIX ? (double)blocks * kBlock * 2.0 * (double)iters
                                           : (double)blocks * kBlock * kChains * (double)iters * per_step;
    *rate = best > 0.f ? ops / (best * 1e-3) : 0.0;
    return LISA_SUCCESS;
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" lisa_status lisa_pipe_rates(int32_t iters, int32_t reps, double* rates, lisa_stream_t stream) {
    if (!rates) return LISA_ERR_NULL;
    if (iters < 16 || reps < 1) return LISA_ERR_VALUE;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0)
        return LISA_ERR_CUDA;
    float* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * (size_t)n_sm * kBlocksPerSm * kBlock) != cudaSuccess) return LISA_ERR_ALLOC;
    cudaStream_t sm = (cudaStream_t)stream;
    lisa_status st = time_op<LISA_PIPE_EX2>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_EX2]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_RCP>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_RCP]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_LG2_EX2>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_LG2_EX2]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_FFMA>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_FFMA]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_FFMA2>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_FFMA2]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_DFMA>(iters, reps, n_sm, buf, sm, &rates[LISA_PIPE_DFMA]);
    if (st == LISA_SUCCESS) st = time_op<LISA_PIPE_MIX>(iters / 4, reps, n_sm, buf, sm, &rates[LISA_PIPE_MIX]);
    cudaStreamSynchronize(sm);
    cudaFree(buf);
    return st;
}

LISA_DEBUG_TU(peaks)
