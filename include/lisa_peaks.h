/*
 * lisa_peaks.h -- measured issue rates of the GB300 arithmetic pipes that bound the fused
 * likelihood kernels (the roofline denominators of the benchmark).  Not part of the method:
 * the paper has no counterpart; this is measurement infrastructure.
 *
 * The fused FP32 likelihood does no dense contraction and moves few bytes per state-bin, so its
 * roofline is set by the MUFU (special-function) pipe -- ex2, rcp, lg2 -- and by the FP32 FMA
 * pipe; the FP64 paths and the FP64 data preparation are bound by the FP64 pipe.  Their per-SM rates are not printed on any data sheet this library can rely on, so
 * lisa_pipe_rates measures them: one kernel per operation runs many independent dependency
 * chains of that single instruction on every SM (8 CTAs of 256 threads per SM, 8 chains per
 * thread) and is timed with CUDA events.  lisa_data_set_profiling / lisa_data_kernel_ms time
 * the likelihood's own kernels.
 */
#ifndef LISA_PEAKS_H
#define LISA_PEAKS_H

#include "lisa_psd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lisa_pipe_op {
    LISA_PIPE_EX2 = 0,      /* ex2.approx.ftz.f32: chain x <- 2^-x */
    LISA_PIPE_RCP = 1,      /* rcp.approx.ftz.f32: chain x <- 1/x + 1 (the add runs on the FMA pipe) */
    LISA_PIPE_LG2_EX2 = 2,  /* lg2.approx.ftz.f32 then ex2.approx.ftz.f32: chain x <- 2^-(log2 x) */
    LISA_PIPE_FFMA = 3,     /* fma.rn.f32: chain x <- x a + b */
    LISA_PIPE_FFMA2 = 4,    /* fma.rn.f32x2 (packed pair): chain x <- x a + b on both halves */
    LISA_PIPE_DFMA = 5,     /* fma.rn.f64: chain x <- x a + b (the FP64 pipe that bounds the FP64
                               paths and the data preparation; iters / 8 steps per chain) */
    LISA_PIPE_MIX = 6,      /* the fused FP32 likelihood's instruction mix per pair block of the
                               A,E,T power-law model (38 packed FP32 operations, 8 ex2, 2 rcp,
                               2 lg2) as independent chains, iters / 4 iterations; reported in
                               state-bins per second (one iteration = two state-bins).  The FMA
                               and MUFU pipes overlap only in part, so this rate is below both
                               single-pipe ceilings: it is what the mix itself allows. */
    LISA_PIPE_N_OPS = 7
} lisa_pipe_op;

/* Measures, on the current device, the sustained rate of each lisa_pipe_op in lane operations
 * per second (one lane operation = one result: an ex2, a reciprocal, a log2 or an FMA; a
 * packed FMA counts two; LISA_PIPE_MIX in state-bins per second) and writes them to
 * rates[LISA_PIPE_N_OPS] (HOST array, caller-owned).
 *  - iters: chain steps per thread (>= 16; 2048 runs each kernel for roughly a millisecond).
 *  - Each kernel is launched once untimed, then timed over `reps` (>= 1) launches on `stream`;
 *    the best repetition is reported.
 *  - The call allocates a small device buffer (the chains' results, so that nothing is
 *    optimised away), synchronises `stream` and frees the buffer before it returns.
 * Errors: LISA_ERR_NULL (rates NULL), LISA_ERR_VALUE (iters < 16 or reps < 1),
 * LISA_ERR_ALLOC, LISA_ERR_CUDA. */
lisa_status lisa_pipe_rates(int32_t iters, int32_t reps, double* rates, lisa_stream_t stream);

/* Per-kernel device times of lisa_psd_loglike on one lisa_data object, for attributing a step's
 * time to its kernels (the roofline of the dominant kernel).
 *
 * lisa_data_set_profiling(data, 1) creates four CUDA events owned by `data` (destroyed with it);
 * while enabled, every lisa_psd_loglike call on `data` that is not being captured into a CUDA
 * graph records them on its stream around its kernels (the state-parameter kernel of an FP32
 * call runs before the first event).  Captured calls record nothing.
 * enable = 0 stops the recording.  Errors: LISA_ERR_NULL, LISA_ERR_CUDA (event creation).
 *
 * lisa_psd_loglike_grad calls are recorded the same way.
 *
 * lisa_data_kernel_ms waits for the most recent recorded call to finish (host synchronisation on
 * its last event) and writes ms[3] (HOST, caller-owned), in milliseconds.  After
 * lisa_psd_loglike: [0] the main likelihood kernel (fused FP32 or plain FP64), [1] the
 * compensated kernel for routed states (0 in FP64 mode), [2] the finalize kernel.  After
 * lisa_psd_loglike_grad: [0] the adjoint kernel (FP32 or FP64), [1] the FP32 call's compensated
 * and fallback passes (0 in FP64 mode), [2] the adjoint epilogue.  Errors: LISA_ERR_NULL;
 * LISA_ERR_VALUE when profiling is off or no call has been recorded since it was enabled;
 * LISA_ERR_CUDA. */
lisa_status lisa_data_set_profiling(lisa_data* data, int32_t enable);
lisa_status lisa_data_kernel_ms(const lisa_data* data, float* ms);

/* Test of the timeout path; no counterpart in the paper.  The fused and compensated likelihood
 * kernels stage bin tables by asynchronous bulk copies and wait for them on mbarriers with a
 * bounded number of polls; a wait that runs out raises the workspace's error word (see
 * lisa_workspace_status), lets the copies already issued land and stops the CTA.
 * wait_limit (>= 1, default 2^20) sets the number of polls for later calls on `data`;
 * skip_copies != 0 makes the fused FP32 kernel issue no copies at all, so its first wait runs
 * out with nothing in flight -- for tests only: the log-likelihoods are then NaN.  Calls already
 * enqueued are not affected.  Errors: LISA_ERR_NULL, LISA_ERR_VALUE (wait_limit 0). */
lisa_status lisa_data_set_test_wait(lisa_data* data, int32_t skip_copies, uint32_t wait_limit);

#ifdef __cplusplus
}
#endif

#endif /* LISA_PEAKS_H */
