/*
 * lisa_psd.h -- C ABI of the GB300 (sm_103a) library for the batched, spline-perturbed
 * Whittle/Wishart log-likelihood of averaged A/E/T periodograms (arXiv:2507.06300).
 *
 * The library evaluates, for every walker x temperature state of a tempered ensemble at once,
 *
 *     log L(theta) = - sum_i nu_i sum_c [ P_c(f_i) / S_c(f_i) + ln S_c(f_i) ]          (1)
 *
 *     S_c(f) = S_n,cc(f | A_OMS, A_TM) 10^{P_n,c(log10 f)}
 *            + S_h,cc(f | A, n)        10^{P_h(log10 f)}                              (2)
 *
 * (1) is the per-bin complex-Wishart log-density -tr(C^-1 Y) - nu log|C| with Y = nu P and a
 * diagonal covariance C = diag(S_AA, S_EE, S_TT), summed over bins (Sec. III.C); the printed
 * factor 1/2 in C is not applied (the periodogram is normalised to the one-sided PSD,
 * Sec. III.A), and nu = 1 is the Whittle likelihood.  (2) is Eq. (splines) of Sec. III.A with
 * the noise template of Eq. (noise_tdi) and the SGWB template of Eq. (pl) / Eq. (Sh).  The
 * perturbations P are variable-knot Akima splines (Appendix A; natural cubic splines as the
 * alternative kind) in x = log10 f, with edge knots fixed at the dataset's x_lo / x_hi and
 * in-between knots (x_k, w_k) in any order; fewer than two in-between knots give the linear
 * interpolant (Sec. III.A).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are DEVICE pointers (cudaMalloc'd or torch-allocated memory on the
 *    current device); everything else is host memory.  The caller owns every array it passes;
 *    the library owns only what lisa_data_create allocates, freed by lisa_data_destroy.
 *  - Calls that take a cudaStream_t are asynchronous and stream-ordered: they enqueue kernels
 *    and return; results are valid once the stream reaches them.  Only lisa_data_create and
 *    lisa_data_set_tiling synchronise (they upload tables and work lists).
 *  - Argument or shape errors return a non-zero lisa_status and launch nothing.  A CUDA
 *    launch error returns LISA_ERR_CUDA.  No C++ exception crosses the ABI.
 *  - A state whose knots or parameters are invalid is not a call failure: lisa_spline_setup
 *    writes the knot bits (LISA_STATE_BAD_COUNT .. LISA_STATE_BAD_AMPLITUDE) to its status word;
 *    such a state, and any state whose parameters are non-finite or whose PSD or log-likelihood
 *    leaves the finite range of the chosen precision, gets log L = -inf and a zero gradient.
 *  - Every layout is row-major (C order) with the shapes given.
 */
#ifndef LISA_PSD_H
#define LISA_PSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lisa_stream_t; /* same type as cudaStream_t; NULL = legacy stream */

typedef enum lisa_status {
    LISA_SUCCESS = 0,
    LISA_ERR_NULL = 1,        /* a required pointer is NULL */
    LISA_ERR_VALUE = 2,       /* a scalar argument is out of range */
    LISA_ERR_SHAPE = 3,       /* sizes disagree with the dataset object */
    LISA_ERR_DATA = 4,        /* input table has non-finite / non-positive / unordered entries */
    LISA_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
    LISA_ERR_ALLOC = 6,       /* device or host allocation failed */
    LISA_ERR_WORKSPACE = 7,   /* workspace or spline buffer too small or misaligned */
    LISA_ERR_TIMEOUT = 8      /* a bounded device-side wait gave up (kernel returned early) */
} lisa_status;

typedef enum lisa_precision {
    LISA_FP32 = 0, /* FP32 tables and per-bin arithmetic, FP64 bin sums (the fast path) */
    LISA_FP64 = 1  /* FP64 throughout (the plain reference path on the GPU) */
} lisa_precision;

typedef enum lisa_spline_kind {
    LISA_SPLINE_AKIMA = 0,   /* Appendix A, SciPy-style end slopes */
    LISA_SPLINE_NATURAL = 1  /* natural cubic (second derivative zero at both edges) */
} lisa_spline_kind;

typedef enum lisa_sgwb_model {
    LISA_SGWB_NONE = 0,       /* noise-only model: no SGWB term and no SGWB spline */
    LISA_SGWB_POWER_LAW = 1,  /* h^2 Omega = A (f / f_ref)^n1           (Eq. pl) */
    LISA_SGWB_BROKEN = 2      /* n1 below f_ref, n2 at and above f_ref (same A at f_ref) */
} lisa_sgwb_model;

typedef enum lisa_tdi_form {
    LISA_TDI_PRINTED = 0,  /* prefactor sin^2(u) sin^4(u) as printed in Eq. (noise_tdi) */
    LISA_TDI_SIN2_2U = 1   /* prefactor sin^2(u) sin^2(2u) */
} lisa_tdi_form;

/* Covariance of the A, E, T data per bin.
 *  LISA_COV_DIAGONAL: C = diag(S_AA, S_EE, S_TT) (Sec. III.A, the paper's analysis).
 *  LISA_COV_FULL: the dense covariance Sec. III.A names as the complete analysis, with six
 *    flexible noise terms (the paper leaves its positive-definite construction to another
 *    reference; this library's reading):
 *      C = D^1/2 R D^1/2 + H,  D = diag(S_n,cc 10^{P_n,c}),  H = diag(S_h,cc 10^{P_h}),
 *      R = L L^T,  L = [[1, 0, 0], [r_AE, s_AE, 0], [r_AT, r_ET s_AT, s_AT s_ET]],
 *      r = z / sqrt(1 + z^2),  s = 1 / sqrt(1 + z^2),
 *    where z_AE, z_AT, z_ET are three more variable-knot splines whose values (not exponents) set
 *    the correlations: positive definite for any spline values, the diagonal model at z = 0.
 *    Requires n_channels = 3; the per-bin term is -nu [tr(C^-1 P) + ln det C] with the Hermitian
 *    averaged periodogram P, of which only the real parts of the off-diagonal entries enter (C is
 *    real). */
typedef enum lisa_cov_model {
    LISA_COV_DIAGONAL = 0,
    LISA_COV_FULL = 1
} lisa_cov_model;

/* Per-state status bits (0 = valid). */
#define LISA_STATE_BAD_COUNT 1     /* in-between knot count outside [0, kmax] */
#define LISA_STATE_BAD_POSITION 2  /* position non-finite or not strictly inside (x_lo, x_hi) */
#define LISA_STATE_DUPLICATE 4     /* two in-between knots share a position */
#define LISA_STATE_BAD_AMPLITUDE 8 /* non-finite knot amplitude */
#define LISA_STATE_BAD_THETA 16    /* non-finite template parameter (oracle-side bit; the GPU
                                      entry points report such a state as log L = -inf) */
#define LISA_STATE_NONFINITE 32    /* the PSD or the log-likelihood came out non-finite
                                      (likewise reported by the GPU as log L = -inf) */

#define LISA_N_THETA 5   /* theta per state: a_oms, a_tm, log10 A, n1, n2 */
#define LISA_MAX_KNOTS 62 /* largest kmax (in-between knots per spline) */

/* One or more datasets, each with its bins and the states evaluated on it.
 * Dataset d owns bins [bin_offset[d], bin_offset[d+1]) and states
 * [state_offset[d], state_offset[d+1]); n_bins = bin_offset[n_datasets],
 * n_states = state_offset[n_datasets].  All arrays are HOST memory, copied at create time. */
typedef struct lisa_data_desc {
    int32_t n_datasets;        /* >= 1 */
    int32_t n_channels;        /* 2 (A, E) or 3 (A, E, T) */
    int32_t sgwb_model;        /* lisa_sgwb_model */
    int32_t tdi_form;          /* lisa_tdi_form */
    const int64_t* bin_offset;   /* [n_datasets+1], nondecreasing, bin_offset[0] = 0 */
    const int64_t* state_offset; /* [n_datasets+1], nondecreasing, state_offset[0] = 0 */
    const double* freq;        /* [n_bins] bin frequencies f_i in Hz, > 0, increasing per dataset */
    const double* nu;          /* [n_bins] degrees of freedom n_i of the averaged periodogram, >= 0 */
    const double* periodogram; /* [n_channels][n_bins] averaged auto-powers P_c(f_i), > 0, finite */
    const double* response;    /* [n_channels][n_bins] SGWB response R_c(f_i) >= 0; NULL if NONE */
    const double* x_lo;        /* [n_datasets] left edge knot position (log10 Hz) */
    const double* x_hi;        /* [n_datasets] right edge knot position, > x_lo */
    const double* f_ref;       /* [n_datasets] power-law reference / break frequency (Hz) > 0 */
    int32_t cov_model;         /* lisa_cov_model */
    const double* periodogram_cross; /* LISA_COV_FULL: [3][n_bins] real parts of the averaged
                                        periodogram's P_AE, P_AT, P_ET (finite); NULL otherwise */
} lisa_data_desc;

typedef struct lisa_data lisa_data; /* opaque: device tables + work decomposition */

/* Per-state template parameters.  theta_dev [n_states][LISA_N_THETA] (device, FP64):
 *   a_oms = A_OMS / 1e-12 m/sqrt(Hz), a_tm = A_TM / 1e-15 m/s^2/sqrt(Hz)   (Table I units)
 *   log10 A, n1, n2 of the SGWB (n2 is read only by LISA_SGWB_BROKEN; for the power law the
 *   slope is n1).  Entries the model does not use are ignored. */
typedef struct lisa_params {
    int32_t n_states;
    const double* theta_dev;
} lisa_params;

/* Variable-knot perturbation splines, n_splines = n_channels + (sgwb_model != NONE)
 * + (cov_model == LISA_COV_FULL ? 3 : 0): spline a = 0..n_channels-1 perturbs the noise of
 * channel A, E (, T); spline n_channels perturbs the SGWB (shared by all channels) when the model
 * has one; with the full covariance the last three are z_AE, z_AT, z_ET.  All arrays are DEVICE
 * memory:
 *   count_dev [n_states][n_splines]           in-between knots k (0..kmax)
 *   x_dev     [n_states][n_splines][kmax]     in-between positions log10 f, any order
 *   w_dev     [n_states][n_splines][kmax+2]   slot 0 = w_0 (left edge), 1+j = knot j,
 *                                             kmax+1 = w_n (right edge)  */
typedef struct lisa_knots {
    int32_t n_states;
    int32_t n_splines;
    int32_t kmax;   /* 0..LISA_MAX_KNOTS */
    int32_t kind;   /* lisa_spline_kind */
    const int32_t* count_dev;
    const double* x_dev;
    const double* w_dev;
} lisa_knots;

/* Tiling of the fused likelihood kernels (chosen by the autotuner; defaults are sane). */
typedef struct lisa_tiling {
    int32_t tile_bins;      /* bins staged per work item: multiple of 32, 64..2048 (..1024 for
                               the dense covariance) */
    int32_t states_per_cta; /* states per work item: power of two, 16..128 */
    int32_t group;          /* bins processed between interval checks: 2, 4 or 8 */
    int32_t ctas_per_sm;    /* persistent grid = SMs x this (0 = occupancy limit) */
} lisa_tiling;

/* Sizes of the dataset object and the layout of the gradient. */
typedef struct lisa_data_info {
    int64_t n_bins, n_states;
    int32_t n_datasets, n_channels, n_splines, sgwb_model;
    int64_t n_items;          /* work items of the fused kernels under the current tiling */
    int32_t n_sm;             /* SMs of the device the object lives on */
    lisa_tiling tiling;
} lisa_data_info;

/* ---- dataset --------------------------------------------------------------------------- */

/* Validates the description, uploads it, and runs the per-bin precompute on `stream`
 * (Sec. II.B/II.C templates per bin in FP64, u = 2 pi f L / c with 1 - cos u = 2 sin^2(u/2),
 * normalisation of the template tables by the periodogram, the constant -sum nu sum_c ln P_c).
 * Synchronises the stream.  On success *out owns device memory until lisa_data_destroy. */
lisa_status lisa_data_create(const lisa_data_desc* desc, lisa_stream_t stream, lisa_data** out);
lisa_status lisa_data_destroy(lisa_data* data);
lisa_status lisa_data_get_info(const lisa_data* data, lisa_data_info* info);
/* Replaces the tiling (rebuilds the work list; synchronous).  Invalid fields -> LISA_ERR_VALUE. */
lisa_status lisa_data_set_tiling(lisa_data* data, const lisa_tiling* tiling);

/* ---- spline setup (knot sort + slopes + coefficients, Appendix A) ------------------------ */

/* Bytes of the caller-allocated spline buffer for this dataset's states and kmax. */
size_t lisa_spline_buf_bytes(const lisa_data* data, int32_t kmax, lisa_precision precision);

/* Sec. III.A knot scheme and Appendix A (one warp per spline): sorts each spline's in-between
 * knots, appends the edges, computes the Akima slopes (or the natural-cubic second derivatives
 * by a warp-parallel tridiagonal solve) and the per-interval cubic coefficients, and writes
 * them to spline_buf_dev (256-byte aligned, at least lisa_spline_buf_bytes long; the layout is
 * private to the library and depends on the precision).  In FP32 mode it also decides which
 * states need the compensated evaluation (ill-conditioned intervals) and records them in the
 * buffer.  state_status_dev [n_states] (may be NULL) receives the LISA_STATE_* bits of each
 * state; the buffer keeps its own copy.  Errors: LISA_ERR_NULL, LISA_ERR_VALUE (kmax or kind),
 * LISA_ERR_SHAPE (n_states / n_splines differ from the data object), LISA_ERR_WORKSPACE. */
lisa_status lisa_spline_setup(const lisa_data* data, const lisa_knots* knots,
                              lisa_precision precision, void* spline_buf_dev, size_t spline_buf_bytes,
                              int32_t* state_status_dev, lisa_stream_t stream);

/* ---- log-likelihood ------------------------------------------------------------------------ */

/* Bytes of scratch workspace the likelihood entry points need (per-(state, tile) partial sums of
 * the fused and of the compensated kernel, per-state FP32 parameters and the compensated
 * kernel's per-state work list).
 * with_grad = 0 for lisa_psd_loglike, 1 for lisa_psd_loglike_grad. */
size_t lisa_workspace_bytes(const lisa_data* data, int32_t kmax, lisa_precision precision,
                            int32_t with_grad);

/* Eq. (1) for every state: fused spline evaluation, PSD assembly (2), per-bin terms and a
 * deterministic FP64 reduction over bins (with LISA_COV_FULL, the dense covariance's per-bin term
 * -nu [tr(C^-1 P) + ln det C], from a per-bin 3x3 solve and log-determinant of C scaled to unit
 * diagonal).  loglike_dev [n_states] (FP64).  spline_buf_dev is
 * the output of lisa_spline_setup with the same precision and kmax.  workspace_dev: at least
 * lisa_workspace_bytes(..., 0) bytes, 256-byte aligned, contents ignored and overwritten.
 * Calls that share a workspace must not overlap on the GPU.  FP32 mode returns LISA_ERR_SHAPE
 * when the states times tiles of the current tiling exceed 2^32 - 1. */
lisa_status lisa_psd_loglike(const lisa_data* data, const lisa_params* params,
                             const void* spline_buf_dev, size_t spline_buf_bytes, int32_t kmax,
                             double* loglike_dev, void* workspace_dev, size_t workspace_bytes,
                             lisa_precision precision, lisa_stream_t stream);

/* Device-side status of the most recent lisa_psd_loglike or lisa_psd_loglike_grad call that
 * used workspace_dev: synchronises `stream` (the stream that call ran on), reads the
 * workspace's error word and returns LISA_SUCCESS, or LISA_ERR_TIMEOUT when a bounded wait of
 * the fused or compensated kernel gave up (that call's kernels stopped early and every log L it
 * wrote is NaN; the CUDA context stays usable).  The likelihood calls themselves are
 * asynchronous and cannot return a device-side status.  Errors: LISA_ERR_NULL,
 * LISA_ERR_WORKSPACE (misaligned), LISA_ERR_CUDA. */
lisa_status lisa_workspace_status(const void* workspace_dev, lisa_stream_t stream);

/* log L and its gradient for every state (hand-written adjoint of Sec. III.C's Wishart term;
 * LISA_COV_DIAGONAL data only, LISA_ERR_VALUE for the full covariance; the spline coefficients
 * are recomputed from the knots, nothing per bin is stored).  grad_dev
 * [n_states][LISA_N_THETA + n_splines*(2*kmax+2)] (FP64): d log L / d theta (a_oms, a_tm,
 * log10 A, n1, n2), then per spline d/d(w slots 0..kmax+1) and d/d(x slots 0..kmax-1);
 * unused slots are 0.  spline_buf_dev must come from lisa_spline_setup on the same knots.
 * FP32 mode: bins on ill-conditioned spline intervals (the states lisa_spline_setup routes) take
 * a compensated pass, and states whose FP32 sums leave the FP32 range (PSD values beyond about
 * 2^+-126 somewhere) are redone within the call by a log-domain pass (log2 of each PSD from the
 * float-float spline values, FP64 for 1/S and the sums) and an FP64 reverse map; such a call
 * takes somewhat longer.  workspace_dev: at least lisa_workspace_bytes(..., precision, 1)
 * bytes, 256-byte aligned (in FP32 mode it also holds that pass's per-state flags). */
lisa_status lisa_psd_loglike_grad(const lisa_data* data, const lisa_params* params,
                                  const lisa_knots* knots, const void* spline_buf_dev,
                                  size_t spline_buf_bytes, double* loglike_dev, double* grad_dev,
                                  void* workspace_dev, size_t workspace_bytes,
                                  lisa_precision precision, lisa_stream_t stream);

/* Model PSD S_c(f_i) of (2) for every state in physical units (FP64; with the full covariance,
 * the diagonal C_cc = S_n,cc 10^{P_n,c} + S_h,cc 10^{P_h}):
 * psd_dev [n_states][n_channels][n_bins_of_its_dataset], states concatenated in order
 * (state s of dataset d starts at sum over earlier states of n_channels * their dataset's
 * bins).  Uses the FP64 spline buffer. */
lisa_status lisa_model_psd(const lisa_data* data, const lisa_params* params,
                           const void* spline_buf_dev_fp64, size_t spline_buf_bytes, int32_t kmax,
                           double* psd_dev, lisa_stream_t stream);

/* ---- data preparation ------------------------------------------------------------------------
 * The inputs of lisa_data_create from frequency-domain data (Sec. III.C).  Frequency samples are
 * uniform, f_k = f0 + k df (the grid of a discrete Fourier transform), and complex values are
 * interleaved (re, im) FP64 pairs. */

/* Synthetic frequency-domain data of a stationary Gaussian process with one-sided PSD S
 * (Sec. II.D: generated directly in the frequency domain, normalised so that E|d(f)|^2 = S(f)):
 *     d_c(f_k) = sqrt(S_c(f_k) / 2) (z_c,k,0 + i z_c,k,1).
 * psd_dev [n_channels][n_freq] (FP64, >= 0), normal_dev [n_channels][n_freq][2] standard normal
 * draws supplied by the caller, d_dev [n_channels][n_freq][2] out (may alias normal_dev).
 * Errors: LISA_ERR_NULL, LISA_ERR_VALUE (n_channels < 1, n_freq < 0). */
lisa_status lisa_fd_synthesize(const double* psd_dev, const double* normal_dev, int32_t n_channels,
                               int64_t n_freq, double* d_dev, lisa_stream_t stream);

/* Averaged periodogram (Sec. III.C): bin i holds the frequency samples
 * [bin_offset[i], bin_offset[i+1]) and
 *     P_c(f_i) = (1 / n_i) sum_k |d_c(f_k)|^2,   nu_i = n_i,   f_i = f0 + df (b0 + b1 - 1) / 2
 * (the diagonal of the averaged periodogram matrix: the A, E, T covariance is diagonal), so that
 * nu_i P_c(f_i) follows the 1x1 complex Wishart (Gamma) law of the likelihood (1).
 * d_dev [n_channels][n_freq][2]; bin_offset_dev [n_bins + 1] (int64, non-decreasing; entries are
 * clamped to [0, n_freq]); out: p_dev [n_channels][n_bins], f_dev [n_bins], nu_dev [n_bins]
 * (FP64).  A bin with no samples gets P = NaN and nu = 0.  Sums are FP64 in a fixed order.
 * Errors: LISA_ERR_NULL, LISA_ERR_VALUE (n_channels < 1, n_freq < 0, n_bins < 0, df <= 0). */
lisa_status lisa_averaged_periodogram(const double* d_dev, int32_t n_channels, int64_t n_freq, double f0,
                                      double df, const int64_t* bin_offset_dev, int64_t n_bins,
                                      double* p_dev, double* f_dev, double* nu_dev, lisa_stream_t stream);

/* ---- allocation-free variant ---------------------------------------------------------------
 * No counterpart in the paper: this is a deployment convenience.
 *
 * lisa_psd_loglike needs a caller-provided scratch workspace.  Some callers cannot obtain one
 * per call: code that runs under a memory manager which forbids further device allocations once
 * a sampler has started (a fixed budget reserved up front, or another framework owning the
 * device heap), or a host sampler written against a C interface with no device allocator at
 * all.  lisa_psd_loglike_noalloc computes exactly what lisa_psd_loglike computes, with the same
 * inputs and outputs, but keeps its scratch (an error flag and the per-state partial sums) in a
 * fixed-size array that lives in the library's own device image, so the call allocates nothing.
 *
 *  - The array holds LISA_NOALLOC_SCRATCH_BYTES (4 MiB): 256 bytes plus 16 bytes per
 *    (state, tile) (the fused and the compensated kernels' partial sums) plus 84 bytes per state
 *    (FP32 parameters, work list), each region rounded up to 256 bytes, i.e.
 *    lisa_workspace_bytes(data, kmax, precision, 0) must not exceed it.  The size depends on the
 *    tiling (lisa_data_set_tiling): the paper-scale workload (131,072 bins, 1,024 states) needs
 *    about 2.1 MiB at 1,024-bin tiles, which fits, but 4.1 MiB at 512-bin tiles, which does not.
 *    Larger problems get LISA_ERR_WORKSPACE and nothing is launched; use lisa_psd_loglike for
 *    them.
 *  - Every GPU that loads the library holds the array until the process exits.
 *  - The device that holds `data` must be current: the array exists once per device, and a
 *    call made with another device current returns LISA_ERR_VALUE.
 *  - Every call looks the array's device address up (cudaGetSymbolAddress, which enqueues
 *    nothing).  The first call on a device may load the library's device code there, so make
 *    it before any stream capture.
 *  - All calls on a device share the one array, and each call overwrites it (the error flag is
 *    cleared on the stream first).  Two calls whose kernels overlap on the GPU race on it:
 *    serialise them (same stream, or events).
 * Arguments, layouts and errors are otherwise those of lisa_psd_loglike. */
#define LISA_NOALLOC_SCRATCH_BYTES (4u * 1024u * 1024u)
lisa_status lisa_psd_loglike_noalloc(const lisa_data* data, const lisa_params* params,
                                     const void* spline_buf_dev, size_t spline_buf_bytes, int32_t kmax,
                                     double* loglike_dev, lisa_precision precision, lisa_stream_t stream);

const char* lisa_status_string(lisa_status status);

#ifdef __cplusplus
}
#endif

#endif /* LISA_PSD_H */
