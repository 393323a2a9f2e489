// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "lisa_debug.cuh"
#include "lisa_psd.h"

#include <nvtx3/nvToolsExt.h>

namespace lisa {

namespace dbg {
// The index-check records of the translation units (lisa_debug.cuh), gathered by lisa_debug_bounds.
cudaError_t read_data(BoundsRecord* out, int reset, const char** file);
cudaError_t read_full(BoundsRecord* out, int reset, const char** file);
cudaError_t read_grad(BoundsRecord* out, int reset, const char** file);
cudaError_t read_loglike(BoundsRecord* out, int reset, const char** file);
cudaError_t read_peaks(BoundsRecord* out, int reset, const char** file);
cudaError_t read_prep(BoundsRecord* out, int reset, const char** file);
cudaError_t read_spline(BoundsRecord* out, int reset, const char** file);
}  // namespace dbg

// An NVTX range over one library call (host side: the range marks the call's launches, which the
// profiler correlates with the kernels); without a profiler attached a push/pop costs nothing
// beyond a null check.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr double kPi = 3.141592653589793238462643;
constexpr double kArm = 2.5e9;                            // arm length L, m (Sec. II.A)
constexpr double kClight = 299792458.0;                   // m/s
constexpr double kH0h = 1.0e5 / 3.0856775814913673e22;   // 100 km/s/Mpc in 1/s
constexpr double kLog2_10 = 3.321928094887362347870319;
constexpr double kLn10 = 2.302585092994045684017991;
constexpr double kLn2 = 0.693147180559945309417232;

constexpr int kRec = 12;         // per-bin fields: x, ell, nu, Goms[3], Gtm[3], Gh[3]
// FP64 bin table: AoS, kRec doubles per bin.  FP32 bin table: blocks of two bins, field k of
// bin 2p+e at [p * kPairRec + 2k + e], so one 16-byte load returns two fields of both bins and
// each field's pair sits in an aligned register pair for the packed FP32x2 instructions.
// Both tables use padded bin indices: every dataset is padded to an even bin count with a
// dummy bin (copy of its last bin with nu = 0).
constexpr int kPairRec = 2 * kRec;
constexpr int kCross = 4;        // FP64 cross-spectral fields per bin (three and a pad)
constexpr int kPairCross = 8;    // FP32 cross-spectral floats per pair block
constexpr int kThreads = 256;    // threads of the plain FP64 likelihood kernel
constexpr int kThreads32 = 128;  // threads of the fused FP32 likelihood kernel
constexpr int kMaxStatesPerItem = 128;  // state lanes of a work item (<= both thread counts)
// Per-interval records, 64 bytes in both precisions:
//   FP64: xl, xr, a, b, c, d, 0, 0 (coefficients about xl, log10 units)
//   FP32: [0] xr  [1] xo  [2..5] c0..c3  [6] xl  [7] conditioning T      (first 32 bytes)
//         [8] xo_lo  [9..12] c0..c3 low parts  [13..15] 0                (second 32 bytes)
//         coefficients about the interval midpoint xo, scaled to log2 units; hi + lo is the
//         float-float value split into two floats.
constexpr int kSplineRec = 8;    // doubles per FP64 record
constexpr int kSplineRec32 = 16; // floats per FP32 record
// States whose FP32 perturbation spline has an interval with conditioning
// T = |c0| + |c1| r + |c2| r^2 + |c3| r^3 (log2 units, r = largest |x - xo| of its bins) above
// this bound are evaluated by the compensated (float-float, log-domain) kernel.
constexpr double kRobustT = 32.0;
constexpr int kRouted = 1 << 16;        // internal status bit: state routed to the compensated kernel
constexpr int kUserBits = 0xffff;       // LISA_STATE_* bits
constexpr int kStatusNonfinite = LISA_STATE_NONFINITE;
constexpr unsigned kWaitLimit = 1u << 20;   // bounded spin on an mbarrier (then give up)
constexpr int kErrTimeout = 1;              // workspace error word: a bounded wait gave up
constexpr int kMaxTileBins = 2048;          // 2 staged tiles x 48 B/bin must fit in 227 KB
constexpr int kMaxTileBinsFull = 1024;      // dense covariance: 2 staged tiles x 64 B/bin
constexpr int kAdjBins = 2048;              // bins per (state, range) in the adjoint
// Work balance of the fused kernel: an item (a tile of bins x a chunk of states) costs
// (bins + kKnotBinsPerDecade x its width in log10 f) per state.  The second term stands for the
// interval advances: knots are drawn uniformly in log10 f, so the low-frequency tiles (few bins,
// wide in log10 f) hold most of them, and each advance stalls its warp on record loads.
constexpr double kKnotBinsPerDecade = 2500.0;
constexpr int kXsStride = 32;               // bins between the host copies of log10 f
constexpr int kBlockItemsPerCta = 16;       // contiguous blocks need this many items per CTA
constexpr double kBlockThreadBins = 128.0;  // and fewer bins per thread and item than this

// One unit of work of the fused kernels: a tile of bins of one dataset and a chunk of its
// states.  Threads map to (state lane, bin sub-range): lane = tid % sc, range = tid / sc.
struct WorkItem {
    int64_t bin0;   // first bin (global index)
    int32_t nb;     // bins in the tile
    int32_t s0;     // first state (global index)
    int32_t ns;     // states in the chunk (<= sc)
    int32_t sc;     // state lanes of this dataset's items (power of two, <= kMaxStatesPerItem)
    int32_t tile;   // tile index within the dataset
    int32_t ds;     // dataset index
};
static_assert(sizeof(WorkItem) == 32, "WorkItem layout");

// One unit of the adjoint: a range of kAdjBins bins of one dataset and up to 32 of its states
// (one warp, lanes = states).
struct AdjUnit {
    int32_t ds, rho, s0, ns;
};

struct DatasetDev {
    int64_t bin0, nbins;     // bin range: bin0 in padded indexing, nbins real bins
    int64_t npad;            // nbins rounded up to even (bins [bin0, bin0 + npad) in the tables)
    int64_t rbin0;           // first bin in the caller's (unpadded) arrays
    int64_t pbase;           // first partial slot of the dataset (partials are [tile][state])
    int64_t psd_base;        // first element of the dataset's states in a model-PSD output
    int32_t s0, ns;          // state range
    int32_t ntiles;          // tiles of tile_bins bins
    int32_t nranges;         // adjoint ranges of kAdjBins bins
    double x_lo, x_hi;       // edge knot positions
    double xb_min, xb_max;   // log10 f of the first and last bin
    double f_ref;
    double K;                // -sum_i nu_i sum_c ln P_c,i
    double Cnu;              // C * sum_i nu_i
};

}  // namespace lisa

struct lisa_data {
    int device = 0;
    int n_sm = 0;
    int32_t n_datasets = 0, C = 0, nsp = 0, sgwb_model = 0, tdi_form = 0;
    int32_t cov = 0;                 // lisa_cov_model
    // LISA_COV_FULL: per bin the real parts of P_AE, P_AT, P_ET over sqrt(P_aa P_bb):
    // FP64 [n_pad][4] (last entry 0), FP32 in blocks of two bins [n_pad / 2][8]
    // (field k of bin 2p+e at [p * 8 + 2k + e], entries 6, 7 zero)
    double* d_cross64 = nullptr;
    float* d_cross32 = nullptr;
    int64_t n_bins = 0, n_states = 0;
    int64_t n_pad = 0;               // padded bin count of the tables
    std::vector<int64_t> h_bin_off, h_state_off;
    // log10 f of every kXsStride-th bin of each dataset and of its last bin (host copy for the
    // work balance), dataset k's entries from h_xs_off[k]
    std::vector<double> h_xs;
    std::vector<int64_t> h_xs_off;
    std::vector<lisa::DatasetDev> h_ds;
    lisa::DatasetDev* d_ds = nullptr;
    int32_t* d_state_ds = nullptr;   // [n_states] dataset of each state
    float* d_rec32 = nullptr;        // [n_pad / 2][kPairRec]
    double* d_rec64 = nullptr;       // [n_pad][kRec]
    double* d_P = nullptr;           // [C][n_bins] periodogram (unpadded; normaliser of the tables)
    float* d_xlo32 = nullptr;        // [n_pad] log10 f - (float)log10 f (low part of x)
    float* d_elllo32 = nullptr;      // [n_pad] low part of ell = log2(f / f_ref)
    lisa_tiling tiling{};
    lisa::WorkItem* d_items = nullptr;
    int32_t* d_cta_first = nullptr;  // fused kernel: first item of each CTA (fgrid + 1 entries)
    int32_t fgrid = 0;               // CTAs of the fused FP32 launch
    int32_t rgrid = 0;               // CTAs of the compensated kernel's persistent launch
    bool fblocks = false;            // contiguous cost-balanced blocks (else longest-first assignment)
    lisa::AdjUnit* d_adj_units = nullptr;
    int64_t n_adj_units = 0;
    int64_t* d_adj_prefix = nullptr; // [n_states] adjoint ranges of all earlier states
    int64_t adj_ranges = 0;          // sum over states of their dataset's ranges
    int64_t n_items = 0;
    int64_t n_partials = 0;          // sum over datasets of states x tiles
    // per-kernel timing of lisa_psd_loglike (lisa_data_set_profiling): events around the main,
    // compensated and finalize kernels of the most recent uncaptured call
    cudaEvent_t prof_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool prof_on = false;
    mutable bool prof_valid = false;
    // polls of a bounded mbarrier wait before the fused and compensated kernels give up, and the
    // test-only switch that makes the fused kernel issue no copies (lisa_data_set_test_wait)
    uint32_t wait_limit = lisa::kWaitLimit;
    int32_t test_skip_copies = 0;
};

namespace lisa {

// Spline buffer layout (64-byte records in both precisions):
//   int32 status[S] | int32 nint[S*nsp] | int32 route_count, route_list[S] | rec[S][nsp][kmax+1]
//   | float2 hull[S] | float xr[S][nsp][kxr_stride(kmax)]
// each region starting on a 256-byte boundary.  xr (FP32 mode) repeats each interval's right end
// contiguously, +inf for the last interval and the padding, so that the interval holding x is
// the number of entries <= x, found from a few independent 16-byte loads.  route_list holds, in no particular order, the
// states the FP32 path sends to the compensated kernel (a record for inspection: the likelihood
// call finds them by their status bit and builds its own work list); hull[s] = (lowest left end,
// highest right end) in x of state s's ill-conditioned intervals, (+inf, -inf) when it has none
// (both unused in FP64 mode).
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
struct SplineLayout {
    size_t off_status, off_nint, off_route, off_rec, off_hull, off_kxr, bytes;
};
constexpr size_t kRecBytes = 64;
// entries per spline of the right-end table: kmax + 1 rounded up to a multiple of 4
__host__ __device__ inline int kxr_stride(int kmax) { return (kmax + 4) & ~3; }
inline SplineLayout spline_layout(int64_t S, int nsp, int kmax) {
    SplineLayout L;
    L.off_status = 0;
    L.off_nint = align256(sizeof(int32_t) * (size_t)S);
    L.off_route = L.off_nint + align256(sizeof(int32_t) * (size_t)S * nsp);
    L.off_rec = L.off_route + align256(sizeof(int32_t) * ((size_t)S + 1));
    L.off_hull = L.off_rec + align256((size_t)S * nsp * (kmax + 1) * kRecBytes);
    L.off_kxr = L.off_hull + align256(sizeof(float) * 2 * (size_t)S);
    L.bytes = L.off_kxr + sizeof(float) * (size_t)S * nsp * kxr_stride(kmax);
    return L;
}

// Workspace layout of the forward entry point:
//   int32 err flag (256 B) | double partial[n_partials]
// Per-state FP32 parameters, derived once per likelihood call from theta (FP64) so that the
// per-bin kernels touch no FP64 arithmetic: a_oms^2, a_tm^2, A = 10^log10A, the SGWB slopes,
// and log2 A and the slopes as float-float pairs for the compensated kernel.
struct StateParams {
    float ao2, at2, Af, n1;
    float n2, lA_hi, lA_lo, n1_lo;
    float n2_lo, pad0, pad1, pad2;
};
static_assert(sizeof(StateParams) == 48, "three float4");

// Work list of the compensated kernel, built per call by the state-parameter kernel: one entry
// per routed state with at least one tile inside the x-extent of its ill-conditioned intervals.
// A unit is one (state, tile); the entries are in the order of a single 64-bit counter,
// (entries << 32) + units, advanced by one atomic add per entry, so u0 increases along the list.
struct RobustEntry {
    int32_t s, t0;      // state, first live tile
    uint32_t u0;        // first unit
    int32_t nt;         // live tiles (>= 1)
    int64_t b0;         // first bin of tile t0 (padded global index)
    uint32_t p0;        // partial slot of (s, t0); tile t0 + k has slot p0 + k
    int32_t nb_last;    // bins in tile t0 + nt - 1 (all earlier tiles hold tile_bins)
};
static_assert(sizeof(RobustEntry) == 32, "two int4");

// Forward workspace: error flag (int32 at 0) and work-list counter (uint64 at 8) in the first
// 256 bytes | FP64 partial sums [state][tile] of the fused kernel | StateParams [S] |
// RobustEntry [S] | int32 entry of each state in the work list (-1: none) [S] | FP64 sums of the
// compensated kernel, one per (state, tile) unit of the work list [up to states x tiles].  The
// two kinds of partial sums live apart, so the two kernels may run at the same time; the
// finalize kernel adds both in a fixed order.
constexpr size_t kWsCounterOff = 8;
inline size_t ws_partials_bytes(const lisa_data* d) { return align256(sizeof(double) * (size_t)d->n_partials); }
inline size_t ws_prm_bytes(const lisa_data* d) { return align256(sizeof(StateParams) * (size_t)d->n_states); }
inline size_t ws_rlist_bytes(const lisa_data* d) { return align256(sizeof(RobustEntry) * (size_t)d->n_states); }
inline size_t ws_rent_bytes(const lisa_data* d) { return align256(sizeof(int32_t) * (size_t)d->n_states); }
struct WsLayout {
    size_t off_partial, off_prm, off_rlist, off_rent, off_rpart, bytes;
};
inline WsLayout ws_layout(const lisa_data* d) {
    WsLayout L;
    L.off_partial = 256;
    L.off_prm = L.off_partial + ws_partials_bytes(d);
    L.off_rlist = L.off_prm + ws_prm_bytes(d);
    L.off_rent = L.off_rlist + ws_rlist_bytes(d);
    L.off_rpart = L.off_rent + ws_rent_bytes(d);
    L.bytes = L.off_rpart + ws_partials_bytes(d);
    return L;
}
inline size_t ws_fwd_bytes(const lisa_data* d) { return ws_layout(d).bytes; }

// Extra workspace of the adjoint entry point (after the forward region); the FP32 call also holds
// a per-state flag (states redone by the fallback pass).
size_t grad_extra_bytes(const lisa_data* d, int kmax, bool fp32);

lisa_status rebuild_work(lisa_data* d);
// The dense-covariance likelihood kernel (LISA_COV_FULL) for the model of d, FP32 bulk or FP64.
cudaError_t launch_full_cov(const lisa_data* d, bool fp32, const double* theta, const StateParams* prm,
                            const int32_t* sstat, const int32_t* nint, const float* kxr, const void* srec, int kmax,
                            double* partial, int* err, cudaStream_t sm);
// Resident CTAs per SM of the fused FP32 kernel under tiling t (its registers and shared memory).
int fused_ctas_per_sm(const lisa_data* d, const lisa_tiling& t);
// Resident CTAs per SM of the compensated kernel for this data object's model.
int robust_ctas_per_sm(const lisa_data* d);

// Per-kernel timing (lisa_data_set_profiling): whether this call records events (profiling on
// and the stream not capturing), and an event record at point k of the call.
inline bool prof_active(const lisa_data* d, cudaStream_t sm) {
    if (!d->prof_on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(sm, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}
inline void prof_mark(const lisa_data* d, bool on, int k, cudaStream_t sm) {
    if (on) cudaEventRecord(d->prof_ev[k], sm);
}
lisa_status check_cuda(cudaError_t e);

}  // namespace lisa
