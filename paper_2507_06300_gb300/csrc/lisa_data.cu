// Dataset object: validation, upload, the per-bin FP64 precompute (templates of Sec. II.B and
// Sec. II.C normalised by the periodogram) and the work decomposition of the fused kernels.
#include <algorithm>
#include <queue>
#include <utility>
#include <cmath>
#include <cstdio>
#include <new>

#include "lisa_internal.cuh"
#include "lisa_debug.h"
#include "lisa_peaks.h"

namespace lisa {

lisa_status check_cuda(cudaError_t e) { return e == cudaSuccess ? LISA_SUCCESS : LISA_ERR_CUDA; }

namespace {

__device__ __forceinline__ int dataset_of_bin(const DatasetDev* ds, int n, int64_t i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ds[mid].bin0 <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-bin precompute in FP64 (one thread per bin).  With u = 2 pi f L / c:
//   A/E noise per unit amplitude^2:  32 T(u) (2 + cos u) S_OMS1,  32 T(u) 4 (1 + cos u + cos^2 u) S_TM1
//   T noise per unit amplitude^2:    64 T(u) (1 - cos u) S_OMS1,  64 T(u) 2 (1 - cos u)^2 S_TM1
//   (Eq. noise_tdi; T(u) = sin^2 u sin^4 u as printed, or sin^2 u sin^2 2u; 1 - cos u is
//   evaluated as 2 sin^2(u/2)), SGWB per unit h^2 Omega: R_c 3 (H0/h)^2 / (4 pi^2 f^3) (Eq. Sh).
// Every table entry is divided by the channel's periodogram P_c(f_i), so the per-bin ratio
// P/S becomes 1/S-hat and the FP32 path works on numbers of order one.
__global__ void prep_kernel(int64_t n_pad, int C, int tdi_form, int sgwb, const double* __restrict__ f,
                            const double* __restrict__ nu, const double* __restrict__ P,
                            const double* __restrict__ R, int64_t n_real, const DatasetDev* __restrict__ ds,
                            int n_ds, double* __restrict__ rec64, float* __restrict__ rec32,
                            float* __restrict__ xlo32, float* __restrict__ elllo32, double* __restrict__ lnP,
                            double* __restrict__ nu_p) {
    int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= n_pad) return;
    int d = dataset_of_bin(ds, n_ds, ip);
    const DatasetDev& D = ds[d];
    const int64_t i = ip - D.bin0;
    const bool dummy = i >= D.nbins;
    const int64_t g = D.rbin0 + (dummy ? D.nbins - 1 : i);   // caller's bin index
    double fi = f[g];
    double u = 2.0 * kPi * fi * kArm / kClight;
    double su, cu;
    sincos(u, &su, &cu);
    double pref;
    if (tdi_form == 0) {
        pref = su * su * su * su * su * su;
    } else {
        double s2u = sin(2.0 * u);
        pref = su * su * s2u * s2u;
    }
    double sh = sin(0.5 * u);
    double omc = 2.0 * sh * sh;
    double lo = 2.0e-3 / fi, cv = 2.0 * kPi * fi / kClight;
    double oms1 = 1.0e-24 * (1.0 + lo * lo * lo * lo) * cv * cv;
    double l2 = 0.4e-3 / fi, h2 = fi / 8.0e-3, ct = 1.0 / (2.0 * kPi * fi * kClight);
    double tm1 = 1.0e-30 * (1.0 + l2 * l2) * (1.0 + h2 * h2 * h2 * h2) * ct * ct;
    double go[3], gt[3], gh[3] = {0.0, 0.0, 0.0};
    go[0] = go[1] = 32.0 * pref * (2.0 + cu) * oms1;
    gt[0] = gt[1] = 32.0 * pref * 4.0 * (1.0 + cu + cu * cu) * tm1;
    go[2] = 64.0 * pref * omc * oms1;
    gt[2] = 64.0 * pref * 2.0 * omc * omc * tm1;
    double conv = 3.0 * kH0h * kH0h / (4.0 * kPi * kPi * fi * fi * fi);
    double r[kRec];
    r[0] = log10(fi);
    r[1] = log2(fi / D.f_ref);
    r[2] = dummy ? 0.0 : nu[g];
    double lsum = 0.0;
    for (int c = 0; c < 3; ++c) {
        double g_o = 0.0, g_t = 0.0, g_h = 0.0;
        if (c < C) {
            double p = P[(size_t)c * n_real + g];
            if (sgwb) gh[c] = R[(size_t)c * n_real + g] * conv;
            g_o = go[c] / p;
            g_t = gt[c] / p;
            g_h = gh[c] / p;
            lsum += log(p);
        }
        r[3 + c] = g_o;
        r[6 + c] = g_t;
        r[9 + c] = g_h;
    }
    lnP[ip] = r[2] * lsum;
    nu_p[ip] = r[2];
    xlo32[ip] = (float)(r[0] - (double)(float)r[0]);
    elllo32[ip] = (float)(r[1] - (double)(float)r[1]);
    const int64_t pb = ip >> 1, e = ip & 1;
    for (int q = 0; q < kRec; ++q) {
        rec64[(size_t)ip * kRec + q] = r[q];
        rec32[(size_t)pb * kPairRec + 2 * q + e] = (float)r[q];
    }
}

// Full covariance: per padded bin the real parts of P_AE, P_AT, P_ET divided by sqrt(P_aa P_bb),
// the off-diagonal entries of the periodogram scaled like the template tables (P-hat_cc = 1).
__global__ void cross_prep_kernel(int64_t n_pad, const double* __restrict__ P, const double* __restrict__ X,
                                  int64_t n_real, const DatasetDev* __restrict__ ds, int n_ds,
                                  double* __restrict__ cross64, float* __restrict__ cross32) {
    const int64_t ip = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= n_pad) return;
    const int d = dataset_of_bin(ds, n_ds, ip);
    const DatasetDev& D = ds[d];
    const int64_t i = ip - D.bin0;
    const int64_t g = D.rbin0 + (i >= D.nbins ? D.nbins - 1 : i);
    const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    const int64_t pb = ip >> 1, e = ip & 1;
    for (int k = 0; k < 3; ++k) {
        const double v = X[(size_t)k * n_real + g] /
                         sqrt(P[(size_t)pr[k][0] * n_real + g] * P[(size_t)pr[k][1] * n_real + g]);
        cross64[(size_t)ip * kCross + k] = v;
        cross32[(size_t)pb * kPairCross + 2 * k + e] = (float)v;
    }
    cross64[(size_t)ip * kCross + 3] = 0.0;
    cross32[(size_t)pb * kPairCross + 6 + e] = 0.f;
}

// Deterministic per-dataset sums (one block per dataset, fixed-order tree):
//   K = -sum_i nu_i sum_c ln P_c,i  and  Cnu = C sum_i nu_i.
__global__ void dataset_sums_kernel(const double* __restrict__ lnP, const double* __restrict__ nu,
                                    DatasetDev* ds, int C) {
    __shared__ double s1[256], s2[256];
    DatasetDev& D = ds[blockIdx.x];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < D.npad; i += blockDim.x) {
        a += lnP[D.bin0 + i];
        b += nu[D.bin0 + i];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D.K = -s1[0];
        D.Cnu = (double)C * s2[0];
    }
}

template <class T>
lisa_status dev_alloc(T** p, size_t n) {
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T)) == cudaSuccess ? LISA_SUCCESS : LISA_ERR_ALLOC;
}

void release(lisa_data* d) {
    for (auto& e : d->prof_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    d->prof_on = false;
    cudaFree(d->d_ds);
    cudaFree(d->d_state_ds);
    cudaFree(d->d_rec32);
    cudaFree(d->d_rec64);
    cudaFree(d->d_P);
    cudaFree(d->d_xlo32);
    cudaFree(d->d_elllo32);
    cudaFree(d->d_cross64);
    cudaFree(d->d_cross32);
    cudaFree(d->d_items);
    cudaFree(d->d_cta_first);
    d->d_cta_first = nullptr;
    cudaFree(d->d_adj_units);
    cudaFree(d->d_adj_prefix);
    d->d_adj_units = nullptr;
    d->d_adj_prefix = nullptr;
    d->d_ds = nullptr;
    d->d_state_ds = nullptr;
    d->d_rec32 = nullptr;
    d->d_rec64 = nullptr;
    d->d_P = nullptr;
    d->d_xlo32 = nullptr;
    d->d_elllo32 = nullptr;
    d->d_cross64 = nullptr;
    d->d_cross32 = nullptr;
    d->d_items = nullptr;
}

int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// Builds the work list for the current tiling: per dataset, chunks of sc states (sc =
// min(states_per_cta, next power of two >= states of the dataset)) times tiles of tile_bins bins.
// With many items per CTA the list is in (dataset, chunk, tile) order and the fused kernel gives
// each CTA a contiguous, cost-balanced block of it, so a CTA mostly walks consecutive tiles of
// the same states; otherwise the items are assigned longest-first (knot-aware cost) to the
// least-loaded CTA and each CTA's share is laid out contiguously.
lisa_status rebuild_work(lisa_data* d) {
    const lisa_tiling& t = d->tiling;
    std::vector<WorkItem> items;
    int64_t pbase = 0;
    for (int k = 0; k < d->n_datasets; ++k) {
        DatasetDev& D = d->h_ds[k];
        D.ntiles = (int32_t)((D.npad + t.tile_bins - 1) / t.tile_bins);
        D.pbase = pbase;
        pbase += (int64_t)D.ns * D.ntiles;
        if (D.ns == 0 || D.npad == 0) continue;
        int sc = std::min(t.states_per_cta, pow2ceil(D.ns));
        sc = std::max(sc, 1);
        for (int32_t s = 0; s < D.ns; s += sc) {
            for (int32_t tile = 0; tile < D.ntiles; ++tile) {
                int64_t b0 = D.bin0 + (int64_t)tile * t.tile_bins;
                int32_t nb = (int32_t)std::min<int64_t>(t.tile_bins, D.bin0 + D.npad - b0);
                WorkItem w;
                w.bin0 = b0;
                w.nb = nb;
                w.s0 = D.s0 + s;
                w.ns = std::min(sc, D.ns - s);
                w.sc = sc;
                w.tile = tile;
                w.ds = k;
                items.push_back(w);
            }
        }
    }
    d->n_partials = pbase;
    const int occ = t.ctas_per_sm > 0 ? t.ctas_per_sm : fused_ctas_per_sm(d, t);
    const int grid = std::max(1, d->n_sm * std::max(occ, 1));
    // contiguous blocks pay off when a CTA has many items and each thread takes few bins from an
    // item (small state chunks: the per-item interval search dominates); with a few items per CTA
    // or wide items, cutting a handful of tiles by cost balances poorly, and a longest-first
    // assignment of the items does better
    double thread_bins = 0.0, weight = 0.0;   // bins one thread takes from an item, state-weighted
    for (const WorkItem& w : items) {
        thread_bins += (double)w.nb * w.sc / kThreads32 * w.ns;
        weight += w.ns;
    }
    d->fblocks = items.size() >= (size_t)kBlockItemsPerCta * (size_t)grid &&
                 thread_bins < kBlockThreadBins * weight;
    // knot-aware cost of each item
    auto x_at = [&](int k, int64_t b) {   // log10 f of bin b of dataset k (b a multiple of
        const double* xs = d->h_xs.data() + d->h_xs_off[k];   // kXsStride, or past the end)
        const int64_t nxs = d->h_xs_off[k + 1] - d->h_xs_off[k];
        const int64_t j = b / kXsStride;
        return j < nxs - 1 ? xs[j] : xs[nxs - 1];
    };
    auto cost_of = [&](const WorkItem& w) {
        const DatasetDev& D = d->h_ds[w.ds];
        const int64_t a = w.bin0 - D.bin0, e = a + w.nb;
        const double dx = D.nbins > 0 ? x_at(w.ds, e) - x_at(w.ds, a) : 0.0;
        return ((double)w.nb + kKnotBinsPerDecade * dx) * (double)w.ns;
    };
    std::vector<int32_t> cta_first((size_t)grid + 1, 0);
    if (d->fblocks) {
        // contiguous blocks of the (dataset, chunk, tile)-ordered list, cut so that every CTA gets
        // the same cost (item boundaries at cost midpoints)
        std::vector<double> pre(items.size() + 1, 0.0);
        for (size_t q = 0; q < items.size(); ++q) pre[q + 1] = pre[q] + cost_of(items[q]);
        size_t q = 0;
        for (int b = 1; b <= grid; ++b) {
            const double target = pre.back() * (double)b / (double)grid;
            while (q < items.size() && 0.5 * (pre[q] + pre[q + 1]) < target) ++q;
            cta_first[b] = (int32_t)(b == grid ? items.size() : q);
        }
    } else {
        // few items per CTA: longest-processing-time-first assignment (costliest item to the
        // least loaded CTA), then each CTA's items laid out contiguously in (dataset, chunk,
        // tile) order, so that consecutive tiles of the same states still carry their intervals
        std::vector<double> cost(items.size());
        std::vector<size_t> order(items.size());
        for (size_t q = 0; q < items.size(); ++q) {
            cost[q] = cost_of(items[q]);
            order[q] = q;
        }
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
        using Load = std::pair<double, int>;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int c = 0; c < grid; ++c) heap.push({0.0, c});
        std::vector<int> owner(items.size());
        for (size_t q : order) {
            Load l = heap.top();
            heap.pop();
            owner[q] = l.second;
            l.first += cost[q];
            heap.push(l);
        }
        std::vector<size_t> perm(items.size());
        for (size_t q = 0; q < items.size(); ++q) perm[q] = q;
        std::stable_sort(perm.begin(), perm.end(), [&](size_t a, size_t b) {
            if (owner[a] != owner[b]) return owner[a] < owner[b];
            const WorkItem &x = items[a], &y = items[b];
            if (x.ds != y.ds) return x.ds < y.ds;
            if (x.s0 != y.s0) return x.s0 < y.s0;
            return x.tile < y.tile;
        });
        std::vector<WorkItem> sorted(items.size());
        for (size_t q = 0; q < items.size(); ++q) {
            sorted[q] = items[perm[q]];
            ++cta_first[(size_t)owner[perm[q]] + 1];
        }
        for (int c = 0; c < grid; ++c) cta_first[c + 1] += cta_first[c];
        items.swap(sorted);
    }
    d->fgrid = grid;
    d->rgrid = std::max(1, d->n_sm * robust_ctas_per_sm(d));
    cudaFree(d->d_items);
    cudaFree(d->d_cta_first);
    d->d_items = nullptr;
    d->d_cta_first = nullptr;
    d->n_items = (int64_t)items.size();
    lisa_status st;
    if ((st = dev_alloc(&d->d_items, items.size())) || (st = dev_alloc(&d->d_cta_first, cta_first.size())))
        return st;
    if (cudaMemcpy(d->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(d->d_cta_first, cta_first.data(), cta_first.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return LISA_ERR_CUDA;
    // device copy of the dataset table (ntiles / pbase changed)
    if (cudaMemcpy(d->d_ds, d->h_ds.data(), d->h_ds.size() * sizeof(DatasetDev),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return LISA_ERR_CUDA;
    return LISA_SUCCESS;
}

}  // namespace lisa

using namespace lisa;

extern "C" {

#ifdef LISA_DEBUG_BOUNDS
namespace lisa {
namespace dbg {
namespace {
// Stores to buf[LISA_IDX(5 + lane, 4)]: every index is out of range and clamped to 3.
__global__ void bounds_selftest_kernel(float* buf) {
    const int i = LISA_IDX((int)threadIdx.x + 5, 4);
    buf[i] = (float)threadIdx.x;
}
}  // namespace
}  // namespace dbg
}  // namespace lisa
#endif

int32_t lisa_debug_bounds_enabled(void) { return lisa::dbg::kBoundsChecked ? 1 : 0; }

lisa_status lisa_debug_bounds(int32_t reset, lisa_bounds_report* out) {
    if (!out) return LISA_ERR_NULL;
    using Reader = cudaError_t (*)(lisa::dbg::BoundsRecord*, int, const char**);
    const Reader readers[] = {lisa::dbg::read_data, lisa::dbg::read_full,  lisa::dbg::read_grad,
                              lisa::dbg::read_loglike, lisa::dbg::read_peaks, lisa::dbg::read_prep,
                              lisa::dbg::read_spline};
    lisa_bounds_report r = {};
    for (Reader rd : readers) {
        lisa::dbg::BoundsRecord b = {};
        const char* file = "";
        if (rd(&b, reset, &file) != cudaSuccess) return LISA_ERR_CUDA;
        if (b.count > 0 && r.count == 0) {
            r.first_index = b.first_index;
            r.first_line = b.first_line;
            std::snprintf(r.first_file, sizeof(r.first_file), "%s", file);
        }
        r.count += (int64_t)b.count;
    }
    *out = r;
    return LISA_SUCCESS;
}

lisa_status lisa_debug_bounds_selftest(lisa_stream_t stream) {
#ifdef LISA_DEBUG_BOUNDS
    float* buf = nullptr;
    if (cudaMalloc(&buf, 4 * sizeof(float)) != cudaSuccess) return LISA_ERR_ALLOC;
    cudaStream_t sm = (cudaStream_t)stream;
    lisa::dbg::bounds_selftest_kernel<<<1, 32, 0, sm>>>(buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    cudaFree(buf);
    return e == cudaSuccess ? LISA_SUCCESS : LISA_ERR_CUDA;
#else
    (void)stream;
    return LISA_ERR_VALUE;
#endif
}

const char* lisa_status_string(lisa_status s) {
    switch (s) {
        case LISA_SUCCESS: return "success";
        case LISA_ERR_NULL: return "a required pointer is NULL";
        case LISA_ERR_VALUE: return "a scalar argument is out of range";
        case LISA_ERR_SHAPE: return "sizes disagree with the dataset object";
        case LISA_ERR_DATA: return "input table has non-finite, non-positive or unordered entries";
        case LISA_ERR_CUDA: return "a CUDA runtime call or kernel launch failed";
        case LISA_ERR_ALLOC: return "device or host allocation failed";
        case LISA_ERR_WORKSPACE: return "workspace or spline buffer too small or misaligned";
        case LISA_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    }
    return "unknown lisa_status";
}

lisa_status lisa_data_create(const lisa_data_desc* desc, lisa_stream_t stream, lisa_data** out) {
    lisa::NvtxRange nvtx_range("lisa_data_create");
    if (!desc || !out) return LISA_ERR_NULL;
    *out = nullptr;
    const lisa_data_desc& q = *desc;
    if (q.n_datasets < 1 || (q.n_channels != 2 && q.n_channels != 3) || q.sgwb_model < 0 ||
        q.sgwb_model > 2 || q.tdi_form < 0 || q.tdi_form > 1 || q.cov_model < 0 || q.cov_model > 1 ||
        (q.cov_model == LISA_COV_FULL && q.n_channels != 3))
        return LISA_ERR_VALUE;
    if (q.cov_model == LISA_COV_FULL && !q.periodogram_cross) return LISA_ERR_NULL;
    if (!q.bin_offset || !q.state_offset || !q.freq || !q.nu || !q.periodogram || !q.x_lo ||
        !q.x_hi || !q.f_ref || (q.sgwb_model != 0 && !q.response))
        return LISA_ERR_NULL;
    const int D = q.n_datasets;
    if (q.bin_offset[0] != 0 || q.state_offset[0] != 0) return LISA_ERR_SHAPE;
    for (int k = 0; k < D; ++k)
        if (q.bin_offset[k + 1] < q.bin_offset[k] || q.state_offset[k + 1] < q.state_offset[k])
            return LISA_ERR_SHAPE;
    const int64_t N = q.bin_offset[D], S = q.state_offset[D];
    if (N < 1 || S > (int64_t)INT32_MAX) return LISA_ERR_SHAPE;
    const int C = q.n_channels;
    // data validation on the host
    for (int k = 0; k < D; ++k) {
        if (!std::isfinite(q.x_lo[k]) || !std::isfinite(q.x_hi[k]) || !(q.x_lo[k] < q.x_hi[k]) ||
            !(q.f_ref[k] > 0.0) || !std::isfinite(q.f_ref[k]))
            return LISA_ERR_DATA;
        for (int64_t i = q.bin_offset[k]; i < q.bin_offset[k + 1]; ++i) {
            if (!(q.freq[i] > 0.0) || !std::isfinite(q.freq[i])) return LISA_ERR_DATA;
            if (i > q.bin_offset[k] && !(q.freq[i] > q.freq[i - 1])) return LISA_ERR_DATA;
        }
    }
    for (int64_t i = 0; i < N; ++i)
        if (!(q.nu[i] >= 0.0) || !std::isfinite(q.nu[i])) return LISA_ERR_DATA;
    for (int64_t i = 0; i < (int64_t)C * N; ++i) {
        if (!(q.periodogram[i] > 0.0) || !std::isfinite(q.periodogram[i])) return LISA_ERR_DATA;
        if (q.sgwb_model != 0 && (!(q.response[i] >= 0.0) || !std::isfinite(q.response[i])))
            return LISA_ERR_DATA;
    }
    if (q.cov_model == LISA_COV_FULL)
        for (int64_t i = 0; i < 3 * N; ++i)
            if (!std::isfinite(q.periodogram_cross[i])) return LISA_ERR_DATA;

    lisa_data* d = new (std::nothrow) lisa_data();
    if (!d) return LISA_ERR_ALLOC;
    cudaGetDevice(&d->device);
    cudaDeviceGetAttribute(&d->n_sm, cudaDevAttrMultiProcessorCount, d->device);
    d->n_datasets = D;
    d->C = C;
    d->sgwb_model = q.sgwb_model;
    d->tdi_form = q.tdi_form;
    d->cov = q.cov_model;
    d->nsp = C + (q.sgwb_model != 0 ? 1 : 0) + (q.cov_model == LISA_COV_FULL ? 3 : 0);
    d->n_bins = N;
    d->n_states = S;
    d->h_bin_off.assign(q.bin_offset, q.bin_offset + D + 1);
    for (int k = 0; k < D; ++k) {
        d->h_xs_off.push_back((int64_t)d->h_xs.size());
        const int64_t n = q.bin_offset[k + 1] - q.bin_offset[k];
        for (int64_t i = 0; i < n; i += kXsStride) d->h_xs.push_back(std::log10(q.freq[q.bin_offset[k] + i]));
        if (n > 0) d->h_xs.push_back(std::log10(q.freq[q.bin_offset[k] + n - 1]));
    }
    d->h_xs_off.push_back((int64_t)d->h_xs.size());
    d->h_state_off.assign(q.state_offset, q.state_offset + D + 1);
    d->h_ds.resize(D);
    std::vector<int32_t> state_ds((size_t)S);
    int64_t psd_base = 0, pad0 = 0;
    for (int k = 0; k < D; ++k) {
        DatasetDev& X = d->h_ds[k];
        X.rbin0 = q.bin_offset[k];
        X.nbins = q.bin_offset[k + 1] - q.bin_offset[k];
        X.npad = X.nbins + (X.nbins & 1);
        X.bin0 = pad0;
        pad0 += X.npad;
        X.s0 = (int32_t)q.state_offset[k];
        X.ns = (int32_t)(q.state_offset[k + 1] - q.state_offset[k]);
        X.x_lo = q.x_lo[k];
        X.x_hi = q.x_hi[k];
        X.xb_min = X.nbins ? std::log10(q.freq[X.rbin0]) : 0.0;
        X.xb_max = X.nbins ? std::log10(q.freq[X.rbin0 + X.nbins - 1]) : 0.0;
        X.f_ref = q.f_ref[k];
        X.ntiles = 0;
        X.pbase = 0;
        X.psd_base = psd_base;
        psd_base += (int64_t)C * X.ns * X.nbins;
        X.K = 0.0;
        X.Cnu = 0.0;
        X.nranges = (int32_t)((X.npad + kAdjBins - 1) / kAdjBins);
        for (int32_t s = X.s0; s < X.s0 + X.ns; ++s) state_ds[s] = k;
    }
    d->n_pad = pad0;
    d->tiling = lisa_tiling{512, 128, 4, 0};
    const int64_t NP = pad0 > 0 ? pad0 : 1;

    lisa_status st = LISA_SUCCESS;
    double *f = nullptr, *nu = nullptr, *R = nullptr, *lnP = nullptr, *nu_p = nullptr, *X = nullptr;
    auto fail = [&](lisa_status e) {
        cudaFree(X);
        cudaFree(f);
        cudaFree(nu);
        cudaFree(R);
        cudaFree(lnP);
        cudaFree(nu_p);
        release(d);
        delete d;
        return e;
    };
    if ((st = dev_alloc(&d->d_ds, D)) || (st = dev_alloc(&d->d_state_ds, (size_t)S)) ||
        (st = dev_alloc(&d->d_rec32, (size_t)NP * kRec)) || (st = dev_alloc(&d->d_rec64, (size_t)NP * kRec)) ||
        (st = dev_alloc(&d->d_P, (size_t)C * N)) || (st = dev_alloc(&d->d_xlo32, (size_t)NP)) ||
        (st = dev_alloc(&d->d_elllo32, (size_t)NP)) || (st = dev_alloc(&nu_p, (size_t)NP)) ||
        (st = dev_alloc(&f, (size_t)N)) ||
        (st = dev_alloc(&nu, (size_t)N)) || (st = dev_alloc(&lnP, (size_t)NP)) ||
        (st = dev_alloc(&R, (size_t)C * N)))
        return fail(st);
    cudaStream_t sm = (cudaStream_t)stream;
    bool ok = cudaMemcpyAsync(d->d_ds, d->h_ds.data(), D * sizeof(DatasetDev), cudaMemcpyHostToDevice, sm) == cudaSuccess &&
              cudaMemcpyAsync(d->d_state_ds, state_ds.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice, sm) == cudaSuccess &&
              cudaMemcpyAsync(f, q.freq, N * sizeof(double), cudaMemcpyHostToDevice, sm) == cudaSuccess &&
              cudaMemcpyAsync(nu, q.nu, N * sizeof(double), cudaMemcpyHostToDevice, sm) == cudaSuccess &&
              cudaMemcpyAsync(d->d_P, q.periodogram, C * N * sizeof(double), cudaMemcpyHostToDevice, sm) == cudaSuccess &&
              (q.sgwb_model == 0 || cudaMemcpyAsync(R, q.response, C * N * sizeof(double), cudaMemcpyHostToDevice, sm) == cudaSuccess);
    if (!ok) return fail(LISA_ERR_CUDA);
    unsigned blocks = (unsigned)((NP + 255) / 256);
    prep_kernel<<<blocks, 256, 0, sm>>>(pad0, C, q.tdi_form, q.sgwb_model != 0, f, nu, d->d_P, R, N, d->d_ds, D,
                                        d->d_rec64, d->d_rec32, d->d_xlo32, d->d_elllo32, lnP, nu_p);
    dataset_sums_kernel<<<D, 256, 0, sm>>>(lnP, nu_p, d->d_ds, C);
    if (cudaGetLastError() != cudaSuccess) return fail(LISA_ERR_CUDA);
    if (d->cov == LISA_COV_FULL) {
        if ((st = dev_alloc(&X, (size_t)3 * N)) || (st = dev_alloc(&d->d_cross64, (size_t)NP * kCross)) ||
            (st = dev_alloc(&d->d_cross32, (size_t)((NP + 1) / 2) * kPairCross)))
            return fail(st);
        if (cudaMemcpyAsync(X, q.periodogram_cross, 3 * N * sizeof(double), cudaMemcpyHostToDevice, sm) != cudaSuccess)
            return fail(LISA_ERR_CUDA);
        cross_prep_kernel<<<blocks, 256, 0, sm>>>(pad0, d->d_P, X, N, d->d_ds, D, d->d_cross64, d->d_cross32);
        if (cudaGetLastError() != cudaSuccess) return fail(LISA_ERR_CUDA);
    }
    if (cudaMemcpyAsync(d->h_ds.data(), d->d_ds, D * sizeof(DatasetDev), cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
        cudaStreamSynchronize(sm) != cudaSuccess)
        return fail(LISA_ERR_CUDA);
    cudaFree(f);
    cudaFree(nu);
    cudaFree(R);
    cudaFree(lnP);
    cudaFree(nu_p);
    cudaFree(X);
    f = nu = R = lnP = nu_p = X = nullptr;
    if ((st = rebuild_work(d))) return fail(st);
    {
        // adjoint decomposition (independent of the tiling): per dataset, ranges x groups of 32
        std::vector<AdjUnit> units;
        std::vector<int64_t> prefix((size_t)S);
        int64_t acc = 0;
        for (int k = 0; k < D; ++k) {
            const DatasetDev& X = d->h_ds[k];
            for (int32_t s2 = 0; s2 < X.ns; ++s2) {
                prefix[(size_t)X.s0 + s2] = acc;
                acc += X.nranges;
            }
            for (int32_t r = 0; r < X.nranges; ++r)
                for (int32_t g = 0; g < X.ns; g += 32) units.push_back(AdjUnit{k, r, X.s0 + g, std::min(32, X.ns - g)});
        }
        d->adj_ranges = acc;
        d->n_adj_units = (int64_t)units.size();
        if ((st = dev_alloc(&d->d_adj_units, units.size())) || (st = dev_alloc(&d->d_adj_prefix, prefix.size())))
            return fail(st);
        if (cudaMemcpy(d->d_adj_units, units.data(), units.size() * sizeof(AdjUnit), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(d->d_adj_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return fail(LISA_ERR_CUDA);
    }
    *out = d;
    return LISA_SUCCESS;
}

lisa_status lisa_data_destroy(lisa_data* d) {
    if (!d) return LISA_ERR_NULL;
    release(d);
    delete d;
    return LISA_SUCCESS;
}

lisa_status lisa_data_set_profiling(lisa_data* d, int32_t enable) {
    if (!d) return LISA_ERR_NULL;
    if (enable && !d->prof_on) {
        for (auto& e : d->prof_ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) return LISA_ERR_CUDA;
    }
    d->prof_on = enable != 0;
    d->prof_valid = false;
    return LISA_SUCCESS;
}

lisa_status lisa_data_set_test_wait(lisa_data* d, int32_t skip_copies, uint32_t wait_limit) {
    if (!d) return LISA_ERR_NULL;
    if (wait_limit < 1) return LISA_ERR_VALUE;
    d->test_skip_copies = skip_copies != 0;
    d->wait_limit = wait_limit;
    return LISA_SUCCESS;
}

lisa_status lisa_data_get_info(const lisa_data* d, lisa_data_info* info) {
    if (!d || !info) return LISA_ERR_NULL;
    info->n_bins = d->n_bins;
    info->n_states = d->n_states;
    info->n_datasets = d->n_datasets;
    info->n_channels = d->C;
    info->n_splines = d->nsp;
    info->sgwb_model = d->sgwb_model;
    info->n_items = d->n_items;
    info->n_sm = d->n_sm;
    info->tiling = d->tiling;
    return LISA_SUCCESS;
}

lisa_status lisa_data_set_tiling(lisa_data* d, const lisa_tiling* t) {
    if (!d || !t) return LISA_ERR_NULL;
    int sc = t->states_per_cta;
    bool pow2 = sc > 0 && (sc & (sc - 1)) == 0;
    if (t->tile_bins < 64 || t->tile_bins > kMaxTileBins || (t->tile_bins % 32) != 0 || !pow2 || sc < 16 ||
        sc > kMaxStatesPerItem || !(t->group == 2 || t->group == 4 || t->group == 8) ||
        t->ctas_per_sm < 0 || t->ctas_per_sm > 32 || (d->cov == LISA_COV_FULL && t->tile_bins > kMaxTileBinsFull))
        return LISA_ERR_VALUE;
    lisa_tiling old = d->tiling;
    d->tiling = *t;
    lisa_status st = rebuild_work(d);
    if (st) {
        d->tiling = old;
        rebuild_work(d);
    }
    return st;
}

size_t lisa_spline_buf_bytes(const lisa_data* d, int32_t kmax, lisa_precision p) {
    if (!d || kmax < 0 || kmax > LISA_MAX_KNOTS) return 0;
    (void)p;
    return spline_layout(d->n_states, d->nsp, kmax).bytes;
}

}  // extern "C"

LISA_DEBUG_TU(data)
