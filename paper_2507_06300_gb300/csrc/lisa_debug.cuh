// Index checks of the debug build.
//
// LISA_IDX(i, n) wraps a tile, bin, interval (knot), record, moment-slot or list index i that
// must lie in [0, n).  A release build compiles it to i.  A build with -DLISA_DEBUG_BOUNDS checks
// it: an index outside [0, n) is counted, the first one seen (its value and source line) is
// recorded in this translation unit's record, and the access goes to the clamped index (0 or
// n - 1), so that the check itself never reads or writes outside the buffer.  The records are read
// (and reset) through lisa_debug_bounds (include/lisa_debug.h); nothing traps.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lisa {
namespace dbg {

// One translation unit's record: violations counted, and the first one's index and line.
struct BoundsRecord {
    unsigned long long count;
    long long first_index;
    int first_line;
    int pad;
};

namespace {
__device__ BoundsRecord g_bounds;   // internal linkage: one record per translation unit

#ifdef LISA_DEBUG_BOUNDS
__device__ __noinline__ long long bounds_fail(long long i, long long n, int line) {
    const unsigned long long c = atomicAdd(&g_bounds.count, 1ull);
    if (c == 0) {
        g_bounds.first_index = i;
        g_bounds.first_line = line;
    }
    return (i < 0 || n <= 0) ? 0 : n - 1;
}
#endif

// The record of this translation unit (host; synchronises the device first), reset to zero when
// reset != 0.
[[maybe_unused]] cudaError_t read_record(BoundsRecord* out, int reset) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_bounds, sizeof(BoundsRecord));
    if (e == cudaSuccess && reset) {
        const BoundsRecord z = {0ull, 0ll, 0, 0};
        e = cudaMemcpyToSymbol(g_bounds, &z, sizeof(BoundsRecord));
    }
    return e;
}
}  // namespace

#ifdef LISA_DEBUG_BOUNDS
template <class I>
__device__ __forceinline__ I checked_index(I i, long long n, int line) {
    const long long v = (long long)i;
    return (v >= 0 && v < n) ? i : (I)bounds_fail(v, n, line);
}
#define LISA_IDX(i, n) ::lisa::dbg::checked_index((i), (long long)(n), __LINE__)
constexpr bool kBoundsChecked = true;
#else
#define LISA_IDX(i, n) (i)
constexpr bool kBoundsChecked = false;
#endif

// Each translation unit exports its record reader under its own name (lisa_debug_bounds gathers
// them); the file name identifies the unit in the report.
#define LISA_DEBUG_TU(name)                                                                    \
    namespace lisa {                                                                           \
    namespace dbg {                                                                            \
    cudaError_t read_##name(BoundsRecord* out, int reset, const char** file) {                 \
        *file = __FILE__;                                                                      \
        return read_record(out, reset);                                                        \
    }                                                                                          \
    }                                                                                          \
    }

}  // namespace dbg
}  // namespace lisa
