/*
 * lisa_debug.h -- the bounds-checked debug build of the library.  Not part of the method: the
 * paper has no counterpart; this is test infrastructure that stands in for a memory checker.
 *
 * The library's kernels wrap their tile, bin, interval (knot), record, moment-slot and list
 * indices in a check that a release build compiles away.  A build with -DLISA_DEBUG_BOUNDS
 * (lib/liblisa_psd_debug.so, built on demand by the package's build module) evaluates it: an
 * index outside its range is counted, the first one (its value, the source file and line) is
 * recorded, and the access goes to the nearest valid index instead, so the check never touches
 * memory outside a buffer and nothing traps.  Every other entry point behaves as in the release
 * build.
 */
#ifndef LISA_DEBUG_H
#define LISA_DEBUG_H

#include "lisa_psd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Index violations seen since the last reset, over all of the library's kernels. */
typedef struct lisa_bounds_report {
    int64_t count;        /* violations counted (0 when none; 0 in a release build) */
    int64_t first_index;  /* the first recorded violation's index (of the first source file
                             in build order that has one) */
    int32_t first_line;   /* its source line */
    char first_file[96];  /* its source file (path as compiled, truncated), "" when count == 0 */
} lisa_bounds_report;

/* 1 when the index checks are compiled in (the debug build), 0 in a release build. */
int32_t lisa_debug_bounds_enabled(void);

/* Waits for the device to finish all work (cudaDeviceSynchronize), then writes the report to
 * `out` (HOST, caller-owned) and, when reset != 0, clears the records.  A release build reports
 * count 0.  Errors: LISA_ERR_NULL (out), LISA_ERR_CUDA. */
lisa_status lisa_debug_bounds(int32_t reset, lisa_bounds_report* out);

/* Debug build only: launches one warp on `stream` whose 32 threads each store to a 4-float device
 * buffer the library allocates and frees, at the checked index 5 + lane (always out of range,
 * clamped to 3 by the check), then synchronises the stream.  Afterwards lisa_debug_bounds reports
 * 32 more violations.  It exists to show that the checks fire.  A release build launches nothing
 * and returns LISA_ERR_VALUE.  Errors: LISA_ERR_ALLOC, LISA_ERR_CUDA. */
lisa_status lisa_debug_bounds_selftest(lisa_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LISA_DEBUG_H */
