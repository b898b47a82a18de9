/*
 * gvom_selftest.h -- self-tests of the library's failure detection. The
 * paper has no counterpart. They let a caller (and the test suite) see the
 * safeguards fire without any fault: the map's data is not touched, the
 * outcome is the status that gvom_get_stats returns, and gvom_reset_stats
 * clears it, after which the map is used as before.
 */
#ifndef GVOM_SELFTEST_H
#define GVOM_SELFTEST_H

#include <stdint.h>

#include "gvom.h"

#ifdef __cplusplus
extern "C" {
#endif

/* 1 if this library was built with GVOM_CHECKED (every computed index into
 * a map's state, scratch or outputs is range-checked in the kernels; an
 * index out of range skips its access and makes gvom_get_stats return
 * GVOM_ERR_BOUNDS), else 0. Host-only. */
GVOM_API int gvom_checked_build(void);

/* Launches one kernel that waits, with the library's bounded barrier wait
 * (the one the column pass uses for its bulk copies), on a barrier that
 * nothing completes. After spin_limit polls the wait gives up and records a
 * timeout in the map's status word: gvom_get_stats then returns
 * GVOM_ERR_TIMEOUT. 1 <= spin_limit <= 2^24, else GVOM_ERR_INVALID_ARG.
 * Stream-ordered. */
GVOM_API int gvom_selftest_wait_timeout(struct gvom_map* map, uint32_t spin_limit, gvom_stream_t stream);

/* Checked builds: launches one kernel that sends the index one past the
 * map's last voxel through the range check; the check records it and the
 * access is skipped, so gvom_get_stats then returns GVOM_ERR_BOUNDS.
 * Other builds have no range checks, so nothing is launched and the call
 * returns GVOM_ERR_INVALID_ARG. Stream-ordered. */
GVOM_API int gvom_selftest_bounds(struct gvom_map* map, gvom_stream_t stream);

/* Checks the per-point pass's integer-pipe conversions (float -> double,
 * double -> int and double -> float, round to nearest, ties to even)
 * against CUDA's own on the GPU: each of the n 64-bit patterns at bits_dev
 * is taken as a double and its low word as a float; every disagreement adds
 * 1 to *mismatches_dev (device uint64, the caller zeroes it). NaN inputs
 * are skipped; the double -> int conversion is checked where the library
 * uses it, |d| < 2^30. Stream-ordered. */
GVOM_API int gvom_selftest_conversions(const uint64_t* bits_dev, int64_t n, uint64_t* mismatches_dev,
                                       gvom_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GVOM_SELFTEST_H */
