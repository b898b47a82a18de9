/*
 * gvom_microbench.h -- throughput probes used as roofline denominators for
 * the map update kernels. The paper has no counterpart; these measure the
 * GPU, not the method.
 */
#ifndef GVOM_MICROBENCH_H
#define GVOM_MICROBENCH_H

#include <stdint.h>

#include "gvom.h"

#ifdef __cplusplus
extern "C" {
#endif

/* L2 atomic throughput probe: `ops` 32-bit atomic adds whose results are
 * unused (reductions), to pseudo-random, mostly distinct words of the
 * caller's device buffer buf_dev[words] (words >= 1024). The access pattern
 * matches the pass counting of gvom_ingest_scan: scattered single-word
 * updates over a buffer of map size. buf_dev's contents change. Returns
 * GVOM_ERR_INVALID_ARG for a null buffer or sizes out of range.
 * Stream-ordered; time it with events on `stream`. */
GVOM_API int gvom_microbench_red(uint32_t* buf_dev, int64_t words, int64_t ops, uint32_t seed,
                                 gvom_stream_t stream);

/* The same probe in its best case for the L2: every warp instruction adds 1
 * to 32 consecutive words (one 128-byte line) at a pseudo-random line of
 * the buffer (words >= 1024; ops = increments, >= 32, a multiple of 32
 * used). The ceiling for pass increments that neighbouring lanes merge or
 * place on one line. Stream-ordered. */
GVOM_API int gvom_microbench_red_coalesced(uint32_t* buf_dev, int64_t words, int64_t ops, uint32_t seed,
                                           gvom_stream_t stream);

/* Measurement hook: with a CUDA event (cudaEvent_t, passed as a pointer)
 * set, every later ingest of this map (gvom_ingest_scan, gvom_update,
 * gvom_update_extract) records that event on its stream after the
 * per-point pass and before the segment walk, so that the caller can time
 * the walk by itself with events on the same stream. NULL turns it off.
 * While it is set the walk's launch no longer overlaps the per-point
 * pass's tail. Host-only. */
GVOM_API int gvom_set_walk_marker(struct gvom_map* map, void* cuda_event);

/* Number of kernels this library has launched since it was loaded (all
 * maps, all entry points; a replay of a captured batch step counts the
 * kernels the graph holds). Host-only; instrumentation for benchmarks. */
GVOM_API int64_t gvom_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GVOM_MICROBENCH_H */
