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

/* Number of kernels this library has launched since it was loaded (all
 * maps, all entry points; a replay of a captured batch step counts the
 * kernels the graph holds). Host-only; instrumentation for benchmarks. */
GVOM_API int64_t gvom_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GVOM_MICROBENCH_H */
