// Self-tests of the library's failure detection (include/gvom_selftest.h).
// The paper has no counterpart. Each one makes a safeguard fire on purpose
// without any fault: a barrier wait that nothing completes gives up after
// its iteration limit, and an index one past the map is caught by the
// checked build's range check before any access. Both record their status
// in the map's status word, which gvom_get_stats reports.
#include "gvom_internal.h"
#include "device_sync.cuh"
#include "exact_convert.cuh"
#include "../../include/gvom_selftest.h"

namespace gvom {
namespace {

// One thread initialises a barrier that expects one arrival, makes none,
// and waits for it with the library's bounded wait.
__global__ void k_wait_selftest(unsigned long long* counters, unsigned limit) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, limit)) atomicOr(counters + kStatus, kStatusTimeout);
}

// The index V (one past the last voxel) through the range check; the
// access it guards is never made.
__global__ void k_bounds_selftest(MapState s) {
    if (threadIdx.x != 0) return;
    const unsigned long long k = s.V;
    if (in_bounds(k, s.V, s.counters)) s.hits[k] = 0u;  // not reached in a checked build
}

// Each input bit pattern taken as a double d and (its low word) as a float
// f: the library's integer-pipe conversions against CUDA's own, counting
// mismatches (the integer conversion only where it is used, |d| < 2^30).
__global__ void k_conversion_selftest(const unsigned long long* __restrict__ bits, long long n,
                                      unsigned long long* __restrict__ mismatches) {
    unsigned long long bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = __longlong_as_double((long long)bits[i]);
        const float f = __uint_as_float((uint32_t)bits[i]);
        if (!isnan(d)) {
            if (fabs(d) < 1073741824.0 && d2i_rne(d) != (int)__double2ll_rn(d)) bad += 1;
            if (__float_as_uint(d2f_rne(d)) != __float_as_uint(__double2float_rn(d))) bad += 1;
        }
        if (!isnan(f) &&
            __double_as_longlong(f2d_exact(f)) != __double_as_longlong((double)f))
            bad += 1;
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace
}  // namespace gvom

extern "C" {

int gvom_selftest_conversions(const uint64_t* bits_dev, int64_t n, uint64_t* mismatches_dev, gvom_stream_t stream) {
    if (!bits_dev || !mismatches_dev || n < 0) return GVOM_ERR_INVALID_ARG;
    if (n == 0) return GVOM_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    gvom::count_launch();
    gvom::k_conversion_selftest<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        (const unsigned long long*)bits_dev, n, (unsigned long long*)mismatches_dev);
    return gvom::cuda_status(cudaGetLastError());
}

int gvom_checked_build(void) {
#ifdef GVOM_CHECKED
    return 1;
#else
    return 0;
#endif
}

int gvom_selftest_wait_timeout(struct gvom_map* map, uint32_t spin_limit, gvom_stream_t stream) {
    if (!map || spin_limit < 1u || spin_limit > (1u << 24)) return GVOM_ERR_INVALID_ARG;
    gvom::count_launch();
    gvom::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(map->s.counters, spin_limit);
    return gvom::cuda_status(cudaGetLastError());
}

int gvom_selftest_bounds(struct gvom_map* map, gvom_stream_t stream) {
    if (!map) return GVOM_ERR_INVALID_ARG;
#ifdef GVOM_CHECKED
    gvom::count_launch();
    gvom::k_bounds_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(map->s);
    return gvom::cuda_status(cudaGetLastError());
#else
    (void)stream;
    return GVOM_ERR_INVALID_ARG;  // without the range checks the access would be real: nothing is launched
#endif
}

}  // extern "C"
