// Roofline probes (include/gvom_microbench.h): L2 reduction-atomic
// throughput on scattered words, the pattern of the pass counts.
#include "gvom_internal.h"
#include "../../include/gvom_microbench.h"

namespace {

// pow2 is the largest power of two <= words; indexes fold [pow2, 2 pow2)
// down by pow2, so every index stays below words.
__global__ void k_red_probe(uint32_t* __restrict__ buf, uint32_t pow2, long long words, long long ops,
                            uint32_t seed) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x = (uint32_t)tid * 0x9E3779B9u ^ seed;
    for (long long i = tid; i < ops; i += nthreads) {
        // xorshift32 stream per thread
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        uint32_t w = x & (2u * pow2 - 1u);
        if (w >= (uint32_t)words) w -= pow2;
        atomicAdd(buf + w, 1u);
    }
}

// Coalesced form: each warp step adds 1 to 32 consecutive words (one
// 128-byte line) at a pseudo-random 32-word-aligned place, the best case of
// a warp's reduction atomics. ops counts the increments (32 per warp step).
__global__ void k_red_probe_coalesced(uint32_t* __restrict__ buf, uint32_t lines_pow2, long long lines,
                                      long long ops, uint32_t seed) {
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    uint32_t x = (uint32_t)gw * 0x9E3779B9u ^ seed;
    for (long long i = gw; i < (ops >> 5); i += nwarps) {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        uint32_t l = x & (2u * lines_pow2 - 1u);
        if (l >= (uint32_t)lines) l -= lines_pow2;
        atomicAdd(buf + (size_t)l * 32 + lane, 1u);
    }
}

int probe_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (sms > 0 ? sms : 1) * 8;
}

}  // namespace

extern "C" int gvom_microbench_red(uint32_t* buf_dev, int64_t words, int64_t ops, uint32_t seed,
                                   gvom_stream_t stream) {
    if (!buf_dev || words < 1024 || words > (1LL << 31) || ops < 1 || ops > (1LL << 40)) return GVOM_ERR_INVALID_ARG;
    uint32_t pow2 = 1;
    while ((long long)pow2 * 2 <= words) pow2 *= 2;
    gvom::count_launch();
    k_red_probe<<<probe_blocks(), 256, 0, (cudaStream_t)stream>>>(buf_dev, pow2, words, ops, seed);
    return cudaGetLastError() == cudaSuccess ? GVOM_OK : GVOM_ERR_CUDA;
}

extern "C" int gvom_microbench_red_coalesced(uint32_t* buf_dev, int64_t words, int64_t ops, uint32_t seed,
                                             gvom_stream_t stream) {
    if (!buf_dev || words < 1024 || words > (1LL << 31) || ops < 32 || ops > (1LL << 40)) return GVOM_ERR_INVALID_ARG;
    const long long lines = words / 32;
    uint32_t pow2 = 1;
    while ((long long)pow2 * 2 <= lines) pow2 *= 2;
    gvom::count_launch();
    k_red_probe_coalesced<<<probe_blocks(), 256, 0, (cudaStream_t)stream>>>(buf_dev, pow2, lines, ops, seed);
    return cudaGetLastError() == cudaSuccess ? GVOM_OK : GVOM_ERR_CUDA;
}
