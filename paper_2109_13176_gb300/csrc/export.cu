// Export of a map in the paper's storage format (G-VOM Sec. III-A): a
// lookup table over the window and a data array of the occupied voxels.
//
// The table holds, for each voxel in logical linear order, the voxel's index
// in the data array if it is occupied (hits >= 1) and -1 - N_m otherwise
// (N_m = its misses, the pass count); the data array holds the occupied
// voxels' hits, misses and lowest return in that same order. The order is
// deterministic: three kernels count occupied voxels per 1024-voxel block,
// scan the block counts, then write each block's voxels at their global
// ranks.
#include "gvom_internal.h"

namespace gvom {

namespace {

constexpr int kLutBlock = 256;
constexpr int kLutPer = 4;                      // consecutive voxels per thread
constexpr int kLutSpan = kLutBlock * kLutPer;   // voxels per block

// Physical slots of the kLutPer consecutive logical voxels from i (those
// past V are not used). When nz is a multiple of kLutPer the run lies in one
// column, whose base takes one division.
__device__ __forceinline__ void logical_to_phys(const Geom& g, uint32_t i, uint32_t (&k)[kLutPer]) {
    const bool one_column = (g.nz % kLutPer) == 0;
#pragma unroll
    for (int j = 0; j < kLutPer; ++j) {
        if (j > 0 && one_column) {
            int pz = (int)(k[0] % (uint32_t)g.nz) + j;  // k[0] = base + pz0
            k[j] = k[0] + j - (pz >= g.nz ? (uint32_t)g.nz : 0u);
            continue;
        }
        const uint32_t ij = i + (uint32_t)j;  // i < V < 2^31
        const uint32_t cz = ij % (uint32_t)g.nz;
        const uint32_t col = ij / (uint32_t)g.nz;
        const uint32_t cy = col % (uint32_t)g.ny, cx = col / (uint32_t)g.ny;
        int px = (int)cx + g.rx;
        px -= (px >= g.nx) ? g.nx : 0;
        int py = (int)cy + g.ry;
        py -= (py >= g.ny) ? g.ny : 0;
        int pz = (int)cz + g.rz;
        pz -= (pz >= g.nz) ? g.nz : 0;
        k[j] = ((uint32_t)px * g.ny + py) * (uint32_t)g.nz + pz;
    }
}

// Exclusive block-wide scan of one value per thread (kLutBlock threads).
__device__ __forceinline__ unsigned int block_exclusive(unsigned int v, unsigned int* warp_sums, unsigned int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int s = 0;
        for (int w = 0; w < kLutBlock / 32; ++w) {
            const unsigned int t = warp_sums[w];
            warp_sums[w] = s;
            s += t;
        }
        *total = s;
    }
    __syncthreads();
    return warp_sums[warp] + x - v;
}

__global__ void __launch_bounds__(kLutBlock) k_lut_count(MapState s, Geom g, long long V, unsigned int* counts) {
    __shared__ unsigned int warp_sums[kLutBlock / 32];
    const long long i0 = (long long)blockIdx.x * kLutSpan + (long long)threadIdx.x * kLutPer;
    unsigned int c = 0;
    if (i0 < V) {
        uint32_t k_[kLutPer];
        logical_to_phys(g, (uint32_t)i0, k_);
#pragma unroll
        for (int k = 0; k < kLutPer; ++k)
            if (i0 + k < V && in_bounds(k_[k], s.V, s.counters)) c += s.hits[k_[k]] != 0u ? 1u : 0u;
    }
    // the block's total only (a reduction, not a scan)
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned int t = threadIdx.x < kLutBlock / 32 ? warp_sums[threadIdx.x] : 0u;
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) counts[blockIdx.x] = t;
    }
}

// One block scans all block counts in place (exclusive) and writes the
// total: 4,096 counts per pass, four per thread (prefixes fit 32 bits, V < 2^31).
__global__ void __launch_bounds__(1024) k_lut_scan(unsigned int* counts, long long nblocks, long long* n_occupied) {
    __shared__ unsigned int warp_sums[32];
    __shared__ unsigned int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nblocks; base += 4096) {
        const long long i = base + 4 * (long long)threadIdx.x;
        unsigned int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i + k < nblocks ? counts[i + k] : 0u;
        const unsigned int t = v[0] + v[1] + v[2] + v[3];
        unsigned int x = t;  // inclusive scan of the thread totals within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int sum = 0;
            for (int w = 0; w < 32; ++w) {
                const unsigned int u = warp_sums[w];
                warp_sums[w] = sum;
                sum += u;
            }
        }
        __syncthreads();
        unsigned int excl = carry + warp_sums[warp] + x - t;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i + k < nblocks) counts[i + k] = excl;
            excl += v[k];
        }
        __syncthreads();                             // every thread has read carry
        if (threadIdx.x == 1023) carry = excl;       // the pass's end
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_occupied = (long long)carry;
}

__global__ void __launch_bounds__(kLutBlock)
    k_lut_write(MapState s, Geom g, long long V, const unsigned int* prefix, long long* lut, uint32_t* d_hits,
                uint32_t* d_passes, float* d_minz, long long cap) {
    __shared__ unsigned int warp_sums[kLutBlock / 32];
    __shared__ unsigned int total;
    const long long i0 = (long long)blockIdx.x * kLutSpan + (long long)threadIdx.x * kLutPer;
    uint32_t k_[kLutPer];
    uint32_t h_[kLutPer], p_[kLutPer];
    float m_[kLutPer];
    unsigned int c = 0;
    if (i0 < V) logical_to_phys(g, (uint32_t)i0, k_);
    // every load before the block scan, so they are in flight together
#pragma unroll
    for (int k = 0; k < kLutPer; ++k) {
        h_[k] = 0;
        p_[k] = 0;
        m_[k] = 0.0f;
        if (i0 + k < V && in_bounds(k_[k], s.V, s.counters)) {
            h_[k] = s.hits[k_[k]];
            p_[k] = s.passes[k_[k]];
            m_[k] = s.minz[k_[k]];
        }
    }
#pragma unroll
    for (int k = 0; k < kLutPer; ++k) c += h_[k] != 0u ? 1u : 0u;
    long long idx = (long long)prefix[blockIdx.x] + block_exclusive(c, warp_sums, &total);
#pragma unroll
    for (int k = 0; k < kLutPer; ++k) {
        if (i0 + k >= V) break;
        if (h_[k] != 0u) {
            lut[i0 + k] = idx;
            if (idx < cap) {
                d_hits[idx] = h_[k];
                d_passes[idx] = p_[k];
                d_minz[idx] = m_[k];
            }
            idx += 1;
        } else {
            lut[i0 + k] = -1 - (long long)p_[k];
        }
    }
}

}  // namespace

long long lut_blocks(long long V) { return (V + kLutSpan - 1) / kLutSpan; }

cudaError_t launch_export_lut(const MapState& s, const Geom& g, unsigned int* counts, long long* n_occupied,
                              long long* lut, uint32_t* dh, uint32_t* dp, float* dm, long long cap, cudaStream_t st) {
    const long long V = (long long)g.nx * g.ny * g.nz;
    const long long nb = lut_blocks(V);
    count_launch();
    k_lut_count<<<(unsigned)nb, kLutBlock, 0, st>>>(s, g, V, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_lut_scan<<<1, 1024, 0, st>>>(counts, nb, n_occupied);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    k_lut_write<<<(unsigned)nb, kLutBlock, 0, st>>>(s, g, V, counts, lut, dh, dp, dm, cap);
    return cudaGetLastError();
}

}  // namespace gvom
