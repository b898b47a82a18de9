// 2D products of the voxel map (G-VOM Sec. III-D) for sm_103a.
//
// k_columns: the column pass. A map column is three contiguous runs of nz
// words (hits, passes, lowest returns; z is the fastest axis), so a group
// of lanes streams each run with 16-byte loads and reduces it with
// shuffles into the height, the positive obstacle band sums, density and
// hard/soft flags. Bandwidth-bound: 12 bytes read per voxel.
// k_slope_negative: the pixel pass, one 16 x 16 tile of the height map per
// block, staged in shared memory with a halo. Defined pixels get the N x N
// least-squares plane (slope, roughness). Undefined pixels get the four-cone
// negative obstacle search, computed for the whole tile at once by a sweep
// per cone direction: the cone of a pixel at ring d is the union of the
// cones of its three forward neighbours at ring d - 1, so each pixel's
// first ring holding ground, and the lowest height on it, follow from the
// neighbours' in O(1).
#include <math.h>

#include "gvom_internal.h"
#include "device_sync.cuh"

namespace gvom {

namespace {

constexpr int kColBlock = 256;

// density = (float)((double)H / (double)(H + M)), the oracle's FP64
// division rounded to float. When H + M < 2^24 both operands are exact
// floats and the quotient's distance to any float rounding midpoint is at
// least 2^-24 of a float ulp, far above the FP64 rounding error, so the
// correctly rounded FP32 division gives the same float; otherwise FP64.
__device__ __forceinline__ float density_of(unsigned long long H, unsigned long long D) {
    if (D < (1ull << 24)) return __fdiv_rn((float)(unsigned int)H, (float)(unsigned int)D);
    return __double2float_rn(__ddiv_rn((double)H, (double)D));
}

// The oracle's test lo <= (double)a - (double)b <= hi for floats a, b and
// float bounds. The FP32 difference decides unless it lies within a
// relative 2^-20 of a bound (where FP32 and FP64 rounding could disagree);
// there the FP64 difference decides. Band holds the four edges of those
// ambiguous zones, computed once.
struct Band {
    float lo, hi;                    // the band
    float lo_m, lo_p, hi_m, hi_p;    // lo -+ tl, hi -+ th
};

__device__ __forceinline__ Band make_band(float lo, float hi) {
    const float tl = fabsf(lo) * 9.5367432e-7f + 1e-30f;
    const float th = fabsf(hi) * 9.5367432e-7f + 1e-30f;
    return Band{lo, hi, lo - tl, lo + tl, hi - th, hi + th};
}

__device__ __forceinline__ bool in_band(float a, float b, const Band& B) {
    const float d = __fsub_rn(a, b);
    if (d < B.lo_m || d > B.hi_p) return false;   // clearly outside
    if (d > B.lo_p && d < B.hi_m) return true;    // clearly inside
    const double e = __dsub_rn((double)a, (double)b);
    return (double)B.lo <= e && e <= (double)B.hi;
}

__device__ __forceinline__ bool in_band(float a, float b, float lo, float hi) { return in_band(a, b, make_band(lo, hi)); }

// The oracle's test (double)hi - (double)lo > thresh, filtered the same way.
__device__ __forceinline__ bool exceeds(float hi, float lo, float thresh) {
    const float d = __fsub_rn(hi, lo);
    if (fabsf(d - thresh) <= fabsf(thresh) * 9.5367432e-7f + 1e-30f)
        return __dsub_rn((double)hi, (double)lo) > (double)thresh;
    return d > thresh;
}

// Scalar column pass for any nz: one warp per column.
__device__ __forceinline__ void column_scalar(const MapState& s, const ExtractParams& p, float* __restrict__ height,
                                              float* __restrict__ density, uint8_t* __restrict__ flags,
                                              long long col) {
    const Geom g = p.g;
    const int lane = threadIdx.x & 31;
    const int cx = (int)((unsigned)col / (unsigned)g.ny), cy = (int)((unsigned)col % (unsigned)g.ny);
    int px = cx + g.rx;
    px -= (px >= g.nx) ? g.nx : 0;
    int py = cy + g.ry;
    py -= (py >= g.ny) ? g.ny : 0;
    const size_t base = ((size_t)px * g.ny + py) * (size_t)g.nz;
    if (!in_bounds(base + g.nz - 1, s.V, s.counters)) return;  // the whole warp (one column)
    const uint32_t* __restrict__ hc = s.hits + base;
    const uint32_t* __restrict__ pc = s.passes + base;
    const float* __restrict__ mc = s.minz + base;

    // Height: the lowest return of the column's occupied voxels (the voxel
    // order along z does not matter for a minimum).
    float h = __int_as_float(0x7f800000);
    bool any = false;
    for (int z = lane; z < g.nz; z += 32) {
        if (hc[z] != 0u) {
            h = fminf(h, mc[z]);
            any = true;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h = fminf(h, __shfl_xor_sync(0xffffffffu, h, o));
    any = __any_sync(0xffffffffu, any);

    unsigned long long H = 0, M = 0;
    if (any) {
        for (int z = lane; z < g.nz; z += 32) {
            const uint32_t nh = hc[z];
            if (nh == 0u) continue;
            if (in_band(mc[z], h, p.obs_min_h, p.obs_max_h)) {
                H += nh;
                M += pc[z];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            H += __shfl_xor_sync(0xffffffffu, H, o);
            M += __shfl_xor_sync(0xffffffffu, M, o);
        }
    }
    if (lane == 0 && in_bounds((size_t)cx * g.ny + cy, (unsigned long long)g.nx * g.ny, s.counters)) {
        const size_t o = (size_t)cx * g.ny + cy;
        if (height) height[o] = any ? h : __int_as_float(0x7fffffff);
        uint8_t f = 0;
        float dens = 0.0f;
        if (H > 0) {
            dens = density_of(H, H + M);
            const bool hard = H * (unsigned long long)p.hard_den >= (unsigned long long)p.hard_num * (H + M);
            f = hard ? 3 : 5;
        }
        if (density) density[o] = dens;
        if (flags) flags[o] = f;
    }
}

// Vector column pass for nz % 4 == 0: LPC lanes per column, each lane
// loading 16 bytes (4 voxels) per run and step, a grid-stride loop over
// column groups.
__global__ void __launch_bounds__(kColBlock) k_columns_scalar(MapState s, ExtractParams p, float* __restrict__ height,
                                                               float* __restrict__ density,
                                                               uint8_t* __restrict__ flags) {
    pdl_wait();
    const long long col = ((long long)blockIdx.x * kColBlock + threadIdx.x) >> 5;
    if (col >= (long long)p.g.nx * p.g.ny) return;
    column_scalar(s, p, height, density, flags, col);
    pdl_done();
}

// One step of the vector column pass for one warp: lane group lane / LPC
// takes column colb + lane / LPC (if below col_end); each lane loads 16
// bytes (4 voxels) per run and step.
template <int LPC>
__device__ __forceinline__ void columns_step(const MapState& s, const ExtractParams& p, float* __restrict__ height,
                                             float* __restrict__ density, uint8_t* __restrict__ flags,
                                             long long colb, long long col_end) {
    const Geom g = p.g;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPC;                  // lane within the column group
    const unsigned gmask = (LPC == 32) ? 0xffffffffu : (((1u << LPC) - 1u) << (lane - sub));
    const int nv = g.nz >> 2;  // 16-byte vectors per run
    const Band band = make_band(p.obs_min_h, p.obs_max_h);
    const long long col = colb + (lane / LPC);
    const bool have = col < col_end;
    int cx = 0, cy = 0;
    size_t base = 0;
    if (have) {
        cx = (int)((unsigned)col / (unsigned)g.ny);
        cy = (int)((unsigned)col % (unsigned)g.ny);
        int px = cx + g.rx;
        px -= (px >= g.nx) ? g.nx : 0;
        int py = cy + g.ry;
        py -= (py >= g.ny) ? g.ny : 0;
        base = ((size_t)px * g.ny + py) * (size_t)g.nz;
        if (!in_bounds(base + g.nz - 1, s.V, s.counters)) base = 0;
    }
    const uint4* hc = reinterpret_cast<const uint4*>(s.hits + base);
    const float4* mc = reinterpret_cast<const float4*>(s.minz + base);
    float h = __int_as_float(0x7f800000);
    bool any = false;
    if (have) {
        for (int v = sub; v < nv; v += LPC) {
            const uint4 hv = __ldg(hc + v);
            const float4 mv = __ldg(mc + v);
            if (hv.x) { h = fminf(h, mv.x); any = true; }
            if (hv.y) { h = fminf(h, mv.y); any = true; }
            if (hv.z) { h = fminf(h, mv.z); any = true; }
            if (hv.w) { h = fminf(h, mv.w); any = true; }
        }
    }
#pragma unroll
    for (int o = LPC / 2; o > 0; o >>= 1) h = fminf(h, __shfl_xor_sync(0xffffffffu, h, o));
    const bool col_any = (__ballot_sync(0xffffffffu, any) & gmask) != 0u;

    // Obstacle band: hits and passes summed over occupied voxels whose
    // lowest return lies in [h + obs_min_h, h + obs_max_h] (FP64
    // difference of the two floats, like the oracle).
    unsigned long long H = 0, M = 0;
    bool inband = false;
    if (have && col_any) {
        const uint4* pcv = reinterpret_cast<const uint4*>(s.passes + base);
        for (int v = sub; v < nv; v += LPC) {
            const uint4 hv = __ldg(hc + v);
            const float4 mv = __ldg(mc + v);
            const uint32_t hs[4] = {hv.x, hv.y, hv.z, hv.w};
            const float ms[4] = {mv.x, mv.y, mv.z, mv.w};
            bool need = false;
            bool in[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                in[k] = hs[k] != 0u && in_band(ms[k], h, band);
                need |= in[k];
            }
            if (need) {
                const uint4 pv = __ldg(pcv + v);
                const uint32_t ps[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (in[k]) {
                        H += hs[k];
                        M += ps[k];
                    }
                inband = true;
            }
        }
    }
    if (__ballot_sync(0xffffffffu, inband)) {  // warp-uniform: offsets stay inside a group
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) {
            H += __shfl_xor_sync(0xffffffffu, H, o);
            M += __shfl_xor_sync(0xffffffffu, M, o);
        }
    }
    if (have && sub == 0 && in_bounds((size_t)cx * g.ny + cy, (unsigned long long)g.nx * g.ny, s.counters)) {
        const size_t o = (size_t)cx * g.ny + cy;
        if (height) height[o] = col_any ? h : __int_as_float(0x7fffffff);
        uint8_t f = 0;
        float dens = 0.0f;
        if (H > 0) {
            dens = density_of(H, H + M);
            const bool hard = H * (unsigned long long)p.hard_den >= (unsigned long long)p.hard_num * (H + M);
            f = hard ? 3 : 5;
        }
        if (density) density[o] = dens;
        if (flags) flags[o] = f;
    }
}

// Vector column pass for nz % 4 == 0: LPC lanes per column, a grid-stride
// loop over column groups.
template <int LPC>
__global__ void __launch_bounds__(kColBlock) k_columns(MapState s, ExtractParams p, float* __restrict__ height,
                                                        float* __restrict__ density, uint8_t* __restrict__ flags) {
    pdl_wait();
    const long long ncols = (long long)p.g.nx * p.g.ny;
    const long long groups_per_warp = 32 / LPC;
    const long long gw = ((long long)blockIdx.x * kColBlock + threadIdx.x) >> 5;
    const long long cstride = (((long long)gridDim.x * kColBlock) >> 5) * groups_per_warp;
    for (long long colb = gw * groups_per_warp; colb < ncols; colb += cstride)
        columns_step<LPC>(s, p, height, density, flags, colb, ncols);
    pdl_done();
}

// ---- TMA-staged column pass (nz % 4 == 0) ----------------------------------
//
// The map state is column-major (z fastest), so C consecutive physical
// columns of hits (and of passes, and of lowest returns) are one contiguous
// run of C * nz * 4 bytes. One thread per block streams such runs into a
// ring of shared-memory stages with 1D bulk copies (cp.async.bulk,
// completion on an mbarrier per stage), kStages chunks ahead; all warps
// reduce the chunk in place, LPC = 8 lanes per column, with no global load
// on the reduction's path. Every mbarrier wait is bounded; a wait that gives
// up sets the map's status word and the block returns after draining the
// copies it issued. Used for nz % 4 == 0 and nz <= 256 (two stages of
// 3 x 32 columns fit shared memory; each stage's transaction count stays
// below the mbarrier's 2^20 bytes).

// Chunk shapes (columns per bulk-copy chunk x stages in flight): the default
// 32 x 2 and the variants the tuner may pick (gvom_tuning.col_shape).
constexpr int kTmaCols = 32;      // columns per chunk of the default shape (and of the batched form)
constexpr int kTmaStages = 2;
constexpr int kTmaBlock = 256;
size_t columns_tma_smem(int nz, int cols = kTmaCols, int stages = kTmaStages) {
    return 128 + (size_t)stages * 3 * cols * nz * sizeof(float);
}
struct ColShape {
    int cols, stages;
};
__host__ __device__ __forceinline__ ColShape col_shape_of(int code) {
    switch (code) {
        case 1: return ColShape{16, 4};
        case 2: return ColShape{32, 3};
        case 3: return ColShape{64, 2};
        default: return ColShape{32, 2};
    }
}

// One chunk of kTmaCols consecutive physical columns of one map.
struct ChunkRef {
    MapState s;
    ExtractParams p;
    float* height;
    float* density;
    uint8_t* flags;
    long long lc;  // the chunk's index within its map
};

// The chunks of one map (kCols columns each).
template <int kCols>
struct OneMapChunks {
    MapState s;
    ExtractParams p;
    float* height;
    float* density;
    uint8_t* flags;
    __device__ __forceinline__ long long total() const {
        return ((long long)p.g.nx * p.g.ny + kCols - 1) / kCols;
    }
    __device__ __forceinline__ ChunkRef at(long long c) const { return ChunkRef{s, p, height, density, flags, c}; }
};

// The chunks of every map of a batch step, map after map (col_prefix counts
// kColTask = kTmaCols columns per unit).
struct BatchChunks {
    BatchTables t;
    __device__ __forceinline__ long long total() const { return t.hdr->col_tasks; }
    __device__ __forceinline__ ChunkRef at(long long c) const {
        const int B = t.hdr->B;
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t.col_prefix[mid] <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchExtract& ex = t.ex[lo];
        return ChunkRef{ex.s, ex.p, ex.height, ex.density, ex.flags, c - t.col_prefix[lo]};
    }
};

// Starts the copies of chunk r into `stage` (stage buffers hold kCols
// columns of zmax voxels; the chunk's own columns are nz long).
template <int kCols>
__device__ __forceinline__ void tma_issue(const ChunkRef& r, int zmax, int stage, unsigned long long* bars, uint32_t* hb,
                                          float* mb, uint32_t* pb) {
    const int nz = r.p.g.nz;
    const long long ncols = (long long)r.p.g.nx * r.p.g.ny;
    const long long c0 = r.lc * kCols;
    const long long cols = ncols - c0 < kCols ? ncols - c0 : kCols;
    const unsigned bytes = (unsigned)(cols * nz * 4);
    const size_t so = (size_t)stage * kCols * zmax;
    if (!in_bounds((unsigned long long)(c0 + cols) * nz - 1, r.s.V, r.s.counters)) {
        mbar_arrive(&bars[stage]);  // nothing copied; the stage completes empty
        return;
    }
    mbar_expect_tx(&bars[stage], 3u * bytes);
    bulk_load(hb + so, r.s.hits + c0 * nz, bytes, &bars[stage]);
    bulk_load(mb + so, r.s.minz + c0 * nz, bytes, &bars[stage]);
    bulk_load(pb + so, r.s.passes + c0 * nz, bytes, &bars[stage]);
}

// The bulk-copy column pass over the chunks of `src` (a persistent grid;
// every map's nz is a multiple of 4 and at most zmax <= 256). A wait that
// gives up sets the status word of the map whose chunk it waited for.
template <int kCols, int kStages, typename Src>
__device__ __forceinline__ void columns_tma_body(const Src& src, int zmax) {
    // kLanes lanes reduce one column: 256 threads cover the chunk's kCols columns
    constexpr int kLanes = kTmaBlock / kCols;
    static_assert(kLanes >= 4 && kLanes <= 32 && (kLanes & (kLanes - 1)) == 0, "lanes per column");
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ int s_fail;
    const long long nchunks = src.total();
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sm);
    uint32_t* hb = reinterpret_cast<uint32_t*>(sm + 128);
    float* mb = reinterpret_cast<float*>(hb + (size_t)kStages * kCols * zmax);
    uint32_t* pb = reinterpret_cast<uint32_t*>(mb + (size_t)kStages * kCols * zmax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane & (kLanes - 1);           // lane within the column's group

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int st = 0; st < kStages; ++st) {
            const long long c = blockIdx.x + (long long)st * gridDim.x;
            if (c < nchunks) tma_issue<kCols>(src.at(c), zmax, st, bars, hb, mb, pb);
        }

    int k = 0;
    for (;; ++k) {
        const long long c = blockIdx.x + (long long)k * gridDim.x;
        if (c >= nchunks) break;
        const int st = k % kStages;
        if (!mbar_wait(&bars[st], (unsigned)((k / kStages) & 1))) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const ChunkRef r = src.at(c);
        const ExtractParams& p = r.p;
        const Geom g = p.g;
        const int nz = g.nz, nv = nz >> 2;
        const long long ncols = (long long)g.nx * g.ny;
        const Band band = make_band(p.obs_min_h, p.obs_max_h);
        const size_t so = (size_t)st * kCols * zmax;
        const uint32_t* hst = hb + so;
        const float* mst = mb + so;
        const uint32_t* pst = pb + so;
        const long long c0 = r.lc * kCols;
        // 8 warps x (32 / kLanes) columns = the chunk's kCols columns
        const int j = warp * (32 / kLanes) + lane / kLanes;
        const long long pc = c0 + j;                 // physical column
        const bool have = pc < ncols;
        const uint4* hv4 = reinterpret_cast<const uint4*>(hst + (size_t)j * nz);
        const float4* mv4 = reinterpret_cast<const float4*>(mst + (size_t)j * nz);
        float h = __int_as_float(0x7f800000);
        bool any = false;
        if (have)
            for (int v = sub; v < nv; v += kLanes) {
                const uint4 a = hv4[v];
                const float4 b = mv4[v];
                if (a.x) { h = fminf(h, b.x); any = true; }
                if (a.y) { h = fminf(h, b.y); any = true; }
                if (a.z) { h = fminf(h, b.z); any = true; }
                if (a.w) { h = fminf(h, b.w); any = true; }
            }
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) h = fminf(h, __shfl_xor_sync(0xffffffffu, h, o));
        const unsigned gm = kLanes == 32 ? 0xffffffffu : (((1u << kLanes) - 1u) << (lane & ~(kLanes - 1)));
        const bool col_any = (__ballot_sync(0xffffffffu, any) & gm) != 0u;
        unsigned long long H = 0, M = 0;
        bool inband = false;
        if (have && col_any)
            for (int v = sub; v < nv; v += kLanes) {
                const uint4 a = hv4[v];
                const float4 b = mv4[v];
                const uint4 pm = reinterpret_cast<const uint4*>(pst + (size_t)j * nz)[v];
                const uint32_t hs[4] = {a.x, a.y, a.z, a.w};
                const float ms[4] = {b.x, b.y, b.z, b.w};
                const uint32_t ps[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (hs[q] != 0u && in_band(ms[q], h, band)) {
                        H += hs[q];
                        M += ps[q];
                        inband = true;
                    }
            }
        if (__ballot_sync(0xffffffffu, inband)) {
#pragma unroll
            for (int o = kLanes / 2; o > 0; o >>= 1) {
                H += __shfl_xor_sync(0xffffffffu, H, o);
                M += __shfl_xor_sync(0xffffffffu, M, o);
            }
        }
        if (have && sub == 0 && in_bounds((unsigned long long)pc * nz + nz - 1, r.s.V, r.s.counters)) {
            // window coordinates of the physical column
            const int px = (int)((unsigned)pc / (unsigned)g.ny), py = (int)((unsigned)pc % (unsigned)g.ny);
            int cx = px - g.rx;
            cx += cx < 0 ? g.nx : 0;
            int cy = py - g.ry;
            cy += cy < 0 ? g.ny : 0;
            const size_t o = (size_t)cx * g.ny + cy;
            if (r.height) r.height[o] = col_any ? h : __int_as_float(0x7fffffff);
            uint8_t f = 0;
            float dens = 0.0f;
            if (H > 0) {
                dens = density_of(H, H + M);
                const bool hard = H * (unsigned long long)p.hard_den >= (unsigned long long)p.hard_num * (H + M);
                f = hard ? 3 : 5;
            }
            if (r.density) r.density[o] = dens;
            if (r.flags) r.flags[o] = f;
        }
        __syncthreads();  // every warp is done with this stage
        if (tid == 0) {
            const long long c2 = c + (long long)kStages * gridDim.x;
            if (c2 < nchunks) tma_issue<kCols>(src.at(c2), zmax, st, bars, hb, mb, pb);
        }
    }
    if (s_fail && tid == 0) {
        // drain the copies this block issued and has not consumed, then report
        for (int q = k; q < k + kStages; ++q) {
            const long long c = blockIdx.x + (long long)q * gridDim.x;
            if (c >= nchunks) break;
            mbar_wait(&bars[q % kStages], (unsigned)((q / kStages) & 1));
        }
        atomicOr(src.at(blockIdx.x + (long long)k * gridDim.x).s.counters + kStatus, kStatusTimeout);
    }
}

template <int kCols, int kStages>
__global__ void __launch_bounds__(kTmaBlock) k_columns_tma(MapState s, ExtractParams p, float* __restrict__ height,
                                                            float* __restrict__ density,
                                                            uint8_t* __restrict__ flags) {
    pdl_wait();
    columns_tma_body<kCols, kStages>(OneMapChunks<kCols>{s, p, height, density, flags}, p.g.nz);
    pdl_done();
}

__global__ void __launch_bounds__(kTmaBlock) k_columns_tma_batch(BatchTables t, int zmax) {
    columns_tma_body<kTmaCols, kTmaStages>(BatchChunks{t}, zmax);
}

// Tile edge of the pixel pass for halo R: for R <= 12 the tile whose row
// with both halos is one warp wide (tile + 2R = 32: each cone sweep step is
// one instruction per lane, and no lane idles), else 16.
// Tile edge of the pixel pass for halo R on an nx x ny map. While R <= 12 a
// tile row plus both halos is one warp wide (32 - 2R). For 12 < R <= 24 it is
// two warps wide (64 - 2R) if the map still has kWideTilesMin such tiles
// (two per SM): a wider tile halves the cone sweep's halo work per pixel.
// Otherwise, and beyond 24, the edge is 16.
constexpr long long kWideTilesMin = 2 * 152;

__host__ __device__ __forceinline__ int tile_for(int R, int nx, int ny) {
    if (R <= 12) return 32 - 2 * R;
    if (R <= 24) {
        const int t = 64 - 2 * R;
        if ((long long)((nx + t - 1) / t) * ((ny + t - 1) / t) >= kWideTilesMin) return t;
    }
    return 16;
}

__host__ __device__ __forceinline__ int tile_edge(const ExtractParams& p) {
    if (p.px_tile > 0) return p.px_tile;  // the tuner's choice
    const int R = p.neg_max_px > p.slope_n / 2 ? p.neg_max_px : p.slope_n / 2;
    return tile_for(R, p.g.nx, p.g.ny);
}
constexpr int kPxBlock = 256;        // eight warps: four sweep one cone direction each, four fit planes
constexpr int kPxBlockBatch = 128;   // the batched form: four warps, fits then cones (more blocks per SM)

// Cone state of a cell, packed into one 64-bit key: the distance D of the
// first ring holding ground in the high word, the lowest height on that ring
// (as order-preserving bits) in the low word. Smaller key = nearer ring,
// then lower height, so the state of a set of cones is their minimum key.
constexpr unsigned long long kNoGround = ~0ull;

__device__ __forceinline__ uint32_t height_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_height(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Order key of a height for the cone states (kNoKey: no ground). Finite
// heights never map to kNoKey, which only a NaN's bits would give.
constexpr uint32_t kNoKey = 0xffffffffu;

__device__ __forceinline__ uint32_t ground_key(float h) { return isnan(h) ? kNoKey : height_key(h); }

// One warp sweeps the cone recurrence of one direction over the tile. The
// cone grows along +u (sgn = +1) or -u (sgn = -1), u = the tile's row axis
// (x) when along_x, else its column axis (y). With Q(c) = min(own key of c
// (distance 0, its height) if c is defined, cone state of c), the cone
// state of a cell is min over its three ring-1 cells n of Q(n), one ring
// further (D + 1): ring d of a cell is the union of rings d - 1 of those
// three cells. A cone whose ring-1 line lies outside the grid along u, or
// whose distance passes neg_max_px, has no ground. Writes the cone value
// (lowest height on the first ring with ground, NaN if none) of each
// tile-interior pixel to val. Ks holds the heights' keys (ground_key), and
// Qbuf two lines of W + 2 states whose first and last entries stay
// kNoGround: the neighbours past the halo's edge, so no read tests v.
template <bool along_x>
__device__ void cone_sweep_warp(const ExtractParams& p, const uint32_t* Ks, int W, int R, int tile, int gx0, int gy0,
                                int sgn, unsigned long long* Qbuf, float* val) {
    // Ks rows are W + 1 words apart and val rows tile + 1, so that the
    // sweeps along y, whose lanes walk down a column, hit distinct banks
    const int WP = W + 1, TP = tile + 1, QL = W + 2;
    const int lane = threadIdx.x & 31;
    const int nmaj = along_x ? p.g.nx : p.g.ny;
    const int g0 = along_x ? gx0 : gy0;  // global coordinate of tile row 0 along u
    const int first = sgn > 0 ? W - 1 : 0;
    const int last = sgn > 0 ? R : R + tile - 1;
    const int nsteps = sgn > 0 ? first - last + 1 : last - first + 1;
    const uint32_t dmax = (uint32_t)p.neg_max_px;
    const float qnan = __int_as_float(0x7fffffff);
    if (lane < 4) Qbuf[(lane >> 1) * QL + (lane & 1) * (W + 1)] = kNoGround;
    __syncwarp();
    for (int st = 0; st < nsteps; ++st) {
        const int u = first - sgn * st;
        unsigned long long* Qcur = Qbuf + (st & 1) * QL + 1;
        const unsigned long long* Qprev = Qbuf + ((st + 1) & 1) * QL + 1;
        const int un = u + sgn;   // the ring-1 line (the previous step's)
        const int gun = g0 + un;  // its global coordinate
        const bool ring_ok = gun >= 0 && gun < nmaj && un >= 0 && un < W;
        const int iu = u - R;
        const bool out_row = iu >= 0 && iu < tile;  // this line holds tile pixels
#pragma unroll 2
        for (int v = lane; v < W; v += 32) {
            unsigned long long c = kNoGround;
            if (ring_ok) {
                const unsigned long long q = min(min(Qprev[v - 1], Qprev[v]), Qprev[v + 1]);
                // (kNoGround's distance word is above any limit)
                if ((uint32_t)(q >> 32) < dmax) c = q + (1ull << 32);
            }
            const uint32_t k = along_x ? Ks[u * WP + v] : Ks[v * WP + u];
            // own ground (distance 0) is nearer than any cone state
            Qcur[v] = k != kNoKey ? (unsigned long long)k : c;
            const int iv = v - R;
            if (out_row && iv >= 0 && iv < tile)
                val[along_x ? iu * TP + iv : iv * TP + iu] = c != kNoGround ? key_height((uint32_t)c) : qnan;
        }
        __syncwarp();
    }
}

// The same sweep with the cone line held in registers when the halo is at
// most 32 * kCells wide: lane l holds cells v = l and (kCells = 2) v = l + 32,
// and reads its neighbours' states of the previous line by warp shuffles
// instead of shared memory. Cells v >= W stay kNoGround (the line's edge).
template <bool along_x, int kCells>
__device__ __forceinline__ void cone_sweep_regs(const ExtractParams& p, const uint32_t* Ks, int W, int R, int tile,
                                                int gx0, int gy0, int sgn, float* val) {
    const int WP = W + 1, TP = tile + 1;
    const int lane = threadIdx.x & 31;
    const int nmaj = along_x ? p.g.nx : p.g.ny;
    const int g0 = along_x ? gx0 : gy0;
    const int first = sgn > 0 ? W - 1 : 0;
    const int last = sgn > 0 ? R : R + tile - 1;
    const int nsteps = sgn > 0 ? first - last + 1 : last - first + 1;
    const uint32_t dmax = (uint32_t)p.neg_max_px;
    const float qnan = __int_as_float(0x7fffffff);
    unsigned long long q0 = kNoGround, q1 = kNoGround;  // the previous line's states of this lane's cells
    for (int st = 0; st < nsteps; ++st) {
        const int u = first - sgn * st;
        const int un = u + sgn;
        const int gun = g0 + un;
        const bool ring_ok = gun >= 0 && gun < nmaj && un >= 0 && un < W;
        const int iu = u - R;
        const bool out_row = iu >= 0 && iu < tile;
        // neighbours v - 1 and v + 1 of each cell on the previous line
        unsigned long long l0, r0, l1 = kNoGround, r1 = kNoGround;
        if (kCells == 1) {
            l0 = __shfl_up_sync(0xffffffffu, q0, 1);
            r0 = __shfl_down_sync(0xffffffffu, q0, 1);
            if (lane == 0) l0 = kNoGround;
            if (lane == 31) r0 = kNoGround;
        } else {
            // cell 31's right neighbour is lane 0's second cell, cell 32's left
            // one lane 31's first cell
            l0 = __shfl_up_sync(0xffffffffu, q0, 1);
            r0 = __shfl_sync(0xffffffffu, lane == 0 ? q1 : q0, (lane + 1) & 31);
            l1 = __shfl_sync(0xffffffffu, lane == 31 ? q0 : q1, (lane + 31) & 31);
            r1 = __shfl_down_sync(0xffffffffu, q1, 1);
            if (lane == 0) l0 = kNoGround;
            if (lane == 31) r1 = kNoGround;
        }
#pragma unroll
        for (int k = 0; k < kCells; ++k) {
            const int v = lane + 32 * k;
            const unsigned long long qm = k == 0 ? q0 : q1, ql = k == 0 ? l0 : l1, qr = k == 0 ? r0 : r1;
            unsigned long long c = kNoGround;
            if (ring_ok) {
                const unsigned long long qq = min(min(ql, qm), qr);
                if ((uint32_t)(qq >> 32) < dmax) c = qq + (1ull << 32);
            }
            unsigned long long nq = kNoGround;
            if (v < W) {
                const uint32_t kk = along_x ? Ks[u * WP + v] : Ks[v * WP + u];
                nq = kk != kNoKey ? (unsigned long long)kk : c;
                const int iv = v - R;
                if (out_row && iv >= 0 && iv < tile)
                    val[along_x ? iu * TP + iv : iv * TP + iu] = c != kNoGround ? key_height((uint32_t)c) : qnan;
            }
            if (k == 0)
                q0 = nq;
            else
                q1 = nq;
        }
    }
}

// Least-squares plane z = a i + b j + c over the defined pixels of the
// (2r+1)^2 window around tile cell (ci, cj), z relative to the centre
// height h0. The normal matrix is integer (exact, so is the singularity
// test); the right-hand side and the solve are FP32.
template <int kR>
__device__ __forceinline__ void plane_fit(const ExtractParams& p, const float* Hs, int WP, int ci, int cj, float h0,
                                          float& sl, float& ro) {
    // kR > 0: compile-time radius (loops unrolled); kR == 0: run-time radius
    const int r = kR > 0 ? kR : p.slope_n / 2;
    int n = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
    float sz = 0.f, siz = 0.f, sjz = 0.f;
#pragma unroll (kR > 0 ? 2 * kR + 1 : 1)
    for (int i = -r; i <= r; ++i)
#pragma unroll (kR > 0 ? 2 * kR + 1 : 1)
        for (int j = -r; j <= r; ++j) {
            const float hv = Hs[(ci + i) * WP + (cj + j)];
            if (isnan(hv)) continue;
            const float z = hv - h0;
            n += 1;
            si += i;
            sj += j;
            sii += i * i;
            sjj += j * j;
            sij += i * j;
            sz += z;
            siz += (float)i * z;
            sjz += (float)j * z;
        }
    // adjugate of [sii sij si; sij sjj sj; si sj n] (symmetric)
    const long long A00 = (long long)sjj * n - (long long)sj * sj;
    const long long A01 = -((long long)sij * n - (long long)sj * si);
    const long long A02 = (long long)sij * sj - (long long)sjj * si;
    const long long A11 = (long long)sii * n - (long long)si * si;
    const long long A12 = -((long long)sii * sj - (long long)sij * si);
    const long long A22 = (long long)sii * sjj - (long long)sij * sij;
    const long long det = (long long)sii * A00 + (long long)sij * A01 + (long long)si * A02;
    if (n < p.slope_min_px || det == 0) return;
    const float inv = 1.0f / (float)det;
    const float a = ((float)A00 * siz + (float)A01 * sjz + (float)A02 * sz) * inv;
    const float b = ((float)A01 * siz + (float)A11 * sjz + (float)A12 * sz) * inv;
    const float c = ((float)A02 * siz + (float)A12 * sjz + (float)A22 * sz) * inv;
    float sse = 0.f;
#pragma unroll (kR > 0 ? 2 * kR + 1 : 1)
    for (int i = -r; i <= r; ++i)
#pragma unroll (kR > 0 ? 2 * kR + 1 : 1)
        for (int j = -r; j <= r; ++j) {
            const float hv = Hs[(ci + i) * WP + (cj + j)];
            if (isnan(hv)) continue;
            const float e = (hv - h0) - (a * (float)i + b * (float)j + c);
            sse += e * e;
        }
    sl = atanf(hypotf(a, b) / p.res);
    ro = sse / (float)n;
}

// One tile of tile x tile pixels per block of four or eight warps: load the
// tile and its halo; warp w < 4 sweeps cone w (+x, -x, +y, -y) and the
// planes of the defined pixels are fitted (by warps 4-7 at the same time,
// or by all warps first); then every pixel combines its four cone values.
__device__ __forceinline__ void tile_body(const ExtractParams& p, const float* __restrict__ height,
                                          float* __restrict__ slope, float* __restrict__ rough,
                                          uint8_t* __restrict__ flags, int tx0, int ty0, int tile, float* smem) {
    const int nx = p.g.nx, ny = p.g.ny;
    const int r = p.slope_n / 2;
    const int R = max(p.neg_max_px, r);
    const int W = tile + 2 * R;
    const int WP = W + 1, TP = tile + 1;                // padded row strides (no bank conflicts down columns)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int tt = tile * tile;
    const int tv = tile * TP;                           // one direction's padded cone values
    const int QL = W + 2;                               // one cone line with its two edge entries
    unsigned long long* Qbufs = reinterpret_cast<unsigned long long*>(smem);  // 4 * 2 lines of cone states
    float* Hs = smem + 16 * QL;                         // W rows of WP heights, NaN outside the grid
    uint32_t* Ks = reinterpret_cast<uint32_t*>(Hs + W * WP);  // their keys (ground_key)
    float* vals = reinterpret_cast<float*>(Ks + W * WP);      // 4 * tile rows of TP cone values
    const int gx0 = tx0 - R, gy0 = ty0 - R;             // global coordinates of tile cell (0, 0)
    const float qnan = __int_as_float(0x7fffffff);
    // t / tile for t < 2^16 as a high multiply: M = ceil(2^32 / tile) is exact
    // there (the error t (M - 2^32 / tile) / 2^32 < 2^-16 stays below 1 / tile)
    const uint32_t M = 0xffffffffu / (uint32_t)tile + 1u;

    // the tile and its halo: each warp takes rows warp, warp + nwarps, ...,
    // four rows (two 32-cell halves each) per round with all eight loads
    // issued before any shared store, so their latencies overlap
    constexpr int kRows = 4;
    for (int i0 = warp; i0 < W; i0 += nwarps * kRows)
        for (int j0 = 0; j0 < W; j0 += 64) {
            float hv[kRows][2];
#pragma unroll
            for (int b = 0; b < kRows; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + b * nwarps, j = j0 + lane + 32 * c;
                    const int gx = gx0 + i, gy = gy0 + j;
                    hv[b][c] = (i < W && j < W && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                                   ? height[(size_t)gx * ny + gy]
                                   : qnan;
                }
#pragma unroll
            for (int b = 0; b < kRows; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = i0 + b * nwarps, j = j0 + lane + 32 * c;
                    if (i < W && j < W) {
                        Hs[i * WP + j] = hv[b][c];
                        Ks[i * WP + j] = ground_key(hv[b][c]);
                    }
                }
        }
    __syncthreads();

    // with eight warps, warps 0-3 sweep the four cones while warps 4-7 fit
    // the planes; with four, all fit, then each sweeps one cone
    const bool split = flags && blockDim.x >= 256;
    const int fit0 = split ? 128 : 0;
    if ((slope || rough) && (!split || warp >= 4)) {
        for (int t = (int)threadIdx.x - fit0; t < tt; t += (int)blockDim.x - fit0) {
            const int li = (int)__umulhi((uint32_t)t, M), lj = t - li * tile;
            const int cx = tx0 + li, cy = ty0 + lj;
            if (cx >= nx || cy >= ny) continue;
            const int ci = li + R, cj = lj + R;
            const float h0 = Hs[ci * WP + cj];
            float sl = qnan, ro = qnan;
            if (!isnan(h0)) {
                if (r == 2)
                    plane_fit<2>(p, Hs, WP, ci, cj, h0, sl, ro);  // the default 5 x 5 window
                else if (r == 1)
                    plane_fit<1>(p, Hs, WP, ci, cj, h0, sl, ro);
                else
                    plane_fit<0>(p, Hs, WP, ci, cj, h0, sl, ro);
            }
            const size_t o = (size_t)cx * ny + cy;
            if (slope) slope[o] = sl;
            if (rough) rough[o] = ro;
        }
    }
    if (flags) {
        // warp w < 4 sweeps cone w (+x, -x, +y, -y); lines of up to 64 cells
        // live in registers, wider ones in shared memory
        if (warp < 4) {
            const int sgn = (warp & 1) ? -1 : 1;
            float* const val = vals + warp * tv;
            if (W <= 32) {
                if (warp < 2)
                    cone_sweep_regs<true, 1>(p, Ks, W, R, tile, gx0, gy0, sgn, val);
                else
                    cone_sweep_regs<false, 1>(p, Ks, W, R, tile, gx0, gy0, sgn, val);
            } else if (W <= 64) {
                if (warp < 2)
                    cone_sweep_regs<true, 2>(p, Ks, W, R, tile, gx0, gy0, sgn, val);
                else
                    cone_sweep_regs<false, 2>(p, Ks, W, R, tile, gx0, gy0, sgn, val);
            } else if (warp < 2) {
                cone_sweep_warp<true>(p, Ks, W, R, tile, gx0, gy0, sgn, Qbufs + warp * 2 * QL, val);
            } else {
                cone_sweep_warp<false>(p, Ks, W, R, tile, gx0, gy0, sgn, Qbufs + warp * 2 * QL, val);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < tt; t += blockDim.x) {
            const int li = (int)__umulhi((uint32_t)t, M), lj = t - li * tile;
            const int cx = tx0 + li, cy = ty0 + lj;
            if (cx >= nx || cy >= ny) continue;
            if (!isnan(Hs[(li + R) * WP + (lj + R)])) continue;
            int nf = 0;
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float v = vals[c * tv + li * TP + lj];
                if (isnan(v)) continue;
                lo = nf ? fminf(lo, v) : v;
                hi = nf ? fmaxf(hi, v) : v;
                nf += 1;
            }
            if (nf >= 2 && exceeds(hi, lo, p.neg_thresh)) flags[(size_t)cx * ny + cy] |= 8u;
        }
    }
    __syncthreads();  // the caller may reuse the shared arrays for its next tile
}

__global__ void __launch_bounds__(kPxBlock, 4)
    k_slope_negative(ExtractParams p, const float* __restrict__ height, float* __restrict__ slope,
                     float* __restrict__ rough, uint8_t* __restrict__ flags) {
    pdl_wait();
    extern __shared__ float smem[];
    const int tile = tile_edge(p);
    tile_body(p, height, slope, rough, flags, blockIdx.y * tile, blockIdx.x * tile, tile, smem);
    pdl_done();
}

// ---- batched maps ----------------------------------------------------------

__device__ __forceinline__ int find_map_x(const long long* __restrict__ prefix, int B, long long u) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Column pass of all maps: persistent warps over 64-column tasks.
__global__ void __launch_bounds__(kColBlock) k_columns_batch(BatchTables t) {
    const int B = t.hdr->B;
    const long long total = t.hdr->col_tasks;
    const long long nwarps = ((long long)gridDim.x * kColBlock) >> 5;
    for (long long u = ((long long)blockIdx.x * kColBlock + threadIdx.x) >> 5; u < total; u += nwarps) {
        const int m = find_map_x(t.col_prefix, B, u);
        const BatchExtract& ex = t.ex[m];
        const long long ncols = (long long)ex.p.g.nx * ex.p.g.ny;
        const long long c0 = (u - t.col_prefix[m]) * kColTask;
        const long long c1 = c0 + kColTask < ncols ? c0 + kColTask : ncols;
        const int nz = ex.p.g.nz;
        if ((nz & 3) == 0) {
            const int nv = nz >> 2;
            if (nv <= 8) {
                for (long long c = c0; c < c1; c += 4) columns_step<8>(ex.s, ex.p, ex.height, ex.density, ex.flags, c, c1);
            } else if (nv <= 16) {
                for (long long c = c0; c < c1; c += 2)
                    columns_step<16>(ex.s, ex.p, ex.height, ex.density, ex.flags, c, c1);
            } else {
                for (long long c = c0; c < c1; c += 1)
                    columns_step<32>(ex.s, ex.p, ex.height, ex.density, ex.flags, c, c1);
            }
        } else {
            for (long long c = c0; c < c1; ++c) column_scalar(ex.s, ex.p, ex.height, ex.density, ex.flags, c);
        }
    }
}

// Plane-fit / cone pass of all maps: a persistent grid over pixel tiles.
__global__ void __launch_bounds__(kPxBlockBatch, 8) k_slope_negative_batch(BatchTables t) {
    extern __shared__ float smem[];
    const int B = t.hdr->B;
    const long long total = t.hdr->tiles;
    for (long long u = blockIdx.x; u < total; u += gridDim.x) {
        const int m = find_map_x(t.tile_prefix, B, u);
        const BatchExtract& ex = t.ex[m];
        const long long lt = u - t.tile_prefix[m];
        const int tile = tile_edge(ex.p);
        const int tiles_y = (ex.p.g.ny + tile - 1) / tile;
        tile_body(ex.p, ex.height, ex.slope, ex.rough, ex.flags, (int)((unsigned)lt / (unsigned)tiles_y) * tile,
                  (int)((unsigned)lt % (unsigned)tiles_y) * tile, tile, smem);
    }
}

size_t slope_negative_smem_tile(int R, int tile) {
    // cone lines (4 directions x 2 lines of W + 2 states), heights and their
    // keys (W rows of W + 1), cone values (4 x tile rows of tile + 1)
    const int W = tile + 2 * R;
    return sizeof(unsigned long long) * 8 * (size_t)(W + 2) + 2 * sizeof(float) * (size_t)W * (W + 1) +
           sizeof(float) * 4 * (size_t)tile * (tile + 1);
}


__global__ void k_gather_voxels(MapState s, Geom g, uint32_t* __restrict__ hits, uint32_t* __restrict__ passes,
                                float* __restrict__ minz) {
    const long long V = (long long)g.nx * g.ny * g.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride) {
        const int cz = (int)(i % g.nz);
        const long long col = i / g.nz;
        const int cy = (int)(col % g.ny), cx = (int)(col / g.ny);
        int px = cx + g.rx;
        px -= (px >= g.nx) ? g.nx : 0;
        int py = cy + g.ry;
        py -= (py >= g.ny) ? g.ny : 0;
        int pz = cz + g.rz;
        pz -= (pz >= g.nz) ? g.nz : 0;
        const size_t k = ((size_t)px * g.ny + py) * (size_t)g.nz + pz;
        if (!in_bounds(k, s.V, s.counters)) continue;
        if (hits) hits[i] = s.hits[k];
        if (passes) passes[i] = s.passes[k];
        if (minz) minz[i] = s.minz[k];
    }
}

// The inverse of k_gather_voxels: logical (window-order) arrays into the
// toroidal state.
__global__ void k_scatter_voxels(MapState s, Geom g, const uint32_t* __restrict__ hits,
                                 const uint32_t* __restrict__ passes, const float* __restrict__ minz) {
    const long long V = (long long)g.nx * g.ny * g.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride) {
        const int cz = (int)(i % g.nz);
        const long long col = i / g.nz;
        const int cy = (int)(col % g.ny), cx = (int)(col / g.ny);
        int px = cx + g.rx;
        px -= (px >= g.nx) ? g.nx : 0;
        int py = cy + g.ry;
        py -= (py >= g.ny) ? g.ny : 0;
        int pz = cz + g.rz;
        pz -= (pz >= g.nz) ? g.nz : 0;
        const size_t k = ((size_t)px * g.ny + py) * (size_t)g.nz + pz;
        if (!in_bounds(k, s.V, s.counters)) continue;
        s.hits[k] = hits[i];
        s.passes[k] = passes[i];
        s.minz[k] = minz[i];
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

size_t slope_negative_smem(const ExtractParams& p) { return slope_negative_smem_tile(tile_halo(p), tile_edge(p)); }

cudaError_t allow_smem(const void* kernel, std::atomic<int>* cache, size_t bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (cache[dev].load(std::memory_order_relaxed) >= (int)bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cache[dev].store((int)bytes, std::memory_order_relaxed);
    return e;
}

int tile_halo(const ExtractParams& p) { return p.neg_max_px > p.slope_n / 2 ? p.neg_max_px : p.slope_n / 2; }

long long tiles_of(const ExtractParams& p) {
    const int t = tile_edge(p);
    return (long long)((p.g.nx + t - 1) / t) * ((p.g.ny + t - 1) / t);
}

// Blocks per SM of the bulk-copy column pass: as many as shared memory
// holds at once (1 KB of each block's share is reserved), at most 4.
long long columns_tma_blocks_per_sm(size_t smem) {
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    long long per_sm = (long long)smem_sm / (long long)(smem + 1024);
    if (per_sm > 4) per_sm = 4;
    return per_sm < 1 ? 1 : per_sm;
}

cudaError_t launch_batch_extract(const BatchTables& t, int max_maps, size_t px_smem, int zmax, cudaStream_t st) {
    (void)max_maps;
    const int sms = sm_count();
    cudaError_t e;
    count_launch();
    if (zmax > 0) {
        const size_t smem = columns_tma_smem(zmax);
        static std::atomic<int> cache[64];
        e = allow_smem((const void*)k_columns_tma_batch, cache, smem);
        if (e != cudaSuccess) return e;
        k_columns_tma_batch<<<(unsigned)(sms * columns_tma_blocks_per_sm(smem)), kTmaBlock, smem, st>>>(t, zmax);
    } else {
        k_columns_batch<<<(unsigned)(sms * 8), kColBlock, 0, st>>>(t);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = px_smem;
    if (smem > 48 * 1024) {
        static std::atomic<int> cache[64];
        e = allow_smem((const void*)k_slope_negative_batch, cache, smem);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    k_slope_negative_batch<<<(unsigned)(sms * 8), kPxBlockBatch, smem, st>>>(t);
    return cudaGetLastError();
}

template <int kCols, int kStages>
cudaError_t launch_columns_tma(const MapState& s, const ExtractParams& p, float* height, float* density,
                               uint8_t* flags, long long cols, cudaStream_t st) {
    const size_t smem = columns_tma_smem(p.g.nz, kCols, kStages);
    static std::atomic<int> cache[64];
    cudaError_t e = allow_smem((const void*)k_columns_tma<kCols, kStages>, cache, smem);
    if (e != cudaSuccess) return e;
    const long long chunks = (cols + kCols - 1) / kCols;
    long long blocks = (long long)sm_count() * columns_tma_blocks_per_sm(smem);
    if (blocks > chunks) blocks = chunks;
    count_launch();
    return launch_pdl(k_columns_tma<kCols, kStages>, dim3((unsigned)blocks), dim3(kTmaBlock), smem, st, s, p, height,
                      density, flags);
}

cudaError_t launch_columns(const MapState& s, const ExtractParams& p, float* height, float* density, uint8_t* flags,
                           cudaStream_t st) {
    const long long cols = (long long)p.g.nx * p.g.ny;
    if ((p.g.nz & 3) == 0 && p.g.nz <= 256 && s.counters != nullptr) {
        // a shape whose stages do not fit shared memory (or exceed a
        // barrier's transaction count) falls back to the default one
        ColShape cs = col_shape_of(p.col_shape);
        if (columns_tma_smem(p.g.nz, cs.cols, cs.stages) > 200 * 1024 ||
            (size_t)3 * cs.cols * p.g.nz * 4 >= (1u << 20))
            cs = col_shape_of(0);
        switch (cs.cols * 16 + cs.stages) {
            case 16 * 16 + 4: return launch_columns_tma<16, 4>(s, p, height, density, flags, cols, st);
            case 32 * 16 + 3: return launch_columns_tma<32, 3>(s, p, height, density, flags, cols, st);
            case 64 * 16 + 2: return launch_columns_tma<64, 2>(s, p, height, density, flags, cols, st);
            default: return launch_columns_tma<32, 2>(s, p, height, density, flags, cols, st);
        }
    }
    count_launch();
    if ((p.g.nz & 3) != 0) {
        const long long blocks = (cols * 32 + kColBlock - 1) / kColBlock;
        return launch_pdl(k_columns_scalar, dim3((unsigned)blocks), dim3(kColBlock), 0, st, s, p, height, density,
                          flags);
    }
    const int nv = p.g.nz / 4;
    const int lpc = nv <= 8 ? 8 : (nv <= 16 ? 16 : 32);
    const long long groups = (cols + (32 / lpc) - 1) / (32 / lpc);  // warps needed for one column each
    long long blocks = (groups * 32 + kColBlock - 1) / kColBlock;
    const long long cap = (long long)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (lpc == 8)
        return launch_pdl(k_columns<8>, dim3((unsigned)blocks), dim3(kColBlock), 0, st, s, p, height, density, flags);
    if (lpc == 16)
        return launch_pdl(k_columns<16>, dim3((unsigned)blocks), dim3(kColBlock), 0, st, s, p, height, density, flags);
    return launch_pdl(k_columns<32>, dim3((unsigned)blocks), dim3(kColBlock), 0, st, s, p, height, density, flags);
}

cudaError_t launch_slope_negative(const ExtractParams& p, const float* height, float* slope, float* rough,
                                  uint8_t* flags, cudaStream_t st) {
    const size_t smem = slope_negative_smem(p);
    if (smem > 48 * 1024) {
        static std::atomic<int> cache[64];
        const cudaError_t e =
            allow_smem((const void*)k_slope_negative, cache, smem);
        if (e != cudaSuccess) return e;
    }
    const int tile = tile_edge(p);
    dim3 grid((p.g.ny + tile - 1) / tile, (p.g.nx + tile - 1) / tile);
    count_launch();
    return launch_pdl(k_slope_negative, grid, dim3(kPxBlock), smem, st, p, height, slope, rough, flags);
}

cudaError_t launch_scatter_voxels(const MapState& s, const Geom& g, const uint32_t* hits, const uint32_t* passes,
                                  const float* minz, cudaStream_t st) {
    const long long V = (long long)g.nx * g.ny * g.nz;
    long long blocks = (V + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    count_launch();
    k_scatter_voxels<<<(unsigned)blocks, 256, 0, st>>>(s, g, hits, passes, minz);
    return cudaGetLastError();
}

cudaError_t launch_gather_voxels(const MapState& s, const Geom& g, uint32_t* hits, uint32_t* passes, float* minz,
                                 cudaStream_t st) {
    const long long V = (long long)g.nx * g.ny * g.nz;
    long long blocks = (V + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    count_launch();
    k_gather_voxels<<<(unsigned)blocks, 256, 0, st>>>(s, g, hits, passes, minz);
    return cudaGetLastError();
}

}  // namespace gvom
