// 2D products of the voxel map (G-VOM Sec. III-D) for sm_103a.
//
// k_columns: one warp per map column streams the column's hits, passes and
// lowest-return heights (contiguous in memory: z is the fastest axis) and
// reduces them with warp shuffles into the height, the positive obstacle
// band sums, density and hard/soft flags.
// k_slope_negative: one thread per pixel over the height map. A defined
// pixel gets the N x N least-squares plane (slope, roughness); an
// undefined one runs the four-cone negative obstacle search. The two are
// exclusive per pixel, so one launch covers both.
#include <math.h>

#include "gvom_internal.h"

namespace gvom {

namespace {

constexpr int kColBlock = 256;

__global__ void __launch_bounds__(kColBlock) k_columns(MapState s, ExtractParams p, float* __restrict__ height,
                                                        float* __restrict__ density, uint8_t* __restrict__ flags) {
    const Geom g = p.g;
    const long long col = ((long long)blockIdx.x * kColBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= (long long)g.nx * g.ny) return;
    const int cx = (int)(col / g.ny), cy = (int)(col % g.ny);
    int px = cx + g.rx;
    px -= (px >= g.nx) ? g.nx : 0;
    int py = cy + g.ry;
    py -= (py >= g.ny) ? g.ny : 0;
    const size_t base = ((size_t)px * g.ny + py) * (size_t)g.nz;
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
        const double hd = (double)h;
        const double lo = (double)p.obs_min_h, hi = (double)p.obs_max_h;
        for (int z = lane; z < g.nz; z += 32) {
            const uint32_t nh = hc[z];
            if (nh == 0u) continue;
            const double above = __dsub_rn((double)mc[z], hd);
            if (lo <= above && above <= hi) {
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
    if (lane == 0) {
        const size_t o = (size_t)cx * g.ny + cy;
        if (height) height[o] = any ? h : __int_as_float(0x7fffffff);
        uint8_t f = 0;
        float dens = 0.0f;
        if (H > 0) {
            dens = __double2float_rn(__ddiv_rn((double)H, (double)(H + M)));
            const bool hard = H * (unsigned long long)p.hard_den >= (unsigned long long)p.hard_num * (H + M);
            f = hard ? 3 : 5;
        }
        if (density) density[o] = dens;
        if (flags) flags[o] = f;
    }
}

constexpr int kPxBlockX = 32, kPxBlockY = 8;

__global__ void __launch_bounds__(kPxBlockX* kPxBlockY)
    k_slope_negative(ExtractParams p, const float* __restrict__ height, float* __restrict__ slope,
                     float* __restrict__ rough, uint8_t* __restrict__ flags) {
    const int nx = p.g.nx, ny = p.g.ny;
    const int cy = blockIdx.x * kPxBlockX + threadIdx.x;
    const int cx = blockIdx.y * kPxBlockY + threadIdx.y;
    if (cx >= nx || cy >= ny) return;
    const size_t o = (size_t)cx * ny + cy;
    const float h0 = height[o];
    const float qnan = __int_as_float(0x7fffffff);

    if (!isnan(h0)) {
        // Least-squares plane z = a i + b j + c over the defined pixels of
        // the N x N window, z relative to the centre height. The normal
        // matrix is integer (exact); the right-hand side is FP32.
        const int r = p.slope_n / 2;
        int n = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
        float sz = 0.f, siz = 0.f, sjz = 0.f;
        for (int i = -r; i <= r; ++i) {
            const int x = cx + i;
            if (x < 0 || x >= nx) continue;
            for (int j = -r; j <= r; ++j) {
                const int y = cy + j;
                if (y < 0 || y >= ny) continue;
                const float hv = height[(size_t)x * ny + y];
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
        }
        float sl = qnan, ro = qnan;
        // adjugate of [sii sij si; sij sjj sj; si sj n] (symmetric)
        const long long A00 = (long long)sjj * n - (long long)sj * sj;
        const long long A01 = -((long long)sij * n - (long long)sj * si);
        const long long A02 = (long long)sij * sj - (long long)sjj * si;
        const long long A11 = (long long)sii * n - (long long)si * si;
        const long long A12 = -((long long)sii * sj - (long long)sij * si);
        const long long A22 = (long long)sii * sjj - (long long)sij * sij;
        const long long det = (long long)sii * A00 + (long long)sij * A01 + (long long)si * A02;
        if (n >= p.slope_min_px && det != 0) {
            const float inv = 1.0f / (float)det;
            const float a = ((float)A00 * siz + (float)A01 * sjz + (float)A02 * sz) * inv;
            const float b = ((float)A01 * siz + (float)A11 * sjz + (float)A12 * sz) * inv;
            const float c = ((float)A02 * siz + (float)A12 * sjz + (float)A22 * sz) * inv;
            float sse = 0.f;
            for (int i = -r; i <= r; ++i) {
                const int x = cx + i;
                if (x < 0 || x >= nx) continue;
                for (int j = -r; j <= r; ++j) {
                    const int y = cy + j;
                    if (y < 0 || y >= ny) continue;
                    const float hv = height[(size_t)x * ny + y];
                    if (isnan(hv)) continue;
                    const float e = (hv - h0) - (a * (float)i + b * (float)j + c);
                    sse += e * e;
                }
            }
            sl = atanf(hypotf(a, b) / p.res);
            ro = sse / (float)n;
        }
        if (slope) slope[o] = sl;
        if (rough) rough[o] = ro;
        return;
    }

    if (slope) slope[o] = qnan;
    if (rough) rough[o] = qnan;
    // Negative obstacle search: four cones (+x, -x, +y, -y), ring by ring.
    int nfound = 0;
    float lo = 0.f, hi = 0.f;
#pragma unroll 1
    for (int cone = 0; cone < 4; ++cone) {
        const int ax = cone < 2 ? 1 : 0;  // 1: the ring is a fixed x
        const int sgn = (cone & 1) ? -1 : 1;
        for (int d = 1; d <= p.neg_max_px; ++d) {
            const int fixed = (ax ? cx : cy) + sgn * d;
            if (fixed < 0 || fixed >= (ax ? nx : ny)) break;
            const int centre = ax ? cy : cx;
            const int lim = ax ? ny : nx;
            const int s0 = max(centre - d, 0), s1 = min(centre + d, lim - 1);
            float best = __int_as_float(0x7f800000);
            bool found = false;
            for (int s = s0; s <= s1; ++s) {
                const float hv = ax ? height[(size_t)fixed * ny + s] : height[(size_t)s * ny + fixed];
                if (!isnan(hv)) {
                    best = fminf(best, hv);
                    found = true;
                }
            }
            if (found) {
                lo = nfound ? fminf(lo, best) : best;
                hi = nfound ? fmaxf(hi, best) : best;
                nfound += 1;
                break;
            }
        }
    }
    if (flags && nfound >= 2 && __dsub_rn((double)hi, (double)lo) > (double)p.neg_thresh) flags[o] |= 8u;
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
        if (hits) hits[i] = s.hits[k];
        if (passes) passes[i] = s.passes[k];
        if (minz) minz[i] = s.minz[k];
    }
}

}  // namespace

cudaError_t launch_columns(const MapState& s, const ExtractParams& p, float* height, float* density, uint8_t* flags,
                           cudaStream_t st) {
    const long long cols = (long long)p.g.nx * p.g.ny;
    const long long blocks = (cols * 32 + kColBlock - 1) / kColBlock;
    count_launch();
    k_columns<<<(unsigned)blocks, kColBlock, 0, st>>>(s, p, height, density, flags);
    return cudaGetLastError();
}

cudaError_t launch_slope_negative(const ExtractParams& p, const float* height, float* slope, float* rough,
                                  uint8_t* flags, cudaStream_t st) {
    dim3 block(kPxBlockX, kPxBlockY);
    dim3 grid((p.g.ny + kPxBlockX - 1) / kPxBlockX, (p.g.nx + kPxBlockY - 1) / kPxBlockY);
    count_launch();
    k_slope_negative<<<grid, block, 0, st>>>(p, height, slope, rough, flags);
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
