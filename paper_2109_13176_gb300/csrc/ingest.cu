// Per-scan ingest (G-VOM Sec. III-C, combined per Sec. III-D) and window
// shift (Sec. III-A origin, Sec. III-D index offset) for sm_103a.
//
// One thread per lidar point: transform in FP64 without fused operations,
// filter, quantise to 1/256 voxel, bin the hit, then walk the exact integer
// traversal from the sensor to the point and count a pass in every other
// window voxel it meets. Pass counts of lanes that stand in the same voxel
// at the same step are merged (__match_any_sync) so that the many rays
// leaving the sensor together cost one L2 atomic per warp, not one per ray.
#include "gvom_internal.h"

namespace gvom {

namespace {

constexpr int kIngestBlock = 256;
constexpr double kQLim = 1073741824.0;  // 2^30: quantised coordinates stay below this magnitude

__device__ __forceinline__ bool in_window(const Geom& g, int cx, int cy, int cz) {
    return (unsigned)cx < (unsigned)g.nx && (unsigned)cy < (unsigned)g.ny && (unsigned)cz < (unsigned)g.nz;
}

__device__ __forceinline__ uint32_t phys_index(const Geom& g, int cx, int cy, int cz) {
    int px = cx + g.rx;
    px -= (px >= g.nx) ? g.nx : 0;
    int py = cy + g.ry;
    py -= (py >= g.ny) ? g.ny : 0;
    int pz = cz + g.rz;
    pz -= (pz >= g.nz) ? g.nz : 0;
    return ((uint32_t)px * (uint32_t)g.ny + (uint32_t)py) * (uint32_t)g.nz + (uint32_t)pz;
}

// Lowest-return height as an atomic float minimum. For v >= 0 the IEEE bit
// patterns order like signed ints; for v < 0 they order in reverse as
// unsigned ints, and any negative float compares above every non-negative
// one as unsigned. Exact for every non-NaN value (+inf is the empty state).
__device__ __forceinline__ void atomic_min_f32(float* addr, float v) {
    if (v >= 0.0f)
        atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else
        atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

// Sec. III-C transform, one row of [R | t]: ((r0 px + r1 py) + r2 pz) + t,
// each operation rounded on its own (no FMA contraction).
__device__ __forceinline__ double xform_row(const double* T, double px, double py, double pz) {
    return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(T[0], px), __dmul_rn(T[1], py)), __dmul_rn(T[2], pz)), T[3]);
}

// Quantise a map-frame coordinate: q = round-half-even(256 (w / res - origin)).
__device__ __forceinline__ bool quantise(double w, double inv_res, long long origin, int* q) {
    const double v = __dsub_rn(__dmul_rn(w, inv_res), (double)origin);
    const double s = v * 256.0;  // exact: scaling by a power of two
    if (!(fabs(s) < kQLim)) return false;
    *q = (int)__double2ll_rn(s);
    return true;
}

// Per-axis state of the exact traversal. The next voxel boundary on this
// axis is reached at t = num / den along the segment (den = |d|); a walk
// that moves up takes the new voxel at t, one that moves down just after t.
struct Axis {
    int c;         // current voxel
    int rem;       // boundaries left to cross
    int dir;       // +1, -1, or 0
    uint32_t num;  // < 2^31 + 256
    uint32_t den;  // |d| < 2^31
};

__device__ __forceinline__ void axis_init(Axis& ax, int a, int b) {
    ax.c = a >> 8;
    const int ce = b >> 8;
    const int d = b - a;
    if (d > 0) {
        ax.dir = 1;
        ax.den = (uint32_t)d;
        ax.num = (uint32_t)(256 * (ax.c + 1) - a);
        ax.rem = ce - ax.c;
    } else if (d < 0) {
        ax.dir = -1;
        ax.den = (uint32_t)(-d);
        ax.num = (uint32_t)(a - 256 * ax.c);
        ax.rem = ax.c - ce;
    } else {
        ax.dir = 0;
        ax.den = 1;
        ax.num = 0;
        ax.rem = 0;
    }
}

// Whether axis i's next crossing comes strictly before axis j's: earlier t,
// or the same t with i moving up and j moving down.
__device__ __forceinline__ bool before(const Axis& i, const Axis& j) {
    const unsigned long long l = (unsigned long long)i.num * j.den;
    const unsigned long long r = (unsigned long long)j.num * i.den;
    return l < r || (l == r && i.dir > j.dir);
}

__device__ __forceinline__ bool same_event(const Axis& i, const Axis& j) {
    return i.dir == j.dir && (unsigned long long)i.num * j.den == (unsigned long long)j.num * i.den;
}

__device__ __forceinline__ void axis_step(Axis& ax) {
    ax.c += ax.dir;
    ax.num += 256u;
    ax.rem -= 1;
}

// Whether the walk has left the window for good on this axis.
__device__ __forceinline__ bool gone(const Axis& ax, int n) {
    return (ax.dir > 0 && ax.c >= n) || (ax.dir < 0 && ax.c < 0);
}

__global__ void __launch_bounds__(kIngestBlock) k_ingest(const IngestArgs a) {
    const long long i = (long long)blockIdx.x * kIngestBlock + threadIdx.x;
    const Geom g = a.g;

    bool valid = false;
    int q[3] = {0, 0, 0};
    float wz = 0.0f;
    int qo[3];
    bool sensor_ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) sensor_ok &= quantise(a.T[4 * k + 3], a.inv_res, a.origin[k], &qo[k]);

    if (i < a.n) {
        const float* p = a.pts + i * a.stride;
        float fx, fy, fz;
        if (a.stride == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p));
            fx = v.x;
            fy = v.y;
            fz = v.z;
        } else {
            fx = __ldg(p);
            fy = __ldg(p + 1);
            fz = __ldg(p + 2);
        }
        if (isfinite(fx) && isfinite(fy) && isfinite(fz) && sensor_ok) {
            const double px = fx, py = fy, pz = fz;
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
            if (r2 > 0.0 && r2 <= a.r2max) {
                const double wx = xform_row(a.T + 0, px, py, pz);
                const double wy = xform_row(a.T + 4, px, py, pz);
                const double wzd = xform_row(a.T + 8, px, py, pz);
                valid = quantise(wx, a.inv_res, a.origin[0], &q[0]) && quantise(wy, a.inv_res, a.origin[1], &q[1]) &&
                        quantise(wzd, a.inv_res, a.origin[2], &q[2]);
                wz = __double2float_rn(wzd);
            }
        }
    }

    int hit_in_window = 0;
    unsigned long long visits = 0;
    if (valid) {
        const int ex = q[0] >> 8, ey = q[1] >> 8, ez = q[2] >> 8;
        if (in_window(g, ex, ey, ez)) {
            const uint32_t k = phys_index(g, ex, ey, ez);
            atomicAdd(a.s.hits + k, 1u);
            atomic_min_f32(a.s.minz + k, wz);
            hit_in_window = 1;
        }

        Axis X, Y, Z;
        axis_init(X, qo[0], q[0]);
        axis_init(Y, qo[1], q[1]);
        axis_init(Z, qo[2], q[2]);
        int total = X.rem + Y.rem + Z.rem;
        // Walk every voxel but the last (the endpoint voxel gets the hit).
        while (total > 0) {
            const bool inside = in_window(g, X.c, Y.c, Z.c);
            const uint32_t key = inside ? phys_index(g, X.c, Y.c, Z.c) : 0xffffffffu;
            const unsigned int active = __activemask();
            const unsigned int peers = __match_any_sync(active, key);
            if (inside) {
                const int lane = threadIdx.x & 31;
                if (lane == __ffs(peers) - 1) atomicAdd(a.s.passes + key, (uint32_t)__popc(peers));
                visits += 1;
            }
            // the axis (or axes) whose boundary comes next
            Axis M = X;
            bool have = X.rem > 0;
            if (Y.rem > 0 && (!have || before(Y, M))) {
                M = Y;
                have = true;
            }
            if (Z.rem > 0 && (!have || before(Z, M))) M = Z;
            const bool sx = X.rem > 0 && same_event(X, M);
            const bool sy = Y.rem > 0 && same_event(Y, M);
            const bool sz = Z.rem > 0 && same_event(Z, M);
            if (sx) axis_step(X);
            if (sy) axis_step(Y);
            if (sz) axis_step(Z);
            total -= (int)sx + (int)sy + (int)sz;
            // once past the window on any axis the walk never comes back
            if (gone(X, g.nx) || gone(Y, g.ny) || gone(Z, g.nz)) break;
        }
    }

    // Counters: one atomic per block and counter.
    __shared__ unsigned long long red[3][kIngestBlock / 32];
    unsigned long long v0 = valid ? 1ull : 0ull, v1 = (unsigned long long)hit_in_window, v2 = visits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][warp] = v0;
        red[1][warp] = v1;
        red[2][warp] = v2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long s = 0;
        for (int w = 0; w < kIngestBlock / 32; ++w) s += red[threadIdx.x][w];
        if (s) atomicAdd(a.s.counters + kRaysValid + threadIdx.x, s);
    }
}

// Fill the state with the empty voxel: no hits, no passes, min height +inf.
__global__ void k_init_state(uint32_t* __restrict__ hits, uint32_t* __restrict__ passes, float* __restrict__ minz,
                             long long V) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride) {
        hits[i] = 0u;
        passes[i] = 0u;
        minz[i] = __int_as_float(0x7f800000);
    }
}

// Clear the voxels that enter the window on a shift by d (new - old origin,
// |d_k| < n_k on every axis). One warp per window column: a column whose x
// or y is new is cleared whole; otherwise only its new z range.
__global__ void k_shift(MapState s, Geom g, int dx, int dy, int dz) {
    const long long col = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= (long long)g.nx * g.ny) return;
    const int cx = (int)(col / g.ny), cy = (int)(col % g.ny);
    const bool new_x = dx > 0 ? cx >= g.nx - dx : cx < -dx;
    const bool new_y = dy > 0 ? cy >= g.ny - dy : cy < -dy;
    int z0, z1;
    if (new_x || new_y) {
        z0 = 0;
        z1 = g.nz;
    } else if (dz > 0) {
        z0 = g.nz - dz;
        z1 = g.nz;
    } else {
        z0 = 0;
        z1 = -dz;
    }
    if (z0 >= z1) return;
    int px = cx + g.rx;
    px -= (px >= g.nx) ? g.nx : 0;
    int py = cy + g.ry;
    py -= (py >= g.ny) ? g.ny : 0;
    const uint32_t base = ((uint32_t)px * g.ny + py) * (uint32_t)g.nz;
    for (int cz = z0 + lane; cz < z1; cz += 32) {
        int pz = cz + g.rz;
        pz -= (pz >= g.nz) ? g.nz : 0;
        s.hits[base + pz] = 0u;
        s.passes[base + pz] = 0u;
        s.minz[base + pz] = __int_as_float(0x7f800000);
    }
}

}  // namespace

cudaError_t launch_init_state(const MapState& s, long long V, cudaStream_t st) {
    const int block = 256;
    long long blocks = (V + block - 1) / block;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    count_launch();
    k_init_state<<<(unsigned)blocks, block, 0, st>>>(s.hits, s.passes, s.minz, V);
    return cudaGetLastError();
}

cudaError_t launch_shift(const MapState& s, const Geom& g_new, const long long d[3], cudaStream_t st) {
    const long long cols = (long long)g_new.nx * g_new.ny;
    const int block = 256;
    const long long blocks = (cols * 32 + block - 1) / block;
    count_launch();
    k_shift<<<(unsigned)blocks, block, 0, st>>>(s, g_new, (int)d[0], (int)d[1], (int)d[2]);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const long long blocks = (a.n + kIngestBlock - 1) / kIngestBlock;
    count_launch();
    k_ingest<<<(unsigned)blocks, kIngestBlock, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gvom
