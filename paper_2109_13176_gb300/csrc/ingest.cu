// Per-scan ingest (G-VOM Sec. III-C, combined per Sec. III-D) and window
// shift (Sec. III-A origin, Sec. III-D index offset) for sm_103a.
//
// The ingest runs in two phases so that every warp does a similar amount
// of traversal work (a ray crosses anywhere from one to several hundred
// voxels, and one thread per ray leaves the GPU idle behind the longest):
//
//  k_rays   one thread per lidar point: FP64 transform as a fixed chain
//           of fused multiply-adds per row (see xform_row), filter,
//           quantisation to 1/256 voxel, the hit and
//           lowest-return update of the endpoint voxel, and the split of
//           the ray's in-window traversal into segments of at most
//           seg_len voxel slabs along its major axis, appended to a work
//           list in segment-major order per warp of rays.
//  k_march  a persistent grid walks the segments. Each segment's first
//           voxel is computed exactly from the rational time at which the
//           major axis enters it, then the exact integer traversal runs to
//           the segment's end and counts one pass per window voxel. Runs
//           of neighbouring lanes that stand in the same voxel at the same
//           step merge their increments (one shuffle and one ballot), so
//           neighbouring rays near the sensor cost one L2 atomic per run.
//
// Counts are order-free sums, so the result is bit-identical to walking
// every ray whole in one thread.
#include "gvom_internal.h"
#include "exact_convert.cuh"
#include "device_sync.cuh"

namespace gvom {

namespace {

constexpr int kRaysBlock = 256;

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

__device__ __forceinline__ int dim_of(const Geom& g, int axis) { return axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz); }

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

// Sec. III-C transform, one row of [R | t]:
// fma(r2, pz, fma(r1, py, fma(r0, px, t))), each fused multiply-add
// rounded once, in this order.
__device__ __forceinline__ double xform_row(const double* T, double px, double py, double pz) {
    return __fma_rn(T[2], pz, __fma_rn(T[1], py, __fma_rn(T[0], px, T[3])));
}

// Quantise a map-frame coordinate to 1/256 voxel from the window origin:
// q = round-half-even(fma(w, S, -256 origin)) with S = 256 (1 / res),
// valid iff |fma(...)| < 2^30. The bound is tested on the exponent bits
// (|s| < 2^30 iff the high word of |s| is below that of 2^30; NaN and
// infinities fail), so no FP64 compare is issued.
__device__ __forceinline__ bool quantise(double w, double S, double neg_o256, int* q) {
    const double s = __fma_rn(w, S, neg_o256);
    if (((unsigned)__double2hiint(s) & 0x7fffffffu) >= 0x41d00000u) return false;
    *q = d2i_rne(s);  // round half to even, on the integer pipe
    return true;
}

// The range filter 0 < r2 <= r2max with r2 = fma(pz, pz, fma(py, py, px px))
// in FP64 (the oracle's). r2 > 0 iff some component is non-zero (squares of
// floats cannot underflow in FP64). The FP32 sum of squares decides unless
// it lies within a relative 2^-20 of r2max (FP32 error <= 3 * 2^-24), where
// the FP64 value decides.
__device__ __forceinline__ bool in_range(float fx, float fy, float fz, float r2max_lo, float r2max_hi, double r2max) {
    if (fx == 0.0f && fy == 0.0f && fz == 0.0f) return false;
    const float r2f = __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
    if (r2f < r2max_lo) return true;
    if (r2f > r2max_hi) return false;
    const double px = fx, py = fy, pz = fz;
    const double r2 = __fma_rn(pz, pz, __fma_rn(py, py, __dmul_rn(px, px)));
    return r2 <= r2max;
}

// The sensor's quantised position, computed once per block and shared.
// Returns false (for every thread) when it cannot be quantised.
__device__ __forceinline__ bool block_sensor(const IngestArgs& a, int qo[3]) {
    __shared__ int s_q[4];
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int k = 0; k < 3; ++k) ok &= quantise(a.T[4 * k + 3], a.S, a.neg_o256[k], &s_q[k]);
        s_q[3] = ok;
    }
    __syncthreads();
    qo[0] = s_q[0];
    qo[1] = s_q[1];
    qo[2] = s_q[2];
    return s_q[3] != 0;
}

__device__ __forceinline__ int iabs(int v) { return v < 0 ? -v : v; }

// v[k] for a run-time k without indexing a local array (keeps v in registers).
template <typename T>
__device__ __forceinline__ T sel3(const T v[3], int k) {
    return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
}

// A ray from sensor a to endpoint b (1/256-voxel units): its major axis M
// (largest |d|, lowest index on ties), the number K of major-axis voxel
// steps from start to end, and the range [klo, khi] of steps k whose major
// slab (c0 + dir k) lies in the window.
struct RayFrame {
    int a[3], b[3], d[3];
    int M;
    int K;
    int klo, khi;
};

// False when no voxel of the ray but possibly its endpoint voxel can be in
// the window: zero extent, an unmoving axis outside the window, or no major
// slab inside it.
__device__ __forceinline__ bool ray_frame(const Geom& g, const int a[3], const int b[3], RayFrame& f) {
    int best = -1;
    f.M = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f.a[k] = a[k];
        f.b[k] = b[k];
        f.d[k] = b[k] - a[k];
        const int ad = iabs(f.d[k]);
        if (ad > best) {
            best = ad;
            f.M = k;
        }
    }
    if (best == 0) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (f.d[k] == 0 && (unsigned)(a[k] >> 8) >= (unsigned)dim_of(g, k)) return false;
    const int M = f.M;
    const int c0 = sel3(a, M) >> 8, ce = sel3(b, M) >> 8, n = dim_of(g, M);
    if (sel3(f.d, M) > 0) {
        f.K = ce - c0;
        f.klo = max(0, -c0);
        f.khi = min(f.K, n - 1 - c0);
    } else {
        f.K = c0 - ce;
        f.klo = max(0, c0 - (n - 1));
        f.khi = min(f.K, c0);
    }
    return f.khi >= f.klo;
}

// One point (index i < a.n): load, filter, FP64 transform and quantisation
// to 1/256 voxel (Sec. III-C). True iff the ray is kept; then q holds the
// endpoint and wz its height as a float.
__device__ __forceinline__ bool point_ray(const IngestArgs& a, long long i, bool sensor_ok, int q[3], float& wz) {
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
    const float r2max_f = (float)a.r2max;
    if (!(isfinite(fx) && isfinite(fy) && isfinite(fz) && sensor_ok &&
          in_range(fx, fy, fz, r2max_f * (1.0f - 9.5367432e-7f), r2max_f * (1.0f + 9.5367432e-7f), a.r2max)))
        return false;
    // exact widening and narrowing on the integer pipe (see exact_convert.cuh)
    const double px = f2d_exact(fx), py = f2d_exact(fy), pz = f2d_exact(fz);
    const double wx = xform_row(a.T + 0, px, py, pz);
    const double wy = xform_row(a.T + 4, px, py, pz);
    const double wzd = xform_row(a.T + 8, px, py, pz);
    const bool valid = quantise(wx, a.S, a.neg_o256[0], &q[0]) && quantise(wy, a.S, a.neg_o256[1], &q[1]) &&
                       quantise(wzd, a.S, a.neg_o256[2], &q[2]);
    wz = d2f_rne(wzd);
    return valid;
}

// The endpoint voxel of a kept ray, if it is in the window: a hit and the
// lowest return (Sec. III-A), in the map and in its ring slot. Returns 1 for
// an in-window hit.
__device__ __forceinline__ int apply_hit(const IngestArgs& a, const int q[3], float wz) {
    const Geom& g = a.g;
    const int ex = q[0] >> 8, ey = q[1] >> 8, ez = q[2] >> 8;
    if (!in_window(g, ex, ey, ez)) return 0;
    const uint32_t k = phys_index(g, ex, ey, ez);
    if (in_bounds(k, a.s.V, a.s.counters)) {
        atomicAdd(a.s.hits + k, 1u);
        atomic_min_f32(a.s.minz + k, wz);
    }
    if (a.slot >= 0) {
        const size_t o = (size_t)a.slot * a.s.V + k;
        if (in_bounds(o, (unsigned long long)a.s.ring_K * a.s.V, a.s.counters)) {
            atomicAdd(a.s.ring_hits + o, 1u);
            atomic_min_f32(a.s.ring_minz + o, wz);
        }
    }
    return 1;
}

// Traversal segments of a kept ray from sensor qo to endpoint q.
__device__ __forceinline__ int segments_of(const IngestArgs& a, const int qo[3], const int q[3]) {
    RayFrame f;
    return ray_frame(a.g, qo, q, f) ? (f.khi - f.klo) / a.seg_len + 1 : 0;
}

// Phase 1: points -> hits, lowest returns, ray records and segment list.
// Called by every thread of a block, for points i = first + threadIdx.x of
// one map (map_id) whose ray records start at ray_base in the scratch.
__device__ __forceinline__ void rays_body(const IngestArgs& a, long long first, const int qo[3], bool sensor_ok,
                                          long long ray_base, unsigned int map_id) {
    const long long i = first + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    int q[3] = {0, 0, 0};
    float wz = 0.0f;
    const bool valid = i < a.n && point_ray(a, i, sensor_ok, q, wz);
    const int nseg = valid ? segments_of(a, qo, q) : 0;
    if (i < a.n && in_bounds(ray_base + i, a.w.cap_points, a.s.counters))
        a.w.rays[ray_base + i] = make_int4(q[0], q[1], q[2], (int)((map_id << 16) | (unsigned)nseg));

    // Reserve this block's slots in the work list with one atomic, then lay
    // each warp's segments out segment-major (all first segments of the
    // warp's rays, then all second segments, ...), so that the lanes that
    // later walk neighbouring items walk neighbouring rays at similar range.
    // Every segment but a ray's last spans seg_len major slabs; the last ones
    // (the ray's end or its exit from the window) vary, so they follow the
    // full ones as one group: a warp of the walk then holds segments of
    // similar length, and fewer of its lanes wait for the longest.
    __shared__ unsigned int warp_tot[kRaysBlock / 32];
    __shared__ unsigned long long block_base;
    unsigned int tot = (unsigned int)nseg;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const int nfull = nseg > 0 ? nseg - 1 : 0;  // this ray's full-length segments
    const int wmax = __reduce_max_sync(0xffffffffu, (unsigned)nfull);
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int s = 0;
        for (int w = 0; w < kRaysBlock / 32; ++w) s += warp_tot[w];
        block_base = s ? atomicAdd(a.w.item_count + kListLen, (unsigned long long)s) : 0ull;
    }
    __syncthreads();
    unsigned long long off = block_base;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    const unsigned int lt = (1u << lane) - 1u;
    for (int j = 0; j < wmax; ++j) {
        const unsigned int m = __ballot_sync(0xffffffffu, nfull > j);
        if (nfull > j) {
            const unsigned long long slot = off + __popc(m & lt);
            if (slot < (unsigned long long)a.w.cap_items)
                a.w.items[slot] = make_uint2((unsigned int)(ray_base + i), (unsigned int)j);
        }
        off += __popc(m);
    }
    {
        // every ray's last segment
        const unsigned int m = __ballot_sync(0xffffffffu, nseg > 0);
        if (nseg > 0) {
            const unsigned long long slot = off + __popc(m & lt);
            if (slot < (unsigned long long)a.w.cap_items)
                a.w.items[slot] = make_uint2((unsigned int)(ray_base + i), (unsigned int)(nseg - 1));
        }
        off += __popc(m);
    }

    // Up to here only the points and this scan's scratch were touched, so
    // the work above overlaps the kernel before (the window shift). The map
    // is touched only once that kernel is complete.
    pdl_wait();
    const int hit_in_window = valid ? apply_hit(a, q, wz) : 0;

    // Counters: one atomic per block and counter.
    __shared__ unsigned long long red[2][kRaysBlock / 32];
    unsigned long long v0 = valid ? 1ull : 0ull, v1 = (unsigned long long)hit_in_window;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        red[0][warp] = v0;
        red[1][warp] = v1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned long long s = 0;
        for (int w = 0; w < kRaysBlock / 32; ++w) s += red[threadIdx.x][w];
        if (s) atomicAdd(a.s.counters + kRaysValid + threadIdx.x, s);
    }
    __syncthreads();  // the shared arrays are reused by the caller's next block
}

// Launched with programmatic dependent launch, it starts before the kernel
// ahead of it (the window shift) is complete: it reads the points and writes
// the scratch, which no kernel before it still uses (the walk and the fused
// ingest release their dependents only at their very end), and waits before
// touching the map (in rays_body).
__global__ void __launch_bounds__(kRaysBlock) k_rays(const IngestArgs a) {
    int qo[3];
    const bool sensor_ok = block_sensor(a, qo);
    rays_body(a, (long long)blockIdx.x * kRaysBlock, qo, sensor_ok, 0, 0u);
    pdl_done();
}

// Phase 2: walk the segments.
//
// Roles: M is the ray's major axis, A and B the other two (in x, y, z
// order after M). For each axis the next voxel boundary is crossed at
// t = num / den along the segment (den = |d|, num measured from the ray's
// start). Axis i's next crossing comes first iff num_i den_j < num_j den_i,
// so the walk keeps the three pairwise differences D_ij = num_i den_j -
// num_j den_i and updates them as axes step (num grows by 256). Both next
// crossings lie within one voxel of the current point along the ray, which
// bounds |D_ij| by 256 max(den) < 2^31, so they fit 32-bit integers.
// An axis that does not move gets a crossing at t = 2 (num 2, den 1),
// beyond the ray's end, so it never steps; likewise the crossings an axis
// would make past the endpoint come after every real one. The walk
// therefore needs only the count of crossings left to the endpoint.
//
// Ties (Sec. III-A half-open voxels): an upward crossing takes effect at
// its t, a downward one just after it. Ordering crossings by (t, down after
// up), all axes sharing the earliest key step together.
//
// A segment that starts at major step k > 0 begins in the first voxel whose
// major coordinate is the new slab. At that instant t* = numStar / denM a
// minor axis stands at P = a + t* d; its voxel is floor(P / 256), except
// when both it and the major axis move down: then the major step (taken
// just after t*) comes with the minor's own crossing at t*, if any, so the
// voxel is ceil(P / 256) - 1.

// q = floor(x / y) for 0 < y < 2^31 and |x / y| < 2^23: an FP32 estimate
// (reciprocal-based, a few units off at most) corrected exactly with 64-bit
// integer remainders.
__device__ __forceinline__ long long floor_div_small(long long x, long long y) {
    // x converted from its two 32-bit halves (FP32 pipe, not the FP64 one)
    const float xf = fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned int)x);
    long long q = (long long)floorf(__fdividef(xf, (float)(int)y));
    long long r = x - q * y;
    while (r < 0) {
        q -= 1;
        r += y;
    }
    while (r >= y) {
        q += 1;
        r -= y;
    }
    return q;
}

// The crossing of an axis at t = num / den (its ordering rank: 0 for an
// upward crossing, which takes effect at t, 1 for a downward one, which
// takes effect just after t). Within one ray num <= |d| + 256 < 2^24 and
// den = |d| < 2^23 (1/256-voxel units), so both fit 32 bits and their
// products 64.
struct Crossing {
    int num, den;
    int rank;
};

// Whether crossing x comes before crossing y in the walk's order (t, then
// upward before downward). Exact.
__device__ __forceinline__ bool cross_before(const Crossing& x, const Crossing& y) {
    const long long l = (long long)x.num * y.den, r = (long long)y.num * x.den;
    return l < r || (l == r && x.rank < y.rank);
}

// How many of an axis's crossings -- the next one at num / den, then one
// every 256 / den, `tot` in all, rank rk -- come no later than crossing e
// in the walk's order (the crossings sharing e's time and rank included).
__device__ __forceinline__ int crossings_upto(int num, int den, int tot, int rk, const Crossing& e) {
    if (tot <= 0) return 0;
    // crossing k (k = 0, 1, ...) comes no later than e iff 256 k den_e <= X,
    // strictly below X when it would step after e at an equal time
    const long long X = (long long)e.num * den - (long long)num * e.den;
    const long long Y = 256LL * e.den;
    long long c;
    if (rk <= e.rank)
        c = X < 0 ? 0 : floor_div_small(X, Y) + 1;
    else
        c = X <= 0 ? 0 : floor_div_small(X - 1, Y) + 1;
    return (int)(c < (long long)tot ? c : (long long)tot);
}

// The walk of one segment, from its first voxel in the window. rem counts
// the crossings still to take: the walk visits its current voxel, takes the
// next crossing group and stops when rem reaches zero, which happens exactly
// on the group that leaves the segment's last major slab, leaves the window
// along a minor axis, or enters the ray's endpoint voxel (whichever comes
// first). Every voxel it visits is therefore in the window and not the
// endpoint voxel: the loop needs no window, exit or endpoint test.
struct Walk {
    int cM, cA, cB;     // current voxel, window coordinates (the index of non-power-of-two windows)
    int dirM, dirA, dirB;
    int nM, nA, nB;     // window extents
    int sM, sA, sB;     // 256 den per axis
    int nsM, nsA;       // -sM, -sA
    // Pairwise crossing-time differences D_ij, biased: x_ij = D_ij + t_ji - 1
    // is >= 0 iff j's crossing comes first, and x_ij + c_ij = D_ij - t_ij is
    // < 0 iff i's comes first (t_ij = 1 iff i moves up and j down, the
    // tie-break; c_ij = 1 - t_ij - t_ji is 0 or 1). The step reads the
    // decisions off sign bits.
    int xMA, xMB, xAB;
    int cMA, cMB, cAB;
    int rem;            // crossings left to take
    int rM, rA, rB;     // ring offsets
    uint32_t kM, kA, kB;  // strides of the state array per role
    // Windows whose extents are all powers of two: the physical index of the
    // current voxel is kept up to date instead of being recomputed. Axis k
    // owns the bit field fm_k of the index (its extent's bits, at its
    // stride), so a unit step is an add of st_k = +-stride_k kept within
    // the field: the field wraps modulo the extent, which is exactly the
    // toroidal addressing, and the other fields are untouched.
    uint32_t key;
    uint32_t fmM, fmA, fmB;
    uint32_t stM, stA, stB;
};

__device__ __forceinline__ int rank_of(int dir) { return dir > 0 ? 0 : 1; }

// a * b + c as an integer multiply-add. The walk's step is bound by the
// integer ALU pipe while the FMA pipe (which executes integer multiply-adds)
// idles, so the step's conditional updates are written as products with the
// 0/1 step flags.
__device__ __forceinline__ int imad_s32(int a, int b, int c) {
    int d;
    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t imad_u32(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Builds the walk of segment j of the ray to endpoint b. False if the
// segment has no voxel to count in the window.
__device__ __forceinline__ bool walk_init(const IngestArgs& a, const int qo[3], const int b[3], int j, Walk& w) {
    const Geom& g = a.g;
    RayFrame f;
    if (!ray_frame(g, qo, b, f)) return false;
    const int M = f.M, A = M == 0 ? 1 : 0, B = M == 2 ? 1 : 2;
    const int kstart = f.klo + j * a.seg_len;
    const int kend = min(f.khi, kstart + a.seg_len - 1);
    const int segM = kend - kstart;  // major steps from the first slab to the last

    const int aM = sel3(f.a, M), dM = sel3(f.d, M);
    const int dirM = dM > 0 ? 1 : -1;
    const long long denM = dM > 0 ? dM : -dM;
    const int c0M = aM >> 8;
    const long long numFirst = dirM > 0 ? 256LL * (c0M + 1) - aM : (long long)aM - 256LL * c0M;
    const long long numStar = numFirst + 256LL * (kstart - 1);

    // the segment's first voxel, and per role its next crossing (num / den),
    // direction, rank and the number of crossings left to the endpoint
    int c[3], dir[3], tot[3], rk[3];
    int num[3], den[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int k = r == 0 ? M : (r == 1 ? A : B);
        const int ak = sel3(f.a, k), dk = sel3(f.d, k), ce = sel3(f.b, k) >> 8;
        int ck;
        if (r == 0) {
            ck = c0M + dirM * kstart;
        } else if (kstart == 0 || dk == 0) {
            ck = ak >> 8;
        } else {
            // position at numStar / denM, in 1/256 voxel, times denM
            const long long X = (long long)ak * denM + numStar * (long long)dk;
            const long long Y = 256LL * denM;
            ck = (int)((dirM < 0 && dk < 0) ? -floor_div_small(-X, Y) - 1 : floor_div_small(X, Y));
        }
        c[r] = ck;
        if (dk != 0) {
            dir[r] = dk > 0 ? 1 : -1;
            den[r] = dk > 0 ? dk : -dk;
            num[r] = dk > 0 ? 256 * (ck + 1) - ak : ak - 256 * ck;
            tot[r] = dk > 0 ? ce - ck : ck - ce;
        } else {
            dir[r] = 1;
            den[r] = 1;
            num[r] = 2;
            tot[r] = 0;
        }
        rk[r] = rank_of(dir[r]);
    }
    const int n3[3] = {dim_of(g, M), dim_of(g, A), dim_of(g, B)};
    // a minor axis already past the window has nothing left to count
    if ((dir[1] > 0 ? c[1] >= n3[1] : c[1] < 0) || (dir[2] > 0 ? c[2] >= n3[2] : c[2] < 0)) return false;

    // The end E: the earliest of the crossing out of the segment's last
    // major slab, the crossing out of the window along A or B, and the ray's
    // last crossing (into the endpoint voxel).
    Crossing E = {0, 1, 0}, last = {0, 1, 0};
    bool have_e = false, have_last = false;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        if (tot[r] > 0) {
            const Crossing x = {num[r] + 256 * (tot[r] - 1), den[r], rk[r]};
            if (!have_last || cross_before(last, x)) last = x;
            have_last = true;
        }
    if (!have_last) return false;  // the segment starts in the endpoint voxel
    E = last;
    have_e = true;
    if (segM + 1 <= tot[0]) {
        const Crossing x = {num[0] + 256 * segM, den[0], rk[0]};
        if (cross_before(x, E)) E = x;
    }
#pragma unroll
    for (int r = 1; r < 3; ++r) {
        const int exit_v = dir[r] > 0 ? n3[r] : -1;
        const int n = dir[r] > 0 ? exit_v - c[r] : c[r] - exit_v;
        if (n >= 1 && n <= tot[r]) {
            const Crossing x = {num[r] + 256 * (n - 1), den[r], rk[r]};
            if (cross_before(x, E)) E = x;
        }
    }
    (void)have_e;

    // The start S: when the segment begins before the window along A or B,
    // the later of the crossings into it.
    Crossing S = {0, 1, 0};
    bool have_s = false;
#pragma unroll
    for (int r = 1; r < 3; ++r) {
        const bool before = dir[r] > 0 ? c[r] < 0 : c[r] >= n3[r];
        if (!before) continue;
        const int n = dir[r] > 0 ? -c[r] : c[r] - (n3[r] - 1);
        if (n > tot[r]) return false;  // the ray ends before it enters
        const Crossing x = {num[r] + 256 * (n - 1), den[r], rk[r]};
        if (!have_s || cross_before(S, x)) S = x;
        have_s = true;
    }
    int rem = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int ce_r = crossings_upto(num[r], den[r], tot[r], rk[r], E);
        int cs_r = 0;
        if (have_s) {
            cs_r = crossings_upto(num[r], den[r], tot[r], rk[r], S);
            // move past S's group: its voxel is the first in the window
            c[r] += dir[r] * cs_r;
            num[r] += 256 * cs_r;
        }
        rem += ce_r - cs_r;
    }
    if (rem <= 0) return false;  // the window is left (or the segment ends) before it is entered

    w.cM = c[0];
    w.cA = c[1];
    w.cB = c[2];
    w.dirM = dir[0];
    w.dirA = dir[1];
    w.dirB = dir[2];
    w.sM = 256 * den[0];
    w.sA = 256 * den[1];
    w.sB = 256 * den[2];
    w.nsM = -w.sM;
    w.nsA = -w.sA;
    const int dMA = (int)((long long)num[0] * den[1] - (long long)num[1] * den[0]);
    const int dMB = (int)((long long)num[0] * den[2] - (long long)num[2] * den[0]);
    const int dAB = (int)((long long)num[1] * den[2] - (long long)num[2] * den[1]);
    // i first on equal t iff i moves up and j down: D_ij < t_ij with
    // t_ij = 1 then, else 0; j first iff D_ij > -t_ji.
    const int tMA = rk[0] < rk[1], tAM = rk[1] < rk[0];
    const int tMB = rk[0] < rk[2], tBM = rk[2] < rk[0];
    const int tAB = rk[1] < rk[2], tBA = rk[2] < rk[1];
    // |D_ij| <= 256 max(den) < 2^31, so the biased forms stay within int32
    w.xMA = dMA + tAM - 1;
    w.xMB = dMB + tBM - 1;
    w.xAB = dAB + tBA - 1;
    w.cMA = 1 - tMA - tAM;
    w.cMB = 1 - tMB - tBM;
    w.cAB = 1 - tAB - tBA;
    w.rem = rem;
    w.nM = n3[0];
    w.nA = n3[1];
    w.nB = n3[2];
    const int rr[3] = {g.rx, g.ry, g.rz};
    const uint32_t st[3] = {(uint32_t)g.ny * (uint32_t)g.nz, (uint32_t)g.nz, 1u};
    w.rM = sel3(rr, M);
    w.rA = sel3(rr, A);
    w.rB = sel3(rr, B);
    w.kM = sel3(st, M);
    w.kA = sel3(st, A);
    w.kB = sel3(st, B);
    // power-of-two windows: the index fields of the first voxel (in the window)
    const uint32_t fm[3] = {((uint32_t)g.nx - 1u) * st[0], ((uint32_t)g.ny - 1u) * st[1], (uint32_t)g.nz - 1u};
    w.fmM = sel3(fm, M);
    w.fmA = sel3(fm, A);
    w.fmB = sel3(fm, B);
    w.stM = w.dirM > 0 ? w.kM : 0u - w.kM;
    w.stA = w.dirA > 0 ? w.kA : 0u - w.kA;
    w.stB = w.dirB > 0 ? w.kB : 0u - w.kB;
    w.key = (((uint32_t)(w.cM + w.rM) * w.kM) & w.fmM) | (((uint32_t)(w.cA + w.rA) * w.kA) & w.fmA) |
            (((uint32_t)(w.cB + w.rB) * w.kB) & w.fmB);
    return true;
}

__device__ __forceinline__ uint32_t walk_index(const Walk& w) {
    int pM = w.cM + w.rM;
    pM -= pM >= w.nM ? w.nM : 0;
    int pA = w.cA + w.rA;
    pA -= pA >= w.nA ? w.nA : 0;
    int pB = w.cB + w.rB;
    pB -= pB >= w.nB ? w.nB : 0;
    return (uint32_t)pM * w.kM + (uint32_t)pA * w.kA + (uint32_t)pB * w.kB;
}

// kBatch = false: one map, whose arguments are a1. kBatch = true: many maps;
// a1 carries only the shared scratch (work list and ray records), each ray
// record names its map, and descs / sensors hold each map's arguments and
// quantised sensor position. Pass increments of lanes of different maps
// never merge: lanes compare the full address.
//
// kSlot: some ray's scan also goes to a ring slot of its map's scan buffer;
// lanes then merge only within one slot.
// Adds each lane's pending visits to the counters of entry `own` (the map's
// own when descs is null): one atomic per warp when every lane holds the
// same entry, else one per lane. All lanes call it.
__device__ __forceinline__ void flush_visits(const IngestArgs& a1, const IngestArgs* descs, unsigned int own,
                                             unsigned long long& visits) {
    int same = 0;
    __match_all_sync(0xffffffffu, own, &same);
    unsigned long long* cnt = own == 0xffffffffu ? nullptr : (descs ? descs[own].s.counters : a1.s.counters);
    if (same) {
        unsigned long long v = visits;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && cnt && v) atomicAdd(cnt + kPassVisits, v);
    } else if (cnt && visits) {
        atomicAdd(cnt + kPassVisits, visits);
    }
    visits = 0;
}

// One step of the walk for every lane of the warp (all lanes call it): a
// live lane visits its current voxel (in the window by construction) and
// takes the next crossing group; the segment's crossing budget ends its walk
// (live turns false). The step is branch-free: a lane that is not live keeps
// stepping its (no longer read) state. item_n counts this lane's visits.
template <bool kBatch, bool kSlot, bool kPow2>
__device__ __forceinline__ void walk_step(Walk& w, bool& live, int lane, uint32_t* passes, uint32_t* spasses,
                                          uint32_t vmap, unsigned long long* cnts, unsigned int& item_n) {
    // On power-of-two windows the masked index cannot leave the map; on
    // others the index is only formed for a voxel inside the window, so no
    // access can leave the state arrays whatever the walk computes.
    const bool visit = kPow2 ? live
                             : live && (unsigned)w.cM < (unsigned)w.nM && (unsigned)w.cA < (unsigned)w.nA &&
                                   (unsigned)w.cB < (unsigned)w.nB;
    const uint32_t key = visit ? (kPow2 ? w.key : walk_index(w)) : 0xffffffffu;
    // runs of neighbouring lanes in the same voxel merge their increments:
    // the run's first lane adds the run's length
    bool boundary;
    if (kBatch) {
        const unsigned long long kk =
            visit ? (unsigned long long)((kSlot && spasses) ? spasses + key : passes + key) : 0ull;
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, kk, 1);  // every lane
        boundary = lane == 0 || prev != kk;
    } else {
        const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);  // every lane
        boundary = lane == 0 || prev != key;
    }
    const unsigned int starts = __ballot_sync(0xffffffffu, boundary);
    if (visit && boundary && in_bounds(key, vmap, cnts)) {
        const unsigned int after = starts & ~((2u << lane) - 1u);
        // the next run's first lane, or 32 past the warp's end (clz(0) = 32)
        const uint32_t run = (uint32_t)(__clz(__brev(after)) - lane);
        atomicAdd(passes + key, run);
        if (kSlot && spasses) atomicAdd(spasses + key, run);
    }
    item_n += visit ? 1u : 0u;
    // An axis steps iff no other axis's crossing comes first. y_ij = D_ij -
    // t_ij as x_ij + c_ij^2 (c_ij is 0 or 1): a multiply-add, on the FMA pipe.
    const int yMA = imad_s32(w.cMA, w.cMA, w.xMA);
    const int yMB = imad_s32(w.cMB, w.cMB, w.xMB);
    const int yAB = imad_s32(w.cAB, w.cAB, w.xAB);
    const int iM = (int)((uint32_t)(w.xMA & w.xMB) >> 31);  // neither A nor B first
    const int iA = (int)((uint32_t)(~yMA & w.xAB) >> 31);   // neither M nor B first
    const int iB = (int)((uint32_t)(~(yMB | yAB)) >> 31);   // neither M nor A first
    if (kPow2) {
        w.key = ((imad_u32((uint32_t)iM, w.stM, w.key)) & w.fmM) |
                ((imad_u32((uint32_t)iA, w.stA, w.key)) & w.fmA) |
                ((imad_u32((uint32_t)iB, w.stB, w.key)) & w.fmB);
    } else {
        w.cM = imad_s32(iM, w.dirM, w.cM);
        w.cA = imad_s32(iA, w.dirA, w.cA);
        w.cB = imad_s32(iB, w.dirB, w.cB);
    }
    w.xMA = imad_s32(iM, w.sA, imad_s32(iA, w.nsM, w.xMA));
    w.xMB = imad_s32(iM, w.sB, imad_s32(iB, w.nsM, w.xMB));
    w.xAB = imad_s32(iA, w.sB, imad_s32(iB, w.nsA, w.xAB));
    w.rem = imad_s32(iM, -1, imad_s32(iA, -1, imad_s32(iB, -1, w.rem)));
    live = live && w.rem > 0;
}

// Walks one segment per lane from its first in-window voxel until its
// crossing budget runs out (live: the lane holds a segment), adding the pass
// increments; returns the number of voxels this lane visited. All lanes of
// the warp call it.
template <bool kBatch, bool kSlot, bool kPow2>
__device__ __forceinline__ unsigned int walk_run(Walk& w, bool live, int lane, uint32_t* passes, uint32_t* spasses,
                                                 uint32_t vmap, unsigned long long* cnts) {
    unsigned int item_n = 0;
    // two steps per vote: a lane that stops after the first one takes a
    // second step that visits nothing
    while (__any_sync(0xffffffffu, live)) {
        walk_step<kBatch, kSlot, kPow2>(w, live, lane, passes, spasses, vmap, cnts, item_n);
        walk_step<kBatch, kSlot, kPow2>(w, live, lane, passes, spasses, vmap, cnts, item_n);
    }
    return item_n;
}

// kPow2: every window of the launch has power-of-two extents (the index of
// the current voxel is stepped, not recomputed).
// Resident blocks per SM the walk is compiled for (registers per thread
// = 65536 / (256 * this)): three keep its segment set-up in registers.
#ifndef GVOM_MARCH_MIN_BLOCKS
#define GVOM_MARCH_MIN_BLOCKS 3
#endif

template <bool kBatch, bool kSlot, bool kPow2>
__global__ void __launch_bounds__(256, GVOM_MARCH_MIN_BLOCKS) k_march(const IngestArgs a1, const IngestArgs* __restrict__ descs, const int4* __restrict__ sensors) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const unsigned long long total_items = a1.w.item_count[kListLen];
    const long long n_items =
        (long long)(total_items < (unsigned long long)a1.w.cap_items ? total_items : a1.w.cap_items);
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;

    int qo1[3] = {0, 0, 0};
    if (!kBatch) block_sensor(a1, qo1);  // the work list only holds rays of a quantisable sensor

    // pass visits not yet added to the counters of entry `own` (per lane;
    // in batch mode the pending entry changes only when a lane's item belongs
    // to a map with other counters, so several entries of one map add once)
    unsigned long long visits = 0;
    unsigned int own = kBatch ? 0xffffffffu : 0u;
    for (long long base = gw * 32; base < n_items; base += nwarps * 32) {
        const long long idx = base + lane;
        Walk w;
        bool live = false;
        unsigned int map = 0;
        unsigned int own_item = own;  // entry owning the counters of this lane's item's map
        uint32_t* passes = a1.s.passes;
        uint32_t* spasses = nullptr;
        uint32_t vmap = a1.s.V;  // voxels of this lane's map (range checks)
        unsigned long long* cnts = a1.s.counters;
        if (kSlot && !kBatch) spasses = a1.s.ring_passes + (size_t)a1.slot * a1.s.V;
        unsigned long long item_visits = 0;
        if (idx < n_items && in_bounds(a1.w.items[idx].x, a1.w.cap_points, a1.s.counters)) {
            const uint2 it = a1.w.items[idx];
            const int4 r = a1.w.rays[it.x];
            const int b[3] = {r.x, r.y, r.z};
            if (kBatch) {
                map = (unsigned int)r.w >> 16;
                const int4 sq = sensors[map];
                const int qo[3] = {sq.x, sq.y, sq.z};
                passes = descs[map].s.passes;
                vmap = descs[map].s.V;
                cnts = descs[map].s.counters;
                own_item = (unsigned int)descs[map].cnt_owner;
                if (kSlot) {
                    const int sl = descs[map].slot;
                    spasses = sl >= 0 ? descs[map].s.ring_passes + (size_t)sl * descs[map].s.V : nullptr;
                }
                live = walk_init(descs[map], qo, b, (int)it.y, w);
            } else {
                live = walk_init(a1, qo1, b, (int)it.y, w);
            }
        }
        const unsigned int item_n = walk_run<kBatch, kSlot, kPow2>(w, live, lane, passes, spasses, vmap, cnts);
        item_visits = item_n;
        if (kBatch && __any_sync(0xffffffffu, own_item != own)) {
            flush_visits(a1, descs, own, visits);
            own = own_item;
        }
        visits += item_visits;
    }

    flush_visits(a1, descs, own, visits);
    if (!kBatch) {
        // the last block to finish empties the work list for the next scan
        // (every thread of every block read its length at the start)
        __syncthreads();
        if (threadIdx.x == 0 && atomicAdd(a1.w.item_count + kListBlocksDone, 1ull) + 1 == gridDim.x) {
            a1.w.item_count[kListLen] = 0;
            a1.w.item_count[kListBlocksDone] = 0;
        }
    }
    // dependents are released only now: the next scan's per-point pass writes
    // the scratch before it waits
    __syncthreads();
    pdl_done();
}

// Fused ingest (tuning fused_ingest = 1): one persistent kernel whose warps
// first list segments and then walk them, so the walk starts on the first
// listed segments while other warps still list, with no launch between.
// Work is assigned statically, as in the two-kernel walk, so no warp claims
// work through a shared counter: global warp g of W lists point tiles
// g, g + W, ... (32 points each) and then walks the list's 32-entry chunks
// g, g + W, .... Entries are int4 (qx, qy, qz, tag) with tag = epoch << 12 |
// segment index; a lane polls its entry's tag, so an entry an earlier scan
// left in the list is never taken for this scan's, and a chunk past the
// list's end is recognised once every tile is listed (the listed-tiles count
// equals the tile count; the reserved count is then final).
//
// Every wait ends: a warp walks only after listing all its tiles, so the
// entries it waits for are written by warps that are listing and do not
// wait. No grid-wide residency is needed for progress; the launch is
// cooperative (at most the blocks that fit at once) all the same, and every
// wait is bounded (kStatusTimeout).

// Lists one 32-point tile (points tile * 32 + lane): hits and lowest
// returns, then the tile's segments at entries reserved with one atomic,
// written in two passes: the coordinates, a fence, then the tags that
// publish them. The count of listed tiles goes up last.
__device__ __forceinline__ void fused_list_tile(const IngestArgs& a, long long tile, const int qo[3], bool sensor_ok,
                                                int lane, unsigned int& n_valid, unsigned int& n_hit) {
    const long long i = tile * 32 + lane;
    int q[3] = {0, 0, 0};
    float wz = 0.0f;
    const bool valid = i < a.n && point_ray(a, i, sensor_ok, q, wz);
    int nseg = 0;
    if (valid) {
        n_valid += 1u;
        n_hit += (unsigned int)apply_hit(a, q, wz);
        nseg = segments_of(a, qo, q);
    }
    const unsigned int tot = __reduce_add_sync(0xffffffffu, (unsigned int)nseg);
    const int nfull = nseg > 0 ? nseg - 1 : 0;  // this ray's full-length segments
    const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned int)nfull);
    unsigned long long base = 0ull;
    if (lane == 0 && tot) base = atomicAdd(a.w.item_count + kFReserved, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 0);
    int4* const items = reinterpret_cast<int4*>(a.w.items);
    const unsigned long long cap = (unsigned long long)a.w.cap_items;
    const unsigned int lt = (1u << lane) - 1u;
    const unsigned int tag = a.epoch << 12;
    for (int pass = 0; pass < 2; ++pass) {
        unsigned long long off = base;
        for (int j = 0; j <= wmax; ++j) {  // j == wmax: every ray's last segment
            const bool last = j == wmax;
            const bool mine = last ? nseg > 0 : nfull > j;
            const unsigned int m = __ballot_sync(0xffffffffu, mine);
            const unsigned long long slot = off + __popc(m & lt);
            if (mine && slot < cap) {
                if (pass == 0) {
                    items[slot] = make_int4(q[0], q[1], q[2], 0);
                } else {
                    const unsigned int seg = last ? (unsigned int)(nseg - 1) : (unsigned int)j;
                    st_relaxed_gpu(reinterpret_cast<uint32_t*>(items + slot) + 3, tag | seg);
                }
            }
            off += __popc(m);
        }
        // the coordinates (and lane 0's reservation) before any tag, and
        // before the count of listed tiles
        if (pass == 0) __threadfence();
    }
    __syncwarp();
    if (lane == 0) atomicAdd(a.w.item_count + kFTilesDone, 1ull);
}

// The list's state as one warp sees it: lane 0 reads the listed-tiles count
// (acquire) and then the reserved count, and shares both. Once every tile is
// listed the reserved count read after it is the list's final length.
__device__ __forceinline__ void fused_list_state(const IngestArgs& a, long long ntiles, int lane, bool& final,
                                                 unsigned long long& end) {
    unsigned long long e = 0ull;
    int f = 0;
    if (lane == 0) {
        f = ld_acquire_gpu(a.w.item_count + kFTilesDone) == (unsigned long long)ntiles;
        e = ld_relaxed_gpu(a.w.item_count + kFReserved);
    }
    final = __shfl_sync(0xffffffffu, f, 0) != 0;
    end = __shfl_sync(0xffffffffu, e, 0);
    if ((unsigned long long)a.w.cap_items < end) end = (unsigned long long)a.w.cap_items;
}

template <bool kPow2>
__global__ void __launch_bounds__(256, GVOM_MARCH_MIN_BLOCKS) k_ingest_fused(const IngestArgs a) {
    pdl_wait();
    int qo[3];
    const bool sensor_ok = block_sensor(a, qo);  // every thread, before the warps part
    const int lane = threadIdx.x & 31;
    const long long ntiles = (a.n + 31) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int4* const items = reinterpret_cast<const int4*>(a.w.items);

    // 1. this warp's point tiles
    unsigned int n_valid = 0, n_hit = 0;  // kept points, in-window hits of this lane's points
    for (long long t = gw; t < ntiles; t += nwarps) fused_list_tile(a, t, qo, sensor_ok, lane, n_valid, n_hit);

    // 2. this warp's chunks of the list
    unsigned long long visits = 0;  // pass visits of this lane's walks
    unsigned long long end = 0;     // entries known to be reserved (warp-uniform)
    bool final = false;             // end is the list's final length (warp-uniform)
    bool gave_up = false;
    for (unsigned long long c = (unsigned long long)gw * 32;; c += (unsigned long long)nwarps * 32) {
        // until the chunk starts inside the list, or the list is final
        for (unsigned int idle = 0; !(c < end) && !final;) {
            fused_list_state(a, ntiles, lane, final, end);
            if (c < end || final) break;
            if (++idle > kSpinLimit) {
                gave_up = true;
                break;
            }
            __nanosleep(idle < 8 ? 128u : 1024u);
        }
        if (gave_up || !(c < end)) break;  // past the final list's end
        // this lane's entry: wait for its tag (it is written by a warp still
        // listing), or learn that it is past the final list's end
        const unsigned long long idx = c + lane;
        bool have = false, entry = false;
        int4 it = make_int4(0, 0, 0, 0);
        for (unsigned int idle = 0;;) {
            if (!have) {
                if (final && idx >= end) {
                    have = true;
                } else if (idx < end) {
                    const unsigned int t = ld_acquire_gpu(reinterpret_cast<const uint32_t*>(items + idx) + 3);
                    if ((t >> 12) == a.epoch) {
                        it = __ldcg(items + idx);
                        it.w = (int)(t & 0xfffu);
                        have = entry = true;
                    }
                }
            }
            if (__all_sync(0xffffffffu, have)) break;
            if (++idle > kSpinLimit) {
                gave_up = true;
                break;
            }
            __nanosleep(64);
            if ((idle & 7u) == 0u) fused_list_state(a, ntiles, lane, final, end);
        }
        if (gave_up) break;
        Walk w;
        bool live = false;
        if (entry) {
            const int b[3] = {it.x, it.y, it.z};
            live = walk_init(a, qo, b, it.w, w);
        }
        visits += walk_run<false, false, kPow2>(w, live, lane, a.s.passes, nullptr, a.s.V, a.s.counters);
    }
    // a wait that ran out: recorded, and this warp's remaining chunks stay
    // unwalked (no warp waits on a walking warp)
    if (gave_up && lane == 0) atomicOr(a.s.counters + kStatus, kStatusTimeout);

    flush_visits(a, nullptr, 0u, visits);
    const unsigned int tv = __reduce_add_sync(0xffffffffu, n_valid);
    const unsigned int th = __reduce_add_sync(0xffffffffu, n_hit);
    if (lane == 0) {
        if (tv) atomicAdd(a.s.counters + kRaysValid, (unsigned long long)tv);
        if (th) atomicAdd(a.s.counters + kHitsInWindow, (unsigned long long)th);
    }
    // the last block to finish leaves the list's words at zero for the next
    // scan (every warp of every block is past its last use of them)
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* const ctr = a.w.item_count;
        __threadfence();
        if (atomicAdd(ctr + kFBlocksDone, 1ull) + 1 == gridDim.x) {
            ctr[kFReserved] = 0;
            ctr[kFTilesDone] = 0;
            ctr[kFBlocksDone] = 0;
        }
    }
    // dependents are released only now (see k_march)
    __syncthreads();
    pdl_done();
}

// Empties the ring slots of `mask` at voxel i: their counts leave the
// combined state, and where an emptied slot held the combined lowest
// return, that becomes the minimum over the slots that stay (+inf if none).
__device__ __forceinline__ void evict_voxel(const MapState& s, unsigned long long mask, uint32_t i) {
    if (!in_bounds(i, s.V, s.counters)) return;
    uint32_t h = 0u, p = 0u;
    bool gone = false;
    for (int j = 0; j < s.ring_K; ++j) {
        if (!((mask >> j) & 1ull)) continue;
        const size_t o = (size_t)j * s.V + i;
        const uint32_t hj = s.ring_hits[o], pj = s.ring_passes[o];
        if ((hj | pj) == 0u) continue;
        h += hj;
        p += pj;
        s.ring_hits[o] = 0u;
        s.ring_passes[o] = 0u;
        if (hj) {
            const float mz = s.ring_minz[o];
            s.ring_minz[o] = __int_as_float(0x7f800000);
            gone |= mz == s.minz[i];
        }
    }
    if ((h | p) != 0u) {
        s.hits[i] -= h;
        s.passes[i] -= p;
    }
    if (gone) {
        float m = __int_as_float(0x7f800000);
        for (int j = 0; j < s.ring_K; ++j)
            if (!((mask >> j) & 1ull)) m = fminf(m, s.ring_minz[(size_t)j * s.V + i]);
        s.minz[i] = m;
    }
}

// Four consecutive voxels from i (a multiple of 4, V % 4 == 0): one 16-byte
// load per array and slot finds the common case, four voxels that no
// emptied slot touched.
__device__ __forceinline__ void evict_quad(const MapState& s, unsigned long long mask, uint32_t i) {
    if (!in_bounds(i + 3ull, s.V, s.counters)) return;
    if ((mask & (mask - 1ull)) == 0ull) {
        // one slot (every scan of the plain and batched paths): the counts of
        // the four voxels leave the map with 16-byte loads and stores
        const int j = __ffsll((long long)mask) - 1;
        const size_t o = (size_t)j * s.V + i;
        uint4* sh = reinterpret_cast<uint4*>(s.ring_hits + o);
        uint4* sp = reinterpret_cast<uint4*>(s.ring_passes + o);
        const uint4 h = *sh, p = *sp;
        if ((h.x | h.y | h.z | h.w | p.x | p.y | p.z | p.w) == 0u) return;
        uint4* mh = reinterpret_cast<uint4*>(s.hits + i);
        uint4* mp = reinterpret_cast<uint4*>(s.passes + i);
        uint4 ah = *mh, ap = *mp;
        ah.x -= h.x; ah.y -= h.y; ah.z -= h.z; ah.w -= h.w;
        ap.x -= p.x; ap.y -= p.y; ap.z -= p.z; ap.w -= p.w;
        *mh = ah;
        *mp = ap;
        *sh = make_uint4(0u, 0u, 0u, 0u);
        *sp = make_uint4(0u, 0u, 0u, 0u);
        if ((h.x | h.y | h.z | h.w) == 0u) return;
        const uint32_t hs[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (hs[e] == 0u) continue;
            const float mz = s.ring_minz[o + e];
            s.ring_minz[o + e] = __int_as_float(0x7f800000);
            if (mz == s.minz[i + e]) {
                float m = __int_as_float(0x7f800000);
                for (int k = 0; k < s.ring_K; ++k)
                    if (k != j) m = fminf(m, s.ring_minz[(size_t)k * s.V + i + e]);
                s.minz[i + e] = m;
            }
        }
        return;
    }
    uint32_t any = 0u;
    for (int j = 0; j < s.ring_K; ++j) {
        if (!((mask >> j) & 1ull)) continue;
        const size_t o = (size_t)j * s.V + i;
        const uint4 h = *reinterpret_cast<const uint4*>(s.ring_hits + o);
        const uint4 p = *reinterpret_cast<const uint4*>(s.ring_passes + o);
        any |= h.x | h.y | h.z | h.w | p.x | p.y | p.z | p.w;
    }
    if (any == 0u) return;
#pragma unroll
    for (int e = 0; e < 4; ++e) evict_voxel(s, mask, i + e);
}

__global__ void __launch_bounds__(256) k_evict(MapState s, unsigned long long mask) {
    pdl_wait();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if ((s.V & 3u) == 0u) {
        if (4u * t < s.V) evict_quad(s, mask, 4u * t);
    } else if (t < s.V) {
        evict_voxel(s, mask, t);
    }
    pdl_done();
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

// Clear the voxels that enter the window on a shift by d = new - old origin
// (|d_k| < n_k on every axis); g is the new window. The entering voxels are
// the union of an x slab (|dx| whole columns deep), a y slab (the remaining
// columns, |dy| deep) and a z slab (|dz| voxels of every remaining column).
// k_shift_columns clears them in one launch: whole columns one warp each,
// the z slab one column per lane.
__device__ __forceinline__ uint32_t column_base(const Geom& g, int cx, int cy) {
    int px = cx + g.rx;
    px -= (px >= g.nx) ? g.nx : 0;
    int py = cy + g.ry;
    py -= (py >= g.ny) ? g.ny : 0;
    return ((uint32_t)px * g.ny + py) * (uint32_t)g.nz;
}

__device__ __forceinline__ void clear_voxel(const MapState& s, uint32_t k) {
    if (!in_bounds(k, s.V, s.counters)) return;
    s.hits[k] = 0u;
    s.passes[k] = 0u;
    s.minz[k] = __int_as_float(0x7f800000);
    for (int j = 0; j < s.ring_K; ++j) {
        const size_t o = (size_t)j * s.V + k;
        s.ring_hits[o] = 0u;
        s.ring_passes[o] = 0u;
        s.ring_minz[o] = __int_as_float(0x7f800000);
    }
}

// One launch for the whole shift: warp units [0, n_cols) clear entering
// columns whole (the x slab, then the rest of the y slab), the units after
// them clear the z slab, 32 columns per unit (one per lane).
__global__ void k_shift_columns(MapState s, Geom g, int dx, int dy, int dz, long long n_xslab, long long n_cols,
                                long long n_units) {
    pdl_wait();
    // Every kernel after it waits for it before touching the map, so its
    // dependents may launch at once: the per-point pass overlaps the shift.
    pdl_done();
    const long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n_units) return;
    const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
    if (u < n_cols) {
        int cx, cy;
        if (u < n_xslab) {
            const int k = (int)((unsigned)u / (unsigned)g.ny);
            cx = dx > 0 ? g.nx - dx + k : k;
            cy = (int)((unsigned)u % (unsigned)g.ny);
        } else {
            const long long w = u - n_xslab;
            const int k = (int)((unsigned)w / (unsigned)ady), l = (int)((unsigned)w % (unsigned)ady);
            cx = (dx > 0 ? 0 : adx) + k;
            cy = dy > 0 ? g.ny - dy + l : l;
        }
        const uint32_t base = column_base(g, cx, cy);
        for (int cz = lane; cz < g.nz; cz += 32) clear_voxel(s, base + (uint32_t)cz);
    } else {
        // the z slab of the columns that stay: one column per lane
        const int wy = g.ny - ady;
        const long long w = (u - n_cols) * 32 + lane;
        if (w < (long long)(g.nx - adx) * wy) {
            const int cx = (dx > 0 ? 0 : adx) + (int)((unsigned)w / (unsigned)wy);
            const int cy = (dy > 0 ? 0 : ady) + (int)((unsigned)w % (unsigned)wy);
            const uint32_t base = column_base(g, cx, cy);
            const int z0 = dz > 0 ? g.nz - dz : 0, z1 = dz > 0 ? g.nz : -dz;
            for (int cz = z0; cz < z1; ++cz) {
                int pz = cz + g.rz;
                pz -= (pz >= g.nz) ? g.nz : 0;
                clear_voxel(s, base + (uint32_t)pz);
            }
        }
    }
}

// ---- batched maps ----------------------------------------------------------

// The map m whose range [prefix[m], prefix[m+1]) holds unit u (0 <= u <
// prefix[B]): the largest m with prefix[m] <= u.
__device__ __forceinline__ int find_map(const long long* __restrict__ prefix, int B, long long u) {
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

// Window shifts of all maps of a batch step, one warp per unit (a whole
// entering column, 32 z-slab columns, or 1024 voxels of a map cleared
// whole), plus each map's quantised sensor position.
__global__ void __launch_bounds__(256) k_shift_batch(BatchTables t) {
    const int B = t.hdr->B;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        // the step's segment work list starts empty (all entries share it)
        t.ing[0].w.item_count[kListLen] = 0;
        t.ing[0].w.item_count[kListBlocksDone] = 0;
    }
    if (tid < B) {
        const IngestArgs& a = t.ing[tid];
        int q[3];
        bool ok = true;
        for (int k = 0; k < 3; ++k) ok &= quantise(a.T[4 * k + 3], a.S, a.neg_o256[k], &q[k]);
        t.sensors[tid] = make_int4(q[0], q[1], q[2], ok ? 1 : 0);
    }
    const int lane = threadIdx.x & 31;
    const long long total = t.hdr->shift_total;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = tid >> 5; u < total; u += nwarps) {
        const int m = find_map(t.shift_prefix, B, u);
        const long long lu = u - t.shift_prefix[m];
        const BatchShift& sh = t.sh[m];
        const Geom g = sh.g;
        if (sh.whole) {
            const long long V = (long long)g.nx * g.ny * g.nz;
            const long long v0 = lu * 1024;
            for (long long v = v0 + lane; v < v0 + 1024 && v < V; v += 32) clear_voxel(sh.s, (uint32_t)v);
            continue;
        }
        const int dx = sh.d[0], dy = sh.d[1], dz = sh.d[2];
        const int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
        const long long n_xslab = (long long)adx * g.ny;
        const long long n_cols = n_xslab + (long long)(g.nx - adx) * ady;
        if (lu < n_cols) {
            int cx, cy;
            if (lu < n_xslab) {
                const int k = (int)((unsigned)lu / (unsigned)g.ny);
                cx = dx > 0 ? g.nx - dx + k : k;
                cy = (int)((unsigned)lu % (unsigned)g.ny);
            } else {
                const long long w = lu - n_xslab;
                const int k = (int)((unsigned)w / (unsigned)ady), l = (int)((unsigned)w % (unsigned)ady);
                cx = (dx > 0 ? 0 : adx) + k;
                cy = dy > 0 ? g.ny - dy + l : l;
            }
            const uint32_t base = column_base(g, cx, cy);
            for (int cz = lane; cz < g.nz; cz += 32) clear_voxel(sh.s, base + (uint32_t)cz);
        } else {
            // 32 z-slab columns per unit, one per lane
            const int wy = g.ny - ady;
            const long long w = (lu - n_cols) * 32 + lane;
            if (w >= (long long)(g.nx - adx) * wy) continue;
            const int cx = (dx > 0 ? 0 : adx) + (int)((unsigned)w / (unsigned)wy);
            const int cy = (dy > 0 ? 0 : ady) + (int)((unsigned)w % (unsigned)wy);
            const uint32_t base = column_base(g, cx, cy);
            const int z0 = dz > 0 ? g.nz - dz : 0, z1 = dz > 0 ? g.nz : -dz;
            for (int cz = z0; cz < z1; ++cz) {
                int pz = cz + g.rz;
                pz -= (pz >= g.nz) ? g.nz : 0;
                clear_voxel(sh.s, base + (uint32_t)pz);
            }
        }
    }
}

// Per-point pass of all maps over the maps' 256-point blocks (one thread
// block each, or fewer looping over them); every block belongs to one map.
__global__ void __launch_bounds__(kRaysBlock) k_rays_batch(BatchTables t) {
    __shared__ int s_m;
    const int B = t.hdr->B;
    const long long total = t.hdr->ray_blocks;
    for (long long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (threadIdx.x == 0) s_m = find_map(t.ray_prefix, B, vb);
        __syncthreads();
        const int m = s_m;
        const int4 sq = t.sensors[m];
        const int qo[3] = {sq.x, sq.y, sq.z};
        rays_body(t.ing[m], (vb - t.ray_prefix[m]) * kRaysBlock, qo, sq.w != 0, t.ray_base[m], (unsigned int)m);
    }
}

// Ring-slot eviction of all buffered maps of a batch step, one warp per
// 1024 voxels of a map.
__global__ void __launch_bounds__(256) k_evict_batch(BatchTables t) {
    const int B = t.hdr->B;
    const long long total = t.hdr->evict_total;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < total; u += nwarps) {
        const int m = find_map(t.evict_prefix, B, u);
        const BatchShift& sh = t.sh[m];
        const uint32_t v0 = (uint32_t)(u - t.evict_prefix[m]) * 1024u;
        if ((sh.s.V & 3u) == 0u) {
            for (uint32_t v = v0 + 4u * lane; v < v0 + 1024u && v < sh.s.V; v += 128) evict_quad(sh.s, sh.evict, v);
        } else {
            for (uint32_t v = v0 + lane; v < v0 + 1024u && v < sh.s.V; v += 32) evict_voxel(sh.s, sh.evict, v);
        }
    }
}

// Blocks of the persistent segment walk: every SM filled to its occupancy.
template <bool kBatch, bool kSlot, bool kPow2>
int march_grid(const MarchShape& shape) {
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    int per_sm = shape.blocks_per_sm;
    if (per_sm <= 0) {
        // resident blocks per SM for 128- and 256-thread blocks, per device
        static std::atomic<int> cache[64][2];  // one per instantiation
        const int b = shape.block == 256 ? 1 : 0;
        nb = dev >= 0 && dev < 64 ? cache[dev][b].load(std::memory_order_relaxed) : 0;
        if (nb <= 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march<kBatch, kSlot, kPow2>, shape.block, 0);
            if (nb > 0 && dev >= 0 && dev < 64) cache[dev][b].store(nb, std::memory_order_relaxed);
        }
        per_sm = nb > 0 ? nb : 1;
    }
    return sms * per_sm;
}

}  // namespace

long long shift_units(const Geom& g, const int d[3], int whole) {
    if (whole) return ((long long)g.nx * g.ny * g.nz + 1023) / 1024;
    const long long adx = d[0] < 0 ? -d[0] : d[0], ady = d[1] < 0 ? -d[1] : d[1];
    long long u = adx * g.ny + (g.nx - adx) * ady;
    if (d[2] != 0) u += ((g.nx - adx) * (g.ny - ady) + 31) / 32;
    return u;
}

long long evict_units(const MapState& s) { return ((long long)s.V + 1023) / 1024; }

template <bool kSlot, bool kPow2>
cudaError_t launch_march_batch(const BatchTables& t, const IngestArgs& shared, const MarchShape& shape,
                               cudaStream_t st) {
    k_march<true, kSlot, kPow2><<<march_grid<true, kSlot, kPow2>(shape), shape.block, 0, st>>>(shared, t.ing,
                                                                                               t.sensors);
    return cudaGetLastError();
}

cudaError_t launch_batch_update(const BatchTables& t, int max_maps, long long max_ray_blocks, const IngestArgs& shared,
                                const MarchShape& shape, bool evict, bool slots, bool pow2, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    cudaError_t e;
    long long sblocks = (long long)sms * 8;
    if (sblocks * 256 < max_maps) sblocks = (max_maps + 255) / 256;
    count_launch();
    k_shift_batch<<<(unsigned)sblocks, 256, 0, st>>>(t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (evict) {
        count_launch();
        k_evict_batch<<<(unsigned)(sms * 8), 256, 0, st>>>(t);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // one block per 256-point block of the largest step the tables allow
    // (blocks past this step's count return at once), so the hardware
    // scheduler balances them
    long long rblocks = max_ray_blocks > 0 ? max_ray_blocks : 1;
    if (rblocks > 0x7fffffffLL) rblocks = 0x7fffffffLL;
    count_launch();
    k_rays_batch<<<(unsigned)rblocks, kRaysBlock, 0, st>>>(t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_launch();
    if (slots) return pow2 ? launch_march_batch<true, true>(t, shared, shape, st)
                           : launch_march_batch<true, false>(t, shared, shape, st);
    return pow2 ? launch_march_batch<false, true>(t, shared, shape, st)
                : launch_march_batch<false, false>(t, shared, shape, st);
}

bool pow2_window(const Geom& g) {
    return ((g.nx & (g.nx - 1)) | (g.ny & (g.ny - 1)) | (g.nz & (g.nz - 1))) == 0;
}

long long max_segments_per_ray(const Geom& g, int seg_len) {
    const int n = g.nx > g.ny ? (g.nx > g.nz ? g.nx : g.nz) : (g.ny > g.nz ? g.ny : g.nz);
    return (n + seg_len - 1) / seg_len;
}

cudaError_t launch_init_state(const MapState& s, long long V, cudaStream_t st) {
    const int block = 256;
    long long blocks = (V + block - 1) / block;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    count_launch();
    k_init_state<<<(unsigned)blocks, block, 0, st>>>(s.hits, s.passes, s.minz, V);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || s.ring_K == 0) return e;
    count_launch();
    k_init_state<<<152 * 16, block, 0, st>>>(s.ring_hits, s.ring_passes, s.ring_minz, V * s.ring_K);
    return cudaGetLastError();
}

cudaError_t launch_evict(const MapState& s, unsigned long long mask, cudaStream_t st) {
    if (s.ring_K == 0 || mask == 0ull) return cudaSuccess;
    const long long threads = (s.V & 3u) == 0u ? (long long)s.V / 4 : (long long)s.V;
    const long long blocks = (threads + 255) / 256;
    count_launch();
    return launch_pdl(k_evict, dim3((unsigned)blocks), dim3(256), 0, st, s, mask);
}

cudaError_t launch_shift(const MapState& s, const Geom& g_new, const long long d[3], cudaStream_t st) {
    const int dx = (int)d[0], dy = (int)d[1], dz = (int)d[2];
    const long long adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
    const long long n_xslab = adx * g_new.ny;
    const long long n_cols = n_xslab + (g_new.nx - adx) * ady;
    const long long n_z = dz != 0 ? ((g_new.nx - adx) * (g_new.ny - ady) + 31) / 32 : 0;
    const long long n_units = n_cols + n_z;
    if (n_units == 0) return cudaSuccess;
    const int block = 256;
    const long long blocks = (n_units * 32 + block - 1) / block;
    count_launch();
    return launch_pdl(k_shift_columns, dim3((unsigned)blocks), dim3(block), 0, st, s, g_new, dx, dy, dz, n_xslab,
                      n_cols, n_units);
}

template <bool kSlot, bool kPow2>
cudaError_t launch_march_one(const IngestArgs& a, const MarchShape& shape, cudaStream_t st) {
    const IngestArgs* none = nullptr;
    const int4* no_sensors = nullptr;
    return launch_pdl(k_march<false, kSlot, kPow2>, dim3(march_grid<false, kSlot, kPow2>(shape)), dim3(shape.block),
                      0, st, a, none, no_sensors);
}

// The fused ingest as a cooperative launch: one block per resident slot
// (march_blocks_per_sm, if set, caps the blocks per SM).
template <bool kPow2>
cudaError_t launch_fused(const IngestArgs& a, const MarchShape& shape, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    static std::atomic<int> cache[64][2];  // resident blocks per SM, per device and block size
    const int b = shape.block == 256 ? 1 : 0;
    int nb = dev >= 0 && dev < 64 ? cache[dev][b].load(std::memory_order_relaxed) : 0;
    if (nb <= 0) {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ingest_fused<kPow2>, shape.block, 0);
        if (e != cudaSuccess) return e;
        if (nb <= 0) return cudaErrorLaunchOutOfResources;
        if (dev >= 0 && dev < 64) cache[dev][b].store(nb, std::memory_order_relaxed);
    }
    const int per_sm = shape.blocks_per_sm > 0 && shape.blocks_per_sm < nb ? shape.blocks_per_sm : nb;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * per_sm));
    cfg.blockDim = dim3((unsigned)shape.block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_ingest_fused<kPow2>, a);
}

cudaError_t launch_ingest(const IngestArgs& a, const MarchShape& shape, cudaStream_t st, cudaEvent_t marker) {
    if (a.n <= 0) return cudaSuccess;
    if (shape.fused) {
        // one kernel lists and walks; the marker precedes it
        cudaError_t e = cudaSuccess;
        if (marker && (e = cudaEventRecord(marker, st)) != cudaSuccess) return e;
        count_launch();
        return pow2_window(a.g) ? launch_fused<true>(a, shape, st) : launch_fused<false>(a, shape, st);
    }
    // the work list is empty here: the previous scan's walk emptied it
    const long long blocks = (a.n + kRaysBlock - 1) / kRaysBlock;
    count_launch();
    cudaError_t e = launch_pdl(k_rays, dim3((unsigned)blocks), dim3(kRaysBlock), 0, st, a);
    if (e != cudaSuccess) return e;
    if (marker && (e = cudaEventRecord(marker, st)) != cudaSuccess) return e;
    count_launch();
    const bool pow2 = pow2_window(a.g);
    if (a.slot >= 0)
        return pow2 ? launch_march_one<true, true>(a, shape, st) : launch_march_one<true, false>(a, shape, st);
    return pow2 ? launch_march_one<false, true>(a, shape, st) : launch_march_one<false, false>(a, shape, st);
}

}  // namespace gvom
