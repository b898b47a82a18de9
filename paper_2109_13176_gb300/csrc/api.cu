// C ABI of libgvom (declared in include/gvom.h): argument checks, device
// state ownership, and stream-ordered launches of the kernels in ingest.cu
// and extract.cu. No exception crosses the ABI; every entry point returns a
// gvom_status.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "gvom_internal.h"
#include "../../include/gvom_microbench.h"

using gvom::ExtractParams;
using gvom::Geom;
using gvom::IngestArgs;
using gvom::MapState;

namespace gvom {
static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace gvom


namespace gvom {

bool valid_config(const gvom_config* c) {
    if (!c) return false;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1 || c->nx > 4096 || c->ny > 4096 || c->nz > 4096) return false;
    if ((long long)c->nx * c->ny * c->nz >= (1LL << 31)) return false;
    if (c->scan_buffer < 0 || c->scan_buffer > GVOM_MAX_SCAN_BUFFER) return false;
    if (!(c->res > 0.0) || !isfinite(c->res)) return false;
    if (!(c->max_range > 0.0) || !isfinite(c->max_range) || !(c->max_range / c->res <= 8192.0)) return false;
    if (!(c->obs_min_h >= 0.0f) || !(c->obs_max_h >= c->obs_min_h) || !isfinite(c->obs_max_h)) return false;
    if (c->hard_den == 0 || c->hard_den > 65535u || c->hard_num > c->hard_den) return false;
    if (c->slope_n < 3 || c->slope_n > 15 || (c->slope_n % 2) == 0) return false;
    if (c->slope_min_px < 3 || c->slope_min_px > c->slope_n * c->slope_n) return false;
    if (c->neg_max_px < 1 || c->neg_max_px > 64) return false;
    if (!isfinite(c->neg_thresh)) return false;
    return true;
}

}  // namespace gvom

namespace gvom {

Geom geom_of(const gvom_map* m) {
    Geom g;
    g.nx = m->cfg.nx;
    g.ny = m->cfg.ny;
    g.nz = m->cfg.nz;
    g.rx = (int)gvom::floor_mod(m->origin[0], m->cfg.nx);
    g.ry = (int)gvom::floor_mod(m->origin[1], m->cfg.ny);
    g.rz = (int)gvom::floor_mod(m->origin[2], m->cfg.nz);
    return g;
}

long long voxels(const gvom_map* m) { return (long long)m->cfg.nx * m->cfg.ny * m->cfg.nz; }

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GVOM_OK;
    if (e == cudaErrorMemoryAllocation) return GVOM_ERR_OUT_OF_MEMORY;
    return GVOM_ERR_CUDA;
}

// The origin must keep every voxel index far inside int64 arithmetic.
bool valid_origin(const int64_t o[3]) {
    for (int k = 0; k < 3; ++k)
        if (o[k] < -(1LL << 40) || o[k] > (1LL << 40)) return false;
    return true;
}

ExtractParams extract_params(const gvom_map* m) {
    ExtractParams p;
    p.g = geom_of(m);
    p.res = (float)m->cfg.res;
    p.obs_min_h = m->cfg.obs_min_h;
    p.obs_max_h = m->cfg.obs_max_h;
    p.hard_num = m->cfg.hard_num;
    p.hard_den = m->cfg.hard_den;
    p.slope_n = m->cfg.slope_n;
    p.slope_min_px = m->cfg.slope_min_px;
    p.neg_max_px = m->cfg.neg_max_px;
    p.neg_thresh = m->cfg.neg_thresh;
    p.px_tile = m->tune.px_tile;
    p.col_shape = m->tune.col_shape;
    return p;
}

// A pose must be finite with a rotation part whose entries lie in [-1, 1]
// (up to rounding), so that no ray is longer than sqrt(3) max_range in the
// map frame; the traversal's 32-bit arithmetic relies on that bound.
bool valid_pose(const double T[12]) {
    for (int k = 0; k < 12; ++k)
        if (!isfinite(T[k])) return false;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            if (fabs(T[4 * r + c]) > 1.0 + 1e-6) return false;
    return true;
}

bool valid_tuning(const gvom_tuning* t) {
    return t && t->seg_len >= 1 && t->seg_len <= 4096 && (t->march_block == 128 || t->march_block == 256) &&
           t->march_blocks_per_sm >= 0 && t->march_blocks_per_sm <= 32 &&
           (t->px_tile == 0 || (t->px_tile >= 4 && t->px_tile <= 64)) && t->col_shape >= 0 && t->col_shape <= 3 &&
           (t->fused_ingest == 0 || t->fused_ingest == 1);
}

// Grows the ray records and the segment work list to hold a scan of n points
// under the current segment length. Waits for the map's stream first when
// buffers in use are replaced.
}  // namespace gvom

namespace {

using gvom::cuda_status;
using gvom::extract_params;
using gvom::geom_of;
using gvom::valid_config;
using gvom::valid_origin;
using gvom::valid_pose;
using gvom::valid_tuning;
using gvom::voxels;

int ensure_capacity(gvom_map* m, long long n, cudaStream_t st) {
    const long long per_ray = gvom::max_segments_per_ray(geom_of(m), m->tune.seg_len);
    if (n <= m->w.cap_points && n * per_ray <= m->w.cap_items) return GVOM_OK;
    long long cap = m->w.cap_points > n ? m->w.cap_points : n;
    if (cap < 4096) cap = 4096;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    cudaFree(m->w.rays);
    cudaFree(m->w.items);
    m->w.rays = nullptr;
    m->w.items = nullptr;
    m->w.cap_points = 0;
    m->w.cap_items = 0;
    e = cudaMalloc(&m->w.rays, sizeof(int4) * (size_t)cap);
    // 16 bytes per entry (the fused ingest's int4 entries), all zero: no
    // entry carries a fused scan's tag before that scan writes it (cleared on
    // the caller's stream, ahead of the kernels that will read the list)
    if (e == cudaSuccess) e = cudaMalloc(&m->w.items, sizeof(int4) * (size_t)(cap * per_ray));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->w.items, 0, sizeof(int4) * (size_t)(cap * per_ray), st);
    if (e != cudaSuccess) {
        cudaFree(m->w.rays);
        cudaFree(m->w.items);
        m->w.rays = nullptr;
        m->w.items = nullptr;
        cudaGetLastError();
        return GVOM_ERR_OUT_OF_MEMORY;
    }
    m->w.cap_points = cap;
    m->w.cap_items = cap * per_ray;
    return GVOM_OK;
}

}  // namespace

extern "C" {

int gvom_tuning_default(gvom_tuning* out) {
    if (!out) return GVOM_ERR_INVALID_ARG;
    out->seg_len = 16;
    out->march_block = 256;
    out->march_blocks_per_sm = 0;
    out->px_tile = 0;
    out->col_shape = 0;
    out->fused_ingest = 0;
    return GVOM_OK;
}

int gvom_set_tuning(gvom_map* m, const gvom_tuning* t) {
    if (!m || !valid_tuning(t)) return GVOM_ERR_INVALID_ARG;
    if (t->px_tile > 0) {
        // the pixel pass's tile and halo must fit one block's shared memory
        gvom_map probe = *m;
        probe.tune = *t;
        if (gvom::slope_negative_smem(extract_params(&probe)) > 200 * 1024) return GVOM_ERR_INVALID_ARG;
    }
    m->tune = *t;
    return GVOM_OK;
}

int gvom_get_tuning(const gvom_map* m, gvom_tuning* out) {
    if (!m || !out) return GVOM_ERR_INVALID_ARG;
    *out = m->tune;
    return GVOM_OK;
}

int gvom_reserve(gvom_map* m, int64_t max_points, gvom_stream_t stream) {
    if (!m || max_points < 0 || max_points > GVOM_MAX_SCAN_POINTS) return GVOM_ERR_INVALID_ARG;
    return ensure_capacity(m, max_points, (cudaStream_t)stream);
}


int gvom_config_default(gvom_config* out) {
    if (!out) return GVOM_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->nx = 128;
    out->ny = 128;
    out->nz = 32;
    out->res = 0.2;
    out->max_range = 100.0;
    out->obs_min_h = 0.3f;
    out->obs_max_h = 2.0f;
    out->hard_num = 1;
    out->hard_den = 2;
    out->slope_n = 5;
    out->slope_min_px = 3;
    out->neg_max_px = 10;
    out->neg_thresh = 0.3f;
    return GVOM_OK;
}

int gvom_create(const gvom_config* cfg, gvom_map** out) {
    if (!out) return GVOM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_config(cfg)) return GVOM_ERR_INVALID_ARG;
    gvom_map* m = new (std::nothrow) gvom_map();
    if (!m) return GVOM_ERR_OUT_OF_MEMORY;
    m->cfg = *cfg;
    gvom_tuning_default(&m->tune);
    cudaGetDevice(&m->device);
    const long long V = voxels(m);
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&m->s.hits, sizeof(uint32_t) * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&m->s.passes, sizeof(uint32_t) * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&m->s.minz, sizeof(float) * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&m->s.counters, sizeof(unsigned long long) * gvom::kCounters);
    if (e == cudaSuccess) e = cudaMalloc(&m->height_scratch, sizeof(float) * (size_t)cfg->nx * cfg->ny);
    if (e == cudaSuccess) e = cudaMalloc(&m->w.item_count, gvom::kScratchWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(m->w.item_count, 0, gvom::kScratchWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&m->lut_counts, sizeof(unsigned int) * (size_t)gvom::lut_blocks(V));
    m->s.V = (uint32_t)V;
    const int K = cfg->scan_buffer;
    if (K > 0) {
        if (e == cudaSuccess) e = cudaMalloc(&m->s.ring_hits, sizeof(uint32_t) * (size_t)V * K);
        if (e == cudaSuccess) e = cudaMalloc(&m->s.ring_passes, sizeof(uint32_t) * (size_t)V * K);
        if (e == cudaSuccess) e = cudaMalloc(&m->s.ring_minz, sizeof(float) * (size_t)V * K);
        if (e == cudaSuccess) m->s.ring_K = K;
    }
    if (e == cudaSuccess) e = cudaMemset(m->s.counters, 0, sizeof(unsigned long long) * gvom::kCounters);
    if (e == cudaSuccess) e = gvom::launch_init_state(m->s, V, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        gvom_destroy(m);
        cudaGetLastError();
        return cuda_status(e);
    }
    *out = m;
    return GVOM_OK;
}

void gvom_destroy(gvom_map* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->s.hits);
    cudaFree(m->s.passes);
    cudaFree(m->s.minz);
    cudaFree(m->s.counters);
    cudaFree(m->height_scratch);
    cudaFree(m->w.rays);
    cudaFree(m->w.items);
    cudaFree(m->w.item_count);
    cudaFree(m->lut_counts);
    cudaFree(m->s.ring_hits);
    cudaFree(m->s.ring_passes);
    cudaFree(m->s.ring_minz);
    if (m->multi) gvom_batch_destroy(m->multi);
    delete m;
}

int gvom_get_config(const gvom_map* m, gvom_config* out) {
    if (!m || !out) return GVOM_ERR_INVALID_ARG;
    *out = m->cfg;
    return GVOM_OK;
}

int gvom_origin_for_pose(const gvom_map* m, const double vehicle_xyz[3], int64_t out_origin[3]) {
    if (!m || !vehicle_xyz || !out_origin) return GVOM_ERR_INVALID_ARG;
    const double inv_res = 1.0 / m->cfg.res;
    const int half[3] = {m->cfg.nx / 2, m->cfg.ny / 2, m->cfg.nz / 2};
    int64_t o[3];
    for (int k = 0; k < 3; ++k) {
        if (!isfinite(vehicle_xyz[k])) return GVOM_ERR_INVALID_ARG;
        const double f = floor(vehicle_xyz[k] * inv_res);
        if (!(fabs(f) < 1e12)) return GVOM_ERR_INVALID_ARG;
        o[k] = (int64_t)f - half[k];
    }
    memcpy(out_origin, o, sizeof(o));
    return GVOM_OK;
}

int gvom_get_origin(const gvom_map* m, int64_t out_origin[3]) {
    if (!m || !out_origin) return GVOM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) out_origin[k] = m->origin[k];
    return GVOM_OK;
}

int gvom_reset(gvom_map* m, const int64_t origin[3], gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:reset");
    if (!m || !origin || !valid_origin(origin)) return GVOM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) m->origin[k] = origin[k];
    m->buf_head = 0;
    m->buf_occupied = 0;
    // the work list starts empty again (after an error mid-scan it may not be)
    const cudaError_t e =
        cudaMemsetAsync(m->w.item_count, 0, gvom::kScratchWords * sizeof(unsigned long long), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(gvom::launch_init_state(m->s, voxels(m), (cudaStream_t)stream));
}

int gvom_shift(gvom_map* m, const int64_t new_origin[3], gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:shift");
    if (!m || !new_origin || !valid_origin(new_origin)) return GVOM_ERR_INVALID_ARG;
    long long d[3];
    bool whole = false, none = true;
    const int n[3] = {m->cfg.nx, m->cfg.ny, m->cfg.nz};
    for (int k = 0; k < 3; ++k) {
        d[k] = new_origin[k] - m->origin[k];
        if (d[k] != 0) none = false;
        if (d[k] >= n[k] || d[k] <= -n[k]) whole = true;
    }
    if (none) return GVOM_OK;
    for (int k = 0; k < 3; ++k) m->origin[k] = new_origin[k];
    if (whole) return cuda_status(gvom::launch_init_state(m->s, voxels(m), (cudaStream_t)stream));
    return cuda_status(gvom::launch_shift(m->s, geom_of(m), d, (cudaStream_t)stream));
}

int gvom_ingest_scan(gvom_map* m, const float* pts_dev, int64_t n, int32_t stride, const double T_ws[12],
                     gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:ingest");
    if (!m || !T_ws || n < 0 || (stride != 3 && stride != 4)) return GVOM_ERR_INVALID_ARG;
    if (n > 0 && !pts_dev) return GVOM_ERR_INVALID_ARG;
    if (n > GVOM_MAX_SCAN_POINTS) return GVOM_ERR_INVALID_ARG;
    if (stride == 4 && (((uintptr_t)pts_dev) & 15u) != 0) return GVOM_ERR_INVALID_ARG;
    if ((((uintptr_t)pts_dev) & 3u) != 0) return GVOM_ERR_INVALID_ARG;
    if (!valid_pose(T_ws)) return GVOM_ERR_INVALID_ARG;
    int rc = n > 0 ? ensure_capacity(m, n, (cudaStream_t)stream) : GVOM_OK;
    if (rc != GVOM_OK) return rc;
    // with a scan buffer, this scan takes the oldest slot (an empty scan too)
    int slot = -1;
    const unsigned long long evict = gvom::take_slots(m, 1, &slot);
    rc = cuda_status(gvom::launch_evict(m->s, evict, (cudaStream_t)stream));
    if (rc != GVOM_OK) return rc;
    if (n == 0) {
        m->scans += 1;
        return GVOM_OK;
    }
    IngestArgs a;
    memset(&a, 0, sizeof(a));
    a.slot = slot;
    a.pts = pts_dev;
    a.n = n;
    a.stride = stride;
    for (int k = 0; k < 12; ++k) a.T[k] = T_ws[k];
    a.S = 256.0 * (1.0 / m->cfg.res);
    a.r2max = m->cfg.max_range * m->cfg.max_range;
    for (int k = 0; k < 3; ++k) a.neg_o256[k] = -256.0 * (double)m->origin[k];
    a.g = geom_of(m);
    a.s = m->s;
    a.w = m->w;
    a.seg_len = m->tune.seg_len;
    gvom::MarchShape shape;
    shape.block = m->tune.march_block;
    shape.blocks_per_sm = m->tune.march_blocks_per_sm;
    shape.fused = false;
    if (m->tune.fused_ingest && slot < 0 &&
        gvom::max_segments_per_ray(a.g, a.seg_len) <= gvom::kFusedMaxSegments) {
        // a captured launch would replay one tag: capturing streams take the
        // two kernels
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            cs = cudaStreamCaptureStatusActive;
        }
        if (cs == cudaStreamCaptureStatusNone) {
            if (m->fused_epoch + 1 >= gvom::kFusedEpochs) {
                // the tags are about to repeat: no entry may keep an old one
                const cudaError_t e = cudaMemsetAsync(m->w.items, 0, sizeof(int4) * (size_t)m->w.cap_items,
                                                      (cudaStream_t)stream);
                if (e != cudaSuccess) return cuda_status(e);
                m->fused_epoch = 0;
            }
            a.epoch = ++m->fused_epoch;
            shape.fused = true;
        }
    }
    m->scans += 1;
    m->points_in += n;
    return cuda_status(gvom::launch_ingest(a, shape, (cudaStream_t)stream, m->walk_marker));
}

int gvom_set_walk_marker(gvom_map* m, void* cuda_event) {
    if (!m) return GVOM_ERR_INVALID_ARG;
    m->walk_marker = (cudaEvent_t)cuda_event;
    return GVOM_OK;
}

int gvom_update(gvom_map* m, const double vehicle_xyz[3], const float* pts_dev, int64_t n, int32_t stride,
                const double T_ws[12], gvom_stream_t stream) {
    if (!m || !vehicle_xyz || !T_ws || n < 0 || (stride != 3 && stride != 4) || (n > 0 && !pts_dev))
        return GVOM_ERR_INVALID_ARG;
    if (!valid_pose(T_ws)) return GVOM_ERR_INVALID_ARG;
    int64_t o[3];
    int rc = gvom_origin_for_pose(m, vehicle_xyz, o);
    if (rc != GVOM_OK) return rc;
    rc = gvom_shift(m, o, stream);
    if (rc != GVOM_OK) return rc;
    return gvom_ingest_scan(m, pts_dev, n, stride, T_ws, stream);
}

int gvom_extract_maps(gvom_map* m, const gvom_maps_out* out, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:extract");
    if (!m || !out) return GVOM_ERR_INVALID_ARG;
    const ExtractParams p = extract_params(m);
    cudaStream_t st = (cudaStream_t)stream;
    float* height = out->height_dev ? out->height_dev : m->height_scratch;
    cudaError_t e = gvom::launch_columns(m->s, p, height, out->density_dev, out->flags_dev, st);
    if (e != cudaSuccess) return cuda_status(e);
    if (out->slope_dev || out->roughness_dev || out->flags_dev)
        e = gvom::launch_slope_negative(p, height, out->slope_dev, out->roughness_dev, out->flags_dev, st);
    return cuda_status(e);
}

int gvom_update_extract(gvom_map* m, const double vehicle_xyz[3], const float* pts_dev, int64_t n, int32_t stride,
                        const double T_ws[12], const gvom_maps_out* out, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:update_extract");
    if (!m || !out) return GVOM_ERR_INVALID_ARG;
    const int rc = gvom_update(m, vehicle_xyz, pts_dev, n, stride, T_ws, stream);
    if (rc != GVOM_OK) return rc;
    return gvom_extract_maps(m, out, stream);
}

int gvom_import_state(gvom_map* m, const int64_t origin[3], const uint32_t* hits_dev, const uint32_t* passes_dev,
                      const float* minz_dev, gvom_stream_t stream) {
    if (!m || !origin || !valid_origin(origin) || !hits_dev || !passes_dev || !minz_dev) return GVOM_ERR_INVALID_ARG;
    if (m->cfg.scan_buffer != 0) return GVOM_ERR_INVALID_ARG;  // a buffer's per-scan slots cannot be restored
    if ((((uintptr_t)hits_dev) | ((uintptr_t)passes_dev) | ((uintptr_t)minz_dev)) & 3u) return GVOM_ERR_INVALID_ARG;
    gvom::NvtxRange nvtx_range("gvom:import_state");
    for (int k = 0; k < 3; ++k) m->origin[k] = origin[k];
    return cuda_status(gvom::launch_scatter_voxels(m->s, geom_of(m), hits_dev, passes_dev, minz_dev,
                                                   (cudaStream_t)stream));
}

int gvom_extract_voxels(gvom_map* m, uint32_t* hits_dev, uint32_t* passes_dev, float* minz_dev,
                        gvom_stream_t stream) {
    if (!m) return GVOM_ERR_INVALID_ARG;
    if (!hits_dev && !passes_dev && !minz_dev) return GVOM_OK;
    return cuda_status(
        gvom::launch_gather_voxels(m->s, geom_of(m), hits_dev, passes_dev, minz_dev, (cudaStream_t)stream));
}

}  // extern "C"

namespace gvom {
unsigned long long take_slots(gvom_map* m, int k, int* slots) {
    const int K = m->cfg.scan_buffer;
    unsigned long long mask = 0;
    for (int j = 0; j < k; ++j) {
        if (K == 0) {
            slots[j] = -1;
            continue;
        }
        const int sl = m->buf_head;
        slots[j] = sl;
        mask |= m->buf_occupied & (1ull << sl);
        m->buf_occupied |= 1ull << sl;
        m->buf_head = sl + 1 == K ? 0 : sl + 1;
    }
    return mask;
}
}  // namespace gvom

extern "C" {

int gvom_ingest_multi(gvom_map* m, int32_t k, const float* const* pts_dev, const int64_t* n, int32_t stride,
                      const double* T_ws, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:ingest_multi");
    if (!m || !pts_dev || !n || !T_ws || k < 1 || k > GVOM_MAX_MULTI_SCANS || (stride != 3 && stride != 4))
        return GVOM_ERR_INVALID_ARG;
    if (m->cfg.scan_buffer > 0 && k > m->cfg.scan_buffer) return GVOM_ERR_INVALID_ARG;
    long long total = 0;
    for (int j = 0; j < k; ++j) {
        if (n[j] < 0 || n[j] > GVOM_MAX_SCAN_POINTS || (n[j] > 0 && !pts_dev[j])) return GVOM_ERR_INVALID_ARG;
        if ((((uintptr_t)pts_dev[j]) & (stride == 4 ? 15u : 3u)) != 0) return GVOM_ERR_INVALID_ARG;
        if (!valid_pose(T_ws + 12 * j)) return GVOM_ERR_INVALID_ARG;
        total += n[j];
    }
    if (total > GVOM_MAX_SCAN_POINTS) return GVOM_ERR_INVALID_ARG;
    return gvom::ingest_multi(m, k, pts_dev, n, stride, T_ws, (cudaStream_t)stream);
}

int gvom_export_lut(gvom_map* m, int64_t* lut_dev, uint32_t* data_hits_dev, uint32_t* data_passes_dev,
                    float* data_minz_dev, int64_t data_capacity, int64_t* n_occupied_dev, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:export_lut");
    if (!m || !lut_dev || !n_occupied_dev || data_capacity < 0) return GVOM_ERR_INVALID_ARG;
    if (data_capacity > 0 && (!data_hits_dev || !data_passes_dev || !data_minz_dev)) return GVOM_ERR_INVALID_ARG;
    return cuda_status(gvom::launch_export_lut(m->s, geom_of(m), m->lut_counts, (long long*)n_occupied_dev,
                                               (long long*)lut_dev, data_hits_dev, data_passes_dev, data_minz_dev,
                                               data_capacity, (cudaStream_t)stream));
}

int gvom_get_stats(gvom_map* m, gvom_stats* out) {
    if (!m || !out) return GVOM_ERR_INVALID_ARG;
    unsigned long long c[gvom::kCounters];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, m->s.counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    out->scans = m->scans;
    out->points_in = m->points_in;
    out->rays_valid = (int64_t)c[gvom::kRaysValid];
    out->hits_in_window = (int64_t)c[gvom::kHitsInWindow];
    out->pass_visits = (int64_t)c[gvom::kPassVisits];
    if (c[gvom::kStatus] & gvom::kStatusBounds) return GVOM_ERR_BOUNDS;
    return (c[gvom::kStatus] & gvom::kStatusTimeout) ? GVOM_ERR_TIMEOUT : GVOM_OK;
}

int gvom_reset_stats(gvom_map* m, gvom_stream_t stream) {
    if (!m) return GVOM_ERR_INVALID_ARG;
    m->scans = 0;
    m->points_in = 0;
    return cuda_status(cudaMemsetAsync(m->s.counters, 0, sizeof(unsigned long long) * gvom::kCounters,
                                       (cudaStream_t)stream));
}

int64_t gvom_kernel_launches(void) { return (int64_t)gvom::g_launches.load(); }

const char* gvom_status_string(int status) {
    switch (status) {
        case GVOM_OK: return "ok";
        case GVOM_NOT_READY: return "not finished yet";
        case GVOM_ERR_INVALID_ARG: return "invalid argument";
        case GVOM_ERR_OUT_OF_MEMORY: return "out of device memory";
        case GVOM_ERR_CUDA: return "CUDA error";
        case GVOM_ERR_TIMEOUT: return "device wait timed out";
        case GVOM_ERR_BOUNDS: return "index out of bounds (checked build)";
        default: return "unknown status";
    }
}

}  // extern "C"
