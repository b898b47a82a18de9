// Batched update of many independent maps (include/gvom.h, gvom_batch_*).
//
// One step folds one scan into each of B maps and, optionally, extracts
// every map's 2D products, with five kernels for the whole batch instead of
// five per map: the shifts of all maps (plus each map's quantised sensor),
// the per-point pass over all maps' points, one persistent segment walk
// over all maps' traversal segments (which balances maps of uneven size),
// the column pass and the pixel pass. The per-step tables (each map's
// pose, point pointer and count, shift, outputs, and the prefix counts the
// kernels use to find a unit's map) are copied to the device from one of
// two pinned buffers, and the kernels read every count from there, so the
// five launches are captured once as a CUDA graph and replayed every step.
#include <math.h>
#include <string.h>

#include <new>

#include "gvom_internal.h"
#include "../../include/gvom_microbench.h"

using gvom::BatchExtract;
using gvom::BatchHeader;
using gvom::BatchShift;
using gvom::BatchTables;
using gvom::ExtractParams;
using gvom::Geom;
using gvom::IngestArgs;

namespace {

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Byte offsets of the table arrays inside one allocation.
struct Layout {
    size_t hdr, ing, sh, ex, shift_prefix, ray_prefix, ray_base, col_prefix, tile_prefix, sensors, evict_prefix,
        bytes;
};

Layout layout_for(int max_maps) {
    Layout L;
    size_t o = 0;
    L.hdr = o;
    o = align16(o + sizeof(BatchHeader));
    L.ing = o;
    o = align16(o + sizeof(IngestArgs) * max_maps);
    L.sh = o;
    o = align16(o + sizeof(BatchShift) * max_maps);
    L.ex = o;
    o = align16(o + sizeof(BatchExtract) * max_maps);
    L.shift_prefix = o;
    o = align16(o + sizeof(long long) * (max_maps + 1));
    L.ray_prefix = o;
    o = align16(o + sizeof(long long) * (max_maps + 1));
    L.ray_base = o;
    o = align16(o + sizeof(long long) * max_maps);
    L.col_prefix = o;
    o = align16(o + sizeof(long long) * (max_maps + 1));
    L.tile_prefix = o;
    o = align16(o + sizeof(long long) * (max_maps + 1));
    L.sensors = o;
    o = align16(o + sizeof(int4) * max_maps);
    L.evict_prefix = o;
    o = align16(o + sizeof(long long) * (max_maps + 1));
    L.bytes = o;
    return L;
}

BatchTables tables_at(char* base, const Layout& L) {
    BatchTables t;
    t.hdr = reinterpret_cast<BatchHeader*>(base + L.hdr);
    t.ing = reinterpret_cast<IngestArgs*>(base + L.ing);
    t.sh = reinterpret_cast<BatchShift*>(base + L.sh);
    t.ex = reinterpret_cast<BatchExtract*>(base + L.ex);
    t.shift_prefix = reinterpret_cast<long long*>(base + L.shift_prefix);
    t.ray_prefix = reinterpret_cast<long long*>(base + L.ray_prefix);
    t.ray_base = reinterpret_cast<long long*>(base + L.ray_base);
    t.col_prefix = reinterpret_cast<long long*>(base + L.col_prefix);
    t.tile_prefix = reinterpret_cast<long long*>(base + L.tile_prefix);
    t.sensors = reinterpret_cast<int4*>(base + L.sensors);
    t.evict_prefix = reinterpret_cast<long long*>(base + L.evict_prefix);
    return t;
}

}  // namespace

struct gvom_batch {
    int max_maps;
    long long max_points;
    int flags;
    Layout L;
    char* d_tables;
    char* h_tables[2];
    cudaEvent_t copied[2];
    int cur;
    gvom::RayScratch w;
    gvom_tuning tune;
    // captured graph and what it was captured for
    cudaGraphExec_t exec;
    cudaStream_t cap_stream;
    int g_B, g_extract, g_slots, g_zmax, g_pow2;
    size_t g_px_smem;  // the captured pixel pass's shared memory per block
    long long g_cap_items;
    long long g_kernels;  // kernels in the captured graph, counted per replay
    long long steps;
    int64_t* new_o;  // 3 * max_maps: this step's origins
};

namespace {

void free_scratch(gvom_batch* b) {
    cudaFree(b->w.rays);
    cudaFree(b->w.items);
    b->w.rays = nullptr;
    b->w.items = nullptr;
    b->w.cap_points = 0;
    b->w.cap_items = 0;
}

void drop_graph(gvom_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Grows the segment work list to hold `items` entries (synchronising first).
int grow_items(gvom_batch* b, long long items, cudaStream_t st) {
    if (items <= b->w.cap_items) return GVOM_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return gvom::cuda_status(e);
    cudaFree(b->w.items);
    b->w.items = nullptr;
    b->w.cap_items = 0;
    const long long cap = items + items / 4;
    e = cudaMalloc(&b->w.items, sizeof(uint2) * (size_t)cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GVOM_ERR_OUT_OF_MEMORY;
    }
    b->w.cap_items = cap;
    drop_graph(b);
    return GVOM_OK;
}

IngestArgs ingest_args(const gvom_map* mp, const float* pts, long long n, int stride, int seg_len, const double* T,
                       const gvom::RayScratch& w) {
    IngestArgs a;
    memset(&a, 0, sizeof(a));
    a.slot = -1;
    a.pts = pts;
    a.n = n;
    a.stride = stride;
    a.seg_len = seg_len;
    for (int k = 0; k < 12; ++k) a.T[k] = T[k];
    a.S = 256.0 * (1.0 / mp->cfg.res);
    a.r2max = mp->cfg.max_range * mp->cfg.max_range;
    for (int k = 0; k < 3; ++k) a.neg_o256[k] = -256.0 * (double)mp->origin[k];
    a.g = gvom::geom_of(mp);
    a.s = mp->s;
    a.w = w;
    return a;
}

}  // namespace

extern "C" {

int gvom_batch_create(int32_t max_maps, int64_t max_points, int32_t flags, gvom_batch** out) {
    if (!out) return GVOM_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_maps < 1 || max_maps > 4096 || max_points < 1 || max_points > GVOM_MAX_SCAN_POINTS ||
        (flags & ~GVOM_BATCH_GRAPH) != 0)
        return GVOM_ERR_INVALID_ARG;
    gvom_batch* b = new (std::nothrow) gvom_batch();
    if (!b) return GVOM_ERR_OUT_OF_MEMORY;
    b->max_maps = max_maps;
    b->max_points = max_points;
    b->flags = flags;
    b->L = layout_for(max_maps);
    gvom_tuning_default(&b->tune);
    cudaError_t e = cudaMalloc(&b->d_tables, b->L.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tables[0], b->L.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_tables[1], b->L.bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->w.item_count, gvom::kScratchWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->w.rays, sizeof(int4) * (size_t)max_points);
    if (e == cudaSuccess) b->w.cap_points = max_points;
    if (e == cudaSuccess) {
        b->new_o = new (std::nothrow) int64_t[3 * (size_t)max_maps];
        if (!b->new_o) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        gvom_batch_destroy(b);
        cudaGetLastError();
        return gvom::cuda_status(e);
    }
    memset(b->h_tables[0], 0, b->L.bytes);
    memset(b->h_tables[1], 0, b->L.bytes);
    *out = b;
    return GVOM_OK;
}

void gvom_batch_destroy(gvom_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    free_scratch(b);
    cudaFree(b->w.item_count);
    cudaFree(b->d_tables);
    cudaFreeHost(b->h_tables[0]);
    cudaFreeHost(b->h_tables[1]);
    if (b->copied[0]) cudaEventDestroy(b->copied[0]);
    if (b->copied[1]) cudaEventDestroy(b->copied[1]);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete[] b->new_o;
    delete b;
}

int gvom_batch_set_tuning(gvom_batch* b, const gvom_tuning* t) {
    if (!b || !gvom::valid_tuning(t)) return GVOM_ERR_INVALID_ARG;
    b->tune = *t;
    drop_graph(b);
    return GVOM_OK;
}

int gvom_batch_step(gvom_batch* b, struct gvom_map* const* maps, int32_t B, const double* vehicle_xyz,
                    const float* const* pts_dev, const int64_t* n, int32_t stride, const double* T_ws,
                    const gvom_maps_out* outs, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:batch_step");
    if (!b || !maps || !vehicle_xyz || !pts_dev || !n || !T_ws || B < 1 || B > b->max_maps ||
        (stride != 3 && stride != 4))
        return GVOM_ERR_INVALID_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    // validate everything before any state changes
    long long total = 0, items = 0;
    size_t px_smem = 0;  // the pixel pass's shared memory: the largest any map of the step needs
    int zmax = 0;  // the largest nz, or -1 when some map cannot use the bulk-copy column pass
    int pow2 = 1;  // every map's window has power-of-two extents (the walk steps its index)
    for (int m = 0; m < B; ++m) {
        const gvom_map* mp = maps[m];
        if (!mp || n[m] < 0 || (n[m] > 0 && !pts_dev[m])) return GVOM_ERR_INVALID_ARG;
        if ((((uintptr_t)pts_dev[m]) & (stride == 4 ? 15u : 3u)) != 0) return GVOM_ERR_INVALID_ARG;
        if (!gvom::valid_pose(T_ws + 12 * m)) return GVOM_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!isfinite(vehicle_xyz[3 * m + k])) return GVOM_ERR_INVALID_ARG;
        for (int j = 0; j < m; ++j)
            if (maps[j] == mp) return GVOM_ERR_INVALID_ARG;  // one update per map per step
        total += n[m];
        items += n[m] * gvom::max_segments_per_ray(gvom::geom_of(mp), b->tune.seg_len);
        gvom::ExtractParams pmp = gvom::extract_params(mp);
        pmp.px_tile = 0;  // the batched passes use their own fixed shapes
        pmp.col_shape = 0;
        const size_t pm = gvom::slope_negative_smem(pmp);
        px_smem = pm > px_smem ? pm : px_smem;
        const int nz = mp->cfg.nz;
        if (zmax >= 0) zmax = ((nz & 3) == 0 && nz <= 256) ? (nz > zmax ? nz : zmax) : -1;
        pow2 &= gvom::pow2_window(gvom::geom_of(mp)) ? 1 : 0;
    }
    if (total > b->max_points) return GVOM_ERR_INVALID_ARG;
    if (zmax < 0) zmax = 0;
    int64_t* new_o = b->new_o;
    for (int m = 0; m < B; ++m) {
        const int rc = gvom_origin_for_pose(maps[m], vehicle_xyz + 3 * m, new_o + 3 * m);
        if (rc != GVOM_OK) return rc;
    }

    // the segment work list for this step's points
    const int grown = grow_items(b, items, st);
    if (grown != GVOM_OK) return grown;

    // fill this step's tables in the pinned buffer not in flight
    const int cur = b->cur;
    cudaError_t e = cudaEventSynchronize(b->copied[cur]);
    if (e != cudaSuccess) return gvom::cuda_status(e);
    BatchTables h = tables_at(b->h_tables[cur], b->L);
    long long shift_total = 0, ray_blocks = 0, col_tasks = 0, tiles = 0, ray_base = 0, evict_total = 0;
    int slots = 0;
    for (int m = 0; m < B; ++m) {
        gvom_map* mp = maps[m];
        // window shift: the host copy of the origin moves now, in enqueue order
        int d[3] = {0, 0, 0};
        int whole = 0;
        const int dims[3] = {mp->cfg.nx, mp->cfg.ny, mp->cfg.nz};
        for (int k = 0; k < 3; ++k) {
            const long long dk = new_o[3 * m + k] - mp->origin[k];
            if (dk >= dims[k] || dk <= -dims[k]) whole = 1;
            d[k] = (int)(whole ? 0 : dk);
        }
        if (whole) d[0] = d[1] = d[2] = 0;
        for (int k = 0; k < 3; ++k) mp->origin[k] = new_o[3 * m + k];
        const Geom g = gvom::geom_of(mp);
        BatchShift& sh = h.sh[m];
        sh.s = mp->s;
        sh.g = g;
        sh.d[0] = d[0];
        sh.d[1] = d[1];
        sh.d[2] = d[2];
        sh.whole = whole;
        h.shift_prefix[m] = shift_total;
        shift_total += gvom::shift_units(g, d, whole);
        int slot = -1;
        sh.evict = gvom::take_slots(mp, 1, &slot);
        h.evict_prefix[m] = evict_total;
        evict_total += sh.evict ? gvom::evict_units(mp->s) : 0;
        slots |= slot >= 0;

        h.ing[m] = ingest_args(mp, pts_dev[m], n[m], stride, b->tune.seg_len, T_ws + 12 * m, b->w);
        h.ing[m].slot = slot;
        h.ing[m].cnt_owner = m;
        h.ray_prefix[m] = ray_blocks;
        ray_blocks += (n[m] + 255) / 256;
        h.ray_base[m] = ray_base;
        ray_base += n[m];
        mp->scans += 1;
        mp->points_in += n[m];

        BatchExtract& ex = h.ex[m];
        ex.s = mp->s;
        ex.p = gvom::extract_params(mp);
        ex.p.px_tile = 0;
        ex.p.col_shape = 0;
        const gvom_maps_out* o = outs ? outs + m : nullptr;
        ex.height = (o && o->height_dev) ? o->height_dev : mp->height_scratch;
        ex.density = o ? o->density_dev : nullptr;
        ex.flags = o ? o->flags_dev : nullptr;
        ex.slope = o ? o->slope_dev : nullptr;
        ex.rough = o ? o->roughness_dev : nullptr;
        h.col_prefix[m] = col_tasks;
        col_tasks += ((long long)g.nx * g.ny + gvom::kColTask - 1) / gvom::kColTask;
        h.tile_prefix[m] = tiles;
        tiles += gvom::tiles_of(ex.p);
    }
    h.shift_prefix[B] = shift_total;
    h.ray_prefix[B] = ray_blocks;
    h.col_prefix[B] = col_tasks;
    h.tile_prefix[B] = tiles;
    h.evict_prefix[B] = evict_total;
    h.hdr->evict_total = evict_total;
    h.hdr->B = B;
    h.hdr->shift_total = shift_total;
    h.hdr->ray_blocks = ray_blocks;
    h.hdr->col_tasks = outs ? col_tasks : 0;
    h.hdr->tiles = outs ? tiles : 0;

    e = cudaMemcpyAsync(b->d_tables, b->h_tables[cur], b->L.bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->copied[cur], st);
    if (e != cudaSuccess) return gvom::cuda_status(e);
    b->cur ^= 1;
    b->steps += 1;

    const BatchTables t = tables_at(b->d_tables, b->L);
    IngestArgs shared;
    memset(&shared, 0, sizeof(shared));
    shared.w = b->w;
    gvom::MarchShape shape;
    shape.block = b->tune.march_block;
    shape.blocks_per_sm = b->tune.march_blocks_per_sm;
    shape.fused = false;
    const long long max_ray_blocks = (b->max_points + 255) / 256 + b->max_maps;
    const int do_extract = outs != nullptr;

    if (!(b->flags & GVOM_BATCH_GRAPH)) {
        e = gvom::launch_batch_update(t, b->max_maps, max_ray_blocks, shared, shape, slots, slots, pow2, st);
        if (e == cudaSuccess && do_extract) e = gvom::launch_batch_extract(t, b->max_maps, px_smem, zmax, st);
        return gvom::cuda_status(e);
    }

    if (!b->exec || b->g_extract != do_extract || b->g_px_smem < px_smem || b->g_cap_items != b->w.cap_items ||
        b->g_slots != slots || b->g_zmax != zmax || b->g_pow2 != pow2) {
        drop_graph(b);
        cudaGraph_t graph = nullptr;
        const long long before = gvom_kernel_launches();
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le =
                gvom::launch_batch_update(t, b->max_maps, max_ray_blocks, shared, shape, slots, slots, pow2,
                                          b->cap_stream);
            if (le == cudaSuccess && do_extract)
                le = gvom::launch_batch_extract(t, b->max_maps, px_smem, zmax, b->cap_stream);
            e = cudaStreamEndCapture(b->cap_stream, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            cudaGetLastError();
            return gvom::cuda_status(e);
        }
        b->g_extract = do_extract;
        b->g_px_smem = px_smem;
        b->g_zmax = zmax;
        b->g_slots = slots;
        b->g_pow2 = pow2;
        b->g_cap_items = b->w.cap_items;
        b->g_kernels = gvom_kernel_launches() - before;
        gvom::count_launch(-b->g_kernels);  // captured, not launched
    }
    gvom::count_launch(b->g_kernels);
    return gvom::cuda_status(cudaGraphLaunch(b->exec, st));
}

}  // extern "C"

namespace gvom {

// Several scans (one per sensor, each with its own pose) folded into one
// map with one per-point pass and one segment walk: the batch tables hold
// one entry per scan, all on the same map and with no shift. The map's
// batch (created here on first use, re-created when a call needs more
// entries or points) runs without a graph.
int ingest_multi(gvom_map* mp, int k, const float* const* pts_dev, const int64_t* n, int stride, const double* T_ws,
                 cudaStream_t st) {
    long long total = 0;
    for (int j = 0; j < k; ++j) total += n[j];
    gvom_batch* b = mp->multi;
    if (!b || b->max_maps < k || b->max_points < total) {
        const int maps = b && b->max_maps > k ? b->max_maps : (k > 8 ? k : 8);
        long long pts = b && b->max_points > total ? b->max_points : total + total / 4;
        if (pts < 1) pts = 1;
        if (pts > GVOM_MAX_SCAN_POINTS) pts = GVOM_MAX_SCAN_POINTS;
        if (b) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_status(e);
            gvom_batch_destroy(b);
            mp->multi = nullptr;
        }
        const int rc = gvom_batch_create(maps, pts, 0, &mp->multi);
        if (rc != GVOM_OK) return rc;
        b = mp->multi;
    }
    const Geom g = geom_of(mp);
    const int rc = grow_items(b, total * max_segments_per_ray(g, mp->tune.seg_len), st);
    if (rc != GVOM_OK) return rc;
    // with a scan buffer every scan takes a slot; the oldest go first
    int slot[GVOM_MAX_SCAN_BUFFER];
    const bool buffered = mp->cfg.scan_buffer > 0;
    const unsigned long long evict = buffered ? take_slots(mp, k, slot) : 0ull;
    const long long evict_total = evict ? evict_units(mp->s) : 0;

    const int cur = b->cur;
    cudaError_t e = cudaEventSynchronize(b->copied[cur]);
    if (e != cudaSuccess) return cuda_status(e);
    BatchTables h = tables_at(b->h_tables[cur], b->L);
    long long ray_blocks = 0, ray_base = 0;
    for (int j = 0; j < k; ++j) {
        BatchShift& sh = h.sh[j];
        memset(&sh, 0, sizeof(sh));
        sh.s = mp->s;
        sh.g = g;
        h.shift_prefix[j] = 0;
        sh.evict = j == 0 ? evict : 0ull;
        h.evict_prefix[j] = j == 0 ? 0 : evict_total;
        h.ing[j] = ingest_args(mp, pts_dev[j], n[j], stride, mp->tune.seg_len, T_ws + 12 * j, b->w);
        h.ing[j].slot = buffered ? slot[j] : -1;
        h.ing[j].cnt_owner = 0;  // every entry is the same map
        h.ray_prefix[j] = ray_blocks;
        ray_blocks += (n[j] + 255) / 256;
        h.ray_base[j] = ray_base;
        ray_base += n[j];
        h.col_prefix[j] = 0;
        h.tile_prefix[j] = 0;
    }
    h.shift_prefix[k] = 0;
    h.ray_prefix[k] = ray_blocks;
    h.col_prefix[k] = 0;
    h.tile_prefix[k] = 0;
    h.hdr->B = k;
    h.hdr->shift_total = 0;
    h.hdr->ray_blocks = ray_blocks;
    h.hdr->col_tasks = 0;
    h.hdr->tiles = 0;
    h.evict_prefix[k] = evict_total;
    h.hdr->evict_total = evict_total;
    mp->scans += k;
    mp->points_in += total;

    e = cudaMemcpyAsync(b->d_tables, b->h_tables[cur], b->L.bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->copied[cur], st);
    if (e != cudaSuccess) return cuda_status(e);
    b->cur ^= 1;

    IngestArgs shared;
    memset(&shared, 0, sizeof(shared));
    shared.w = b->w;
    MarchShape shape;
    shape.block = mp->tune.march_block;
    shape.blocks_per_sm = mp->tune.march_blocks_per_sm;
    shape.fused = false;
    const long long max_ray_blocks = (b->max_points + 255) / 256 + b->max_maps;
    return cuda_status(launch_batch_update(tables_at(b->d_tables, b->L), b->max_maps, max_ray_blocks, shared, shape,
                                           evict != 0ull, buffered, pow2_window(g), st));
}

}  // namespace gvom
