/*
 * gvom.h -- C ABI of the GB300 voxel map update (G-VOM, Overbye & Saripalli,
 * arXiv 2109.13176).
 *
 * One map is a fixed-size, robot-centred voxel window (Sec. III-A) held
 * resident in device memory. Each lidar scan is folded into it (Sec. III-C
 * pointcloud processing, combined per Sec. III-D), and the 2D products of
 * Sec. III-D (height, positive obstacles, slope, roughness, negative
 * obstacles) are extracted from it on demand.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers; everything else is host.
 *  - Work is enqueued on the given CUDA stream (NULL = the legacy default
 *    stream) and returns before it runs. Device inputs must stay valid and
 *    unchanged until the stream reaches the call. Calls on one map must be
 *    ordered (one stream, or events between streams).
 *  - Every function returns a gvom_status (0 on success). Arguments are
 *    checked before anything is enqueued, so a call that fails with
 *    GVOM_ERR_INVALID_ARG leaves the map unchanged. GVOM_ERR_CUDA reports a
 *    CUDA error seen while enqueueing; the map's state is then undefined
 *    until gvom_reset, which returns it to an empty, defined state.
 *  - Invalid points are not errors: non-finite points, points at range 0 or
 *    beyond max_range, and points too far from the window to quantise are
 *    dropped and counted in gvom_stats.
 *  - The library owns the map's device state (allocated by gvom_create,
 *    freed by gvom_destroy). The caller owns point, pose and output buffers.
 *
 * Layouts:
 *  - Voxel (ix, iy, iz), 0 <= ix < nx ..., is window-relative: it is the
 *    world voxel origin + (ix, iy, iz). Logical linear index
 *    ((ix * ny) + iy) * nz + iz. 2D products are [ix * ny + iy].
 *  - Points are float32 xyz in the sensor frame, `stride` floats apart (3
 *    for packed xyz, 4 for xyz + padding/intensity).
 *  - T_ws is the row-major 3x4 world-from-sensor transform [R | t], FP64,
 *    finite, with every entry of the rotation part R in [-1, 1] (a rotation;
 *    1e-6 of rounding slack); other poses are rejected as invalid arguments.
 */
#ifndef GVOM_H
#define GVOM_H

#include <stdint.h>

#if defined(__GNUC__)
#define GVOM_API __attribute__((visibility("default")))
#else
#define GVOM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream. */
typedef struct CUstream_st* gvom_stream_t;

typedef enum gvom_status {
    GVOM_OK = 0,
    GVOM_NOT_READY = 1,          /* gvom_pipeline_query: the scan is still in flight */
    GVOM_ERR_INVALID_ARG = -1,   /* a null pointer, size or parameter out of range */
    GVOM_ERR_OUT_OF_MEMORY = -2, /* device allocation failed */
    GVOM_ERR_CUDA = -3,          /* a CUDA call failed */
    GVOM_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    GVOM_ERR_BOUNDS = -5         /* a checked build caught an index out of range */
} gvom_status;

/* Map parameters (Sec. III-A map size and resolution; Sec. III-D obstacle,
 * slope and negative obstacle parameters, which the paper leaves unnamed).
 * Limits: 1 <= nx, ny, nz <= 4096 with nx * ny * nz < 2^31; res > 0;
 * 0 < max_range with max_range / res <= 8192; 0 <= obs_min_h <= obs_max_h;
 * 0 < hard_den <= 65535, hard_num <= hard_den; slope_n odd in [3, 15];
 * 3 <= slope_min_px <= slope_n^2; 1 <= neg_max_px <= 64;
 * 0 <= scan_buffer <= GVOM_MAX_SCAN_BUFFER.
 *
 * Scan buffer (Sec. III-A, III-B: per-scan maps kept in a buffer and
 * combined). With scan_buffer = K > 0 the map also keeps each of its last K
 * scans' own counts and lowest returns (K more copies of the voxel state,
 * 12 bytes per voxel each), moved with the window like the map. Every scan
 * (an empty one too; each scan of gvom_ingest_multi, which then takes at
 * most K) takes the slot of the oldest, whose counts are first taken out of
 * the map (exact: counts subtract) and whose lowest returns are recomputed
 * from the slots that stay. The map thus always equals the combination of
 * its last K scans: counts summed, lowest return the minimum. gvom_reset
 * empties the buffer. K = 0: every scan accumulates (an unbounded buffer). */
#define GVOM_MAX_SCAN_BUFFER 64
typedef struct gvom_config {
    int32_t nx, ny, nz;   /* window size in voxels */
    int32_t scan_buffer;  /* 0: the map accumulates every scan; K in [1, 64]:
                             the map is the combination of its last K scans
                             (Sec. III-A map buffer; see below) */
    double res;           /* voxel edge, metres */
    double max_range;     /* returns beyond this range are dropped, metres */
    float obs_min_h;      /* positive obstacle band above ground, metres */
    float obs_max_h;
    uint32_t hard_num;    /* hard obstacle iff density >= hard_num / hard_den */
    uint32_t hard_den;
    int32_t slope_n;      /* N of the N x N plane fit */
    int32_t slope_min_px; /* defined pixels needed for a fit */
    int32_t neg_max_px;   /* negative obstacle search distance, pixels */
    float neg_thresh;     /* negative obstacle threshold on Delta H, metres */
} gvom_config;

/* Caller-owned device buffers for the 2D products, nx * ny elements each,
 * [ix * ny + iy]. Any pointer may be NULL to skip that product (height is
 * still computed internally when another product needs it).
 *  height:    lowest return of the lowest occupied voxel of the column,
 *             metres (world z); NaN where the column has no return.
 *  density:   H / (H + M) over the column's obstacle voxels, 0 where there
 *             is no positive obstacle.
 *  flags:     bit0 positive obstacle, bit1 hard, bit2 soft, bit3 negative.
 *  slope:     radians; NaN where no plane could be fitted.
 *  roughness: mean squared plane-fit residual, m^2; NaN likewise. */
typedef struct gvom_maps_out {
    float* height_dev;
    float* density_dev;
    uint8_t* flags_dev;
    float* slope_dev;
    float* roughness_dev;
} gvom_maps_out;

/* Largest scan gvom_ingest_scan accepts, in points. */
#define GVOM_MAX_SCAN_POINTS ((int64_t)0x7fffffff)

/* Launch shapes (results never depend on them; speed does, and the
 * autotuner picks them per workload).
 * Traversal: a ray's in-window part is cut into segments of at most
 * seg_len voxel slabs along its major axis, and a persistent grid of
 * march_block-thread blocks (march_blocks_per_sm per SM, 0 = as many as
 * fit) walks them.
 * Extraction of one map (gvom_extract_maps, gvom_update_extract):
 * px_tile is the edge of the pixel pass's tiles (0 = the built-in rule),
 * col_shape the column pass's bulk-copy chunks: 0 = 32 columns x 2 stages,
 * 1 = 16 x 4, 2 = 32 x 3, 3 = 64 x 2 (a shape that does not fit shared
 * memory for the map's nz falls back to 0). The batched and allocation-free
 * extractions keep their built-in shapes.
 * Ingest of one map (gvom_ingest_scan): fused_ingest = 1 has one persistent
 * cooperative kernel (a grid of resident blocks) both list and walk a scan's
 * segments: each warp lists its own 32-point tiles, then walks its own
 * 32-entry chunks of the list as their entries appear; 0 runs the two
 * kernels (list, then walk). The two kernels are faster on the workloads
 * measured; the autotuner times both. The fused
 * kernel serves maps without a scan buffer, with at most 4096 segments per
 * ray, on streams that are not capturing a graph; other ingests use the two
 * kernels whatever this field says.
 * Limits: 1 <= seg_len <= 4096; march_block in {128, 256};
 * 0 <= march_blocks_per_sm <= 32; px_tile 0 or in [4, 64] with the tile and
 * its halo (the larger of neg_max_px and slope_n / 2) fitting 200 KiB of
 * shared memory; 0 <= col_shape <= 3; fused_ingest 0 or 1. */
typedef struct gvom_tuning {
    int32_t seg_len;
    int32_t march_block;
    int32_t march_blocks_per_sm;
    int32_t px_tile;
    int32_t col_shape;
    int32_t fused_ingest;
} gvom_tuning;

/* Counters since gvom_create (or gvom_reset_stats). */
typedef struct gvom_stats {
    int64_t scans;          /* ingest calls */
    int64_t points_in;      /* points offered */
    int64_t rays_valid;     /* points kept (finite, in range, quantisable) */
    int64_t hits_in_window; /* kept points whose endpoint voxel is in the window */
    int64_t pass_visits;    /* pass-count increments (ray/voxel crossings) */
} gvom_stats;

/* Fills *out with defaults: 128 x 128 x 32 voxels at 0.2 m, max range 100 m,
 * obstacle band [0.3, 2.0] m, hard density 1/2, 5 x 5 fit needing 3 pixels,
 * negative search 10 pixels, threshold 0.3 m. */
GVOM_API int gvom_config_default(gvom_config* out);

/* Allocates a map and its device state (12 bytes per voxel plus counters)
 * on the current CUDA device. The map starts empty at origin (0, 0, 0).
 * Synchronises the device once. *out is set to NULL on failure. */
GVOM_API int gvom_create(const gvom_config* cfg, struct gvom_map** out);

/* Frees the map's device state. Synchronises the device. NULL is a no-op. */
GVOM_API void gvom_destroy(struct gvom_map* map);

/* The configuration the map was created with. */
GVOM_API int gvom_get_config(const struct gvom_map* map, gvom_config* out);

/* Default tuning: seg_len 16, march_block 256, blocks per SM as fit,
 * built-in pixel tiles, 32-column 2-stage column chunks, two-kernel ingest. */
GVOM_API int gvom_tuning_default(gvom_tuning* out);

/* Sets / reads the map's tuning (see gvom_tuning). Takes effect from the
 * next ingest. Host-only. */
GVOM_API int gvom_set_tuning(struct gvom_map* map, const gvom_tuning* tuning);
GVOM_API int gvom_get_tuning(const struct gvom_map* map, gvom_tuning* out);

/* Sizes the map's per-scan scratch (16 bytes per point for ray records
 * plus 16 bytes per traversal segment, at most ceil(max(nx,ny,nz)/seg_len)
 * segments per point) for scans of up to max_points points, so that no
 * later ingest has to grow it. Growing waits for `stream` and reallocates.
 * Call it before capturing ingests into a CUDA graph. */
GVOM_API int gvom_reserve(struct gvom_map* map, int64_t max_points, gvom_stream_t stream);

/* Window origin for a vehicle position (Sec. III-A: the origin is a whole
 * number of voxels; Sec. III-D: the combined map is placed at the newest
 * map): out = floor(vehicle_xyz / res) - (nx/2, ny/2, nz/2), FP64. Host-only. */
GVOM_API int gvom_origin_for_pose(const struct gvom_map* map, const double vehicle_xyz[3], int64_t out_origin[3]);

/* Current window origin (world voxel of window voxel (0,0,0)). Host-only. */
GVOM_API int gvom_get_origin(const struct gvom_map* map, int64_t out_origin[3]);

/* Empties the map (and its scan buffer) and places it at `origin`; also
 * the way back to a defined state after GVOM_ERR_CUDA. Stream-ordered. */
GVOM_API int gvom_reset(struct gvom_map* map, const int64_t origin[3], gvom_stream_t stream);

/* Moves the window to new_origin (Sec. III-D combination by index offset):
 * voxels in both windows keep their metrics, voxels entering the window
 * start empty, voxels leaving are dropped. Only the entering slabs are
 * written (the state is stored with toroidal addressing). Stream-ordered. */
GVOM_API int gvom_shift(struct gvom_map* map, const int64_t new_origin[3], gvom_stream_t stream);

/* Folds one scan into the map (Sec. III-C, Sec. III-D combination rule):
 * each point is transformed by T_ws in FP64, each world coordinate
 * w_i = fma(T[i][2], pz, fma(T[i][1], py, fma(T[i][0], px, T[i][3])))
 * with every fused multiply-add rounded once, in this order; points are
 * kept iff finite with 0 < fma(pz, pz, fma(py, py, px * px)) <=
 * max_range^2 (FP64); each coordinate is quantised to 1/256 voxel as
 * round-half-even(fma(w, 256 / res, -256 origin)); the endpoint voxel gains a hit
 * and its lowest-return height is lowered to the point's z (float32);
 * every other window voxel the sensor-to-point segment meets (half-open
 * voxels, exact integer traversal) gains a pass. pts_dev: n points,
 * stride 3 or 4 floats, 16-byte aligned when stride is 4; 0 <= n <=
 * GVOM_MAX_SCAN_POINTS. Stream-ordered; the pose is copied at call time.
 * When n exceeds the scratch sized so far (gvom_reserve), the call first
 * waits for `stream` and grows it. */
GVOM_API int gvom_ingest_scan(struct gvom_map* map, const float* pts_dev, int64_t n, int32_t stride,
                     const double T_ws[12], gvom_stream_t stream);

/* gvom_shift to gvom_origin_for_pose(vehicle_xyz), then gvom_ingest_scan. */
GVOM_API int gvom_update(struct gvom_map* map, const double vehicle_xyz[3], const float* pts_dev, int64_t n,
                int32_t stride, const double T_ws[12], gvom_stream_t stream);

/* Computes the 2D products of Sec. III-D into caller buffers. The map may
 * keep internal scratch for the height map. Stream-ordered. */
GVOM_API int gvom_extract_maps(struct gvom_map* map, const gvom_maps_out* out, gvom_stream_t stream);

/* Allocation-free variant of gvom_extract_maps. The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * at the time they want the maps (a control loop that fixed its memory at
 * start-up, a framework that owns every device buffer through its own pool,
 * or code that may not enter the CUDA allocator), and that therefore cannot
 * hold a gvom_map, whose creation allocates.
 * The caller passes its own voxel grid in logical (window) order -- the
 * layout gvom_extract_voxels writes -- with cfg describing it, and its own
 * output buffers (as for gvom_extract_maps; any may be NULL). Nothing is
 * allocated, freed or copied through the allocator. When out->height_dev is
 * NULL the height map between the two extraction passes is kept in a fixed
 * device array inside the library, 512 x 512 pixels (1 MiB) at most, which
 * every GPU that loads the library holds until the process exits.
 * Limits and errors: cfg must be valid and nx * ny <= 262144, else
 * GVOM_ERR_INVALID_ARG with nothing enqueued. Alignment: when nz is a
 * multiple of 4 the three grids must start on 16-byte boundaries (they are
 * read with 16-byte loads), else on 4-byte ones; the float outputs on
 * 4-byte ones; a misaligned pointer is GVOM_ERR_INVALID_ARG.
 * Set-up: the first call on each device looks the array up (with that
 * device current); make that first call before any stream capture. A first
 * call made while `stream` is capturing returns GVOM_ERR_INVALID_ARG and
 * enqueues nothing. The looked-up address lives until the process exits:
 * do not use the library across a cudaDeviceReset.
 * Sharing: all calls on a device share the array and it keeps the last
 * call's contents (every pixel is rewritten before it is read, so nothing
 * needs clearing); calls that may overlap on the GPU (different streams
 * without ordering between them) and leave height_dev NULL race on it.
 * Stream-ordered. */
GVOM_API int gvom_extract_maps_noalloc(const gvom_config* cfg, const uint32_t* hits_dev, const uint32_t* passes_dev,
                                       const float* minz_dev, const gvom_maps_out* out, gvom_stream_t stream);

/* Copies the voxel state in logical (window-relative) order into caller
 * device buffers of nx*ny*nz elements. minz is +inf where a voxel has no
 * return. Any pointer may be NULL. Stream-ordered. */
GVOM_API int gvom_extract_voxels(struct gvom_map* map, uint32_t* hits_dev, uint32_t* passes_dev, float* minz_dev,
                        gvom_stream_t stream);

/* Checkpoint restore (the paper has no counterpart; for restarting a
 * server or moving a map between processes). Replaces the whole state of a
 * map without a scan buffer: the window is placed at `origin` and its
 * voxels take the caller's arrays, in logical (window) order as
 * gvom_extract_voxels writes them (nx*ny*nz elements each, 4-byte
 * aligned). A checkpoint is gvom_get_origin plus gvom_extract_voxels; the
 * counters of gvom_get_stats are not part of it. Maps with a scan buffer
 * (scan_buffer > 0) cannot be restored this way, because their per-scan
 * slots are not exported: GVOM_ERR_INVALID_ARG. Stream-ordered. */
GVOM_API int gvom_import_state(struct gvom_map* map, const int64_t origin[3], const uint32_t* hits_dev,
                               const uint32_t* passes_dev, const float* minz_dev, gvom_stream_t stream);

/* Folds k scans from different sensors into the map in one per-point pass
 * and one traversal launch (Sec. III: several pointclouds feed one map).
 * Scan j has n[j] points at pts_dev[j] (device, same stride for all, as
 * gvom_ingest_scan) and its own sensor-to-world pose T_ws + 12*j. The
 * window does not move (shift first with gvom_shift). The result equals
 * k calls of gvom_ingest_scan, in any order: counts add and the lowest
 * return is a minimum. 1 <= k <= GVOM_MAX_MULTI_SCANS; the points of all
 * scans together must not exceed GVOM_MAX_SCAN_POINTS. Invalid arguments
 * change nothing. The map keeps the tables this needs between calls and
 * may synchronise the stream when they grow. Stream-ordered. */
#define GVOM_MAX_MULTI_SCANS 4096
GVOM_API int gvom_ingest_multi(struct gvom_map* map, int32_t k, const float* const* pts_dev, const int64_t* n,
                               int32_t stride, const double* T_ws, gvom_stream_t stream);

/* One scan's whole update: gvom_update then gvom_extract_maps, in one call
 * (Sec. III-C, III-D). Arguments, ownership and errors as those two calls;
 * an invalid argument changes nothing. Stream-ordered. */
GVOM_API int gvom_update_extract(struct gvom_map* map, const double vehicle_xyz[3], const float* pts_dev, int64_t n,
                                 int32_t stride, const double T_ws[12], const gvom_maps_out* out,
                                 gvom_stream_t stream);

/* Exports the map in the paper's storage format (Sec. III-A): a lookup
 * table with one int64 entry per voxel, in logical (window) order, holding
 * the voxel's index in the data array if it is occupied (hits >= 1) and
 * -1 - N_m otherwise (N_m = its misses, i.e. pass count); and the data
 * array of the occupied voxels' hits, misses and lowest return, in the
 * same linear order. The number of occupied voxels is written to
 * *n_occupied_dev (device int64); data entries at or beyond data_capacity
 * are not written (call again with larger buffers if *n_occupied_dev
 * exceeds it). Deterministic. Stream-ordered. */
GVOM_API int gvom_export_lut(struct gvom_map* map, int64_t* lut_dev, uint32_t* data_hits_dev,
                             uint32_t* data_passes_dev, float* data_minz_dev, int64_t data_capacity,
                             int64_t* n_occupied_dev, gvom_stream_t stream);

/* Reads the counters. Synchronises with the map's last enqueued work
 * (device-wide synchronisation). Returns GVOM_ERR_TIMEOUT (with *out still
 * filled) if, since creation or the last gvom_reset_stats, a bounded wait
 * inside one of the map's kernels gave up; that kernel's outputs are then
 * incomplete. */
GVOM_API int gvom_get_stats(struct gvom_map* map, gvom_stats* out);

/* Zeroes the counters and the timeout status. Stream-ordered. */
GVOM_API int gvom_reset_stats(struct gvom_map* map, gvom_stream_t stream);

/* ---- Batched update of many maps ---------------------------------------
 * Many independent maps (a fleet, or several sensors each with its own map)
 * updated together: one step shifts every map to the origin of its vehicle
 * position, folds one scan into each (exactly what gvom_update does for one
 * map) and optionally extracts each map's 2D products (exactly what
 * gvom_extract_maps does). All maps of a step run in a handful of kernels
 * whose traversal work is balanced across maps of uneven scan size; with
 * GVOM_BATCH_GRAPH the step is captured once as a CUDA graph and replayed. */
typedef struct gvom_batch gvom_batch;

#define GVOM_BATCH_GRAPH 1 /* capture the step's kernels in a CUDA graph, replay it */

/* Creates a batch context for steps of up to max_maps maps and max_points
 * points in total (sum over the maps of one step). Allocates device tables,
 * the shared per-step scratch (16 bytes per point, plus the segment work
 * list, grown on demand), two pinned staging buffers and, with
 * GVOM_BATCH_GRAPH, an internal capture stream. 1 <= max_maps <= 4096. */
GVOM_API int gvom_batch_create(int32_t max_maps, int64_t max_points, int32_t flags, gvom_batch** out);

/* Frees the context. Synchronises the device. NULL is a no-op. */
GVOM_API void gvom_batch_destroy(gvom_batch* batch);

/* Traversal tuning for the batch (see gvom_tuning); drops a captured graph. */
GVOM_API int gvom_batch_set_tuning(gvom_batch* batch, const gvom_tuning* tuning);

/* One step over maps[0 .. B-1] (distinct maps, any configurations, on the
 * current device): map m shifts to gvom_origin_for_pose(vehicle_xyz + 3m),
 * ingests n[m] points at pts_dev[m] (stride 3 or 4, alignment as for
 * gvom_ingest_scan) with pose T_ws + 12m, and, if outs is not NULL, writes
 * its 2D products to outs[m] (NULL buffers are skipped as in
 * gvom_extract_maps). Results equal B separate gvom_update +
 * gvom_extract_maps calls bit for bit. The sum of n[m] must not exceed the
 * context's max_points. Steps of one context must be issued on one stream
 * (or ordered by events): the device tables are rewritten each step. The
 * first step, or one whose shape needs more scratch, waits for `stream`.
 * Stream-ordered otherwise. Arguments are checked before any map changes. */
GVOM_API int gvom_batch_step(gvom_batch* batch, struct gvom_map* const* maps, int32_t B, const double* vehicle_xyz,
                             const float* const* pts_dev, const int64_t* n, int32_t stride, const double* T_ws,
                             const gvom_maps_out* outs, gvom_stream_t stream);

/* ---- Asynchronous scan pipeline ----------------------------------------
 * The paper runs pointcloud processing and map processing as independent
 * stages (Sec. III). A pipeline drives one map with three streams joined by
 * events: upload (host points to a device staging slot), map (window shift
 * for the vehicle position, ingest, extraction of every product) and
 * download (the products to host). Scan t's upload and scan t-1's download
 * overlap scan t's compute; the map sees its scans in submission order.
 * Three slots of
 * staging and products: a submit blocks on the host until the scan three
 * submissions back has finished. Results equal gvom_update followed by
 * gvom_extract_maps for each scan in order. The map must not be used
 * through other calls while scans are in flight. */
typedef struct gvom_pipeline gvom_pipeline;

/* 1 <= max_points <= GVOM_MAX_SCAN_POINTS / 4 (points per scan). Reserves
 * the map's per-scan scratch for max_points. */
GVOM_API int gvom_pipeline_create(struct gvom_map* map, int64_t max_points, gvom_pipeline** out);
/* Waits for every scan in flight, then frees the pipeline (not the map). */
GVOM_API void gvom_pipeline_destroy(gvom_pipeline* pipeline);
/* Enqueues one scan: n points at pts_host (host memory; page-locked memory
 * lets the copy overlap), stride 3 or 4 floats, pose T_ws, vehicle position
 * vehicle_xyz (as gvom_update). out_host: NULL, or host buffers (page-locked
 * for overlap; NULL members skipped) that receive this scan's products. The
 * buffers must stay valid until the scan has finished. *ticket receives the
 * scan's number (1, 2, ...). */
GVOM_API int gvom_pipeline_submit(gvom_pipeline* pipeline, const double vehicle_xyz[3], const float* pts_host,
                                  int64_t n, int32_t stride, const double T_ws[12], const gvom_maps_out* out_host,
                                  int64_t* ticket);
/* GVOM_OK once the scan's products are in host memory, GVOM_NOT_READY
 * before; never blocks. */
GVOM_API int gvom_pipeline_query(gvom_pipeline* pipeline, int64_t ticket);
/* Blocks until the scan has finished. */
GVOM_API int gvom_pipeline_wait(gvom_pipeline* pipeline, int64_t ticket);
/* The device buffers holding the products of a scan (nx * ny each, layout of
 * gvom_maps_out), valid from its completion until three more scans have
 * been submitted. GVOM_ERR_INVALID_ARG once the slot has been reused. */
GVOM_API int gvom_pipeline_products(gvom_pipeline* pipeline, int64_t ticket, gvom_maps_out* out_dev);

/* Human-readable name of a status code (static storage). */
GVOM_API const char* gvom_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GVOM_H */
