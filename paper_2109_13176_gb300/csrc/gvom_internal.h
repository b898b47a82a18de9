// Internal declarations shared by the CUDA translation units of libgvom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gvom.h"

namespace gvom {

// An NVTX range around one phase of a call (visible in Nsight tools as
// gvom:<phase> on the calling thread; no cost worth measuring without a tool
// attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Programmatic dependent launch. The path's kernels are launched with
// launch_pdl: a kernel waits until its predecessor's memory is visible
// before touching it (pdl_wait, first thing), and lets its own successor
// start launching once its block has done its main work (pdl_done), so the
// successor's launch overlaps this kernel's tail rather than its body.
// Launched without the attribute, both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_done() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Window geometry as the kernels see it. Voxel state is stored with
// toroidal addressing: the world voxel W lives at physical slot
// (W mod n) on every axis, so a window shift only rewrites the voxels that
// enter the window. A window-relative voxel c (0 <= c < n) is world voxel
// origin + c, i.e. physical slot (c + r) mod n with r = origin mod n.
struct Geom {
    int nx, ny, nz;
    int rx, ry, rz;
};

// Device state of one map. A map with a scan buffer (scan_buffer = K > 0)
// also keeps its last K scans' own states in a ring of K slots ([K][V] per
// array, same toroidal addressing); the main arrays always hold their
// combination (counts summed, lowest return the minimum).
struct MapState {
    uint32_t* hits;
    uint32_t* passes;
    float* minz;
    unsigned long long* counters;  // kCounters entries
    uint32_t* ring_hits;           // K * V, or null
    uint32_t* ring_passes;
    float* ring_minz;
    int ring_K;                    // 0: no buffer
    uint32_t V;                    // voxels of the window (< 2^31)
};

// counters[kStatus]: bit kStatusTimeout -- a bounded device wait of one of
// the map's kernels gave up (gvom_get_stats: GVOM_ERR_TIMEOUT); bit
// kStatusBounds -- a checked build caught an index out of range
// (GVOM_ERR_BOUNDS).
enum Counter { kPointsIn = 0, kRaysValid = 1, kHitsInWindow = 2, kPassVisits = 3, kStatus = 4, kCounters = 5 };
constexpr unsigned long long kStatusTimeout = 1ull;
constexpr unsigned long long kStatusBounds = 2ull;

#ifdef __CUDACC__
// Range check of a computed index. In a checked build (GVOM_CHECKED), an
// index at or past n records kStatusBounds in the status word (when there
// is one) and the caller skips the access; otherwise it is always true and
// costs nothing.
__device__ __forceinline__ bool in_bounds(unsigned long long i, unsigned long long n, unsigned long long* counters) {
#ifdef GVOM_CHECKED
    if (i < n) return true;
    if (counters) atomicOr(counters + kStatus, kStatusBounds);
    return false;
#else
    (void)i;
    (void)n;
    (void)counters;
    return true;
#endif
}
#endif

// Per-scan scratch of the two-phase ingest, owned by the map: one record
// per point (quantised endpoint and its number of traversal segments), the
// segment work list, and its length.
struct RayScratch {
    int4* rays;               // cap_points entries: (qx, qy, qz, nseg)
    // cap_items entries: (point index, segment index) as uint2 for the
    // two-kernel ingest; on plain maps 16 bytes per entry are allocated, and
    // the fused ingest uses them as int4 (qx, qy, qz, epoch << 12 | segment)
    uint2* items;
    unsigned long long* item_count; // kScratchWords words (ScratchWord)
    long long cap_points;
    long long cap_items;
};

// Words of RayScratch::item_count. Two-kernel ingest: the list's length and
// the walk's blocks done with it. Fused ingest, each word on a 128-byte line
// of its own (its warps poll them while others add to them): list entries
// reserved, point tiles listed, blocks done. Every kernel leaves its words at
// zero when it ends.
enum ScratchWord {
    kListLen = 0, kListBlocksDone = 1,
    kFReserved = 16, kFTilesDone = 32, kFBlocksDone = 48,
    kScratchWords = 64
};

// Per-scan arguments of the ingest kernels (passed by value).
struct IngestArgs {
    const float* pts;
    long long n;
    int stride;
    int seg_len;              // major-axis voxel slabs per traversal segment
    double T[12];
    double S;            // 256 * (1 / res): 1/256-voxel units per metre
    double neg_o256[3];  // -256 * origin (exact)
    double r2max;
    Geom g;
    MapState s;
    RayScratch w;
    int slot;            // ring slot this scan also goes to, -1: none
    int cnt_owner;       // batch entry whose counters this entry's visits go to
    unsigned int epoch;  // fused ingest: this scan's list tag, 1 .. kFusedEpochs - 1
};

// Fused ingest: list entries carry the scan's tag in their top 20 bits and
// the segment index in the low 12 (so at most kFusedMaxSegments per ray).
constexpr unsigned int kFusedEpochs = 1u << 20;
constexpr long long kFusedMaxSegments = 1 << 12;

// Launch shape of the segment walk (tunable).
struct MarchShape {
    int block;                // threads per block
    int blocks_per_sm;        // 0: as many as fit
    bool fused;               // one persistent kernel lists and walks (plain maps, no slot)
};

struct ExtractParams {
    Geom g;
    float res;
    float obs_min_h, obs_max_h;
    uint32_t hard_num, hard_den;
    int slope_n, slope_min_px;
    int neg_max_px;
    float neg_thresh;
    int px_tile;    // pixel tile edge, 0: the built-in rule (gvom_tuning.px_tile)
    int col_shape;  // column pass chunk shape code, 0: 32 columns x 2 stages (gvom_tuning.col_shape)
};

// ---- Batched update of many maps (tables filled by the host each step) ----

// Window shift of one map in a batch step.
struct BatchShift {
    MapState s;
    Geom g;          // the new window
    int d[3];        // new - old origin (|d_k| < n_k unless whole)
    int whole;       // 1: clear the whole map
    unsigned long long evict;  // ring slots emptied after the shift (bit j: slot j)
};

// Extraction of one map in a batch step.
struct BatchExtract {
    MapState s;
    ExtractParams p;
    float* height;   // never null (the map's scratch when the caller asked for none)
    float* density;
    uint8_t* flags;
    float* slope;
    float* rough;
};

// Step totals, read by the kernels from device memory so that a captured
// graph replays with new counts.
struct BatchHeader {
    int B;
    int pad;
    long long shift_total;   // warp units of the shift kernel
    long long ray_blocks;    // 256-point blocks of the per-point pass
    long long col_tasks;     // 64-column warp tasks of the column pass
    long long tiles;         // pixel tiles of the plane-fit / cone pass
    long long evict_total;   // 1024-voxel units of the eviction kernel
};

// Device pointers into one allocation of a batch's tables.
struct BatchTables {
    BatchHeader* hdr;
    IngestArgs* ing;          // [max_maps]
    BatchShift* sh;           // [max_maps]
    BatchExtract* ex;         // [max_maps]
    long long* shift_prefix;  // [max_maps + 1]
    long long* ray_prefix;    // [max_maps + 1], in 256-point blocks
    long long* ray_base;      // [max_maps], first ray record of each map
    long long* col_prefix;    // [max_maps + 1], in tasks
    long long* tile_prefix;   // [max_maps + 1]
    int4* sensors;            // [max_maps], written on the device
    long long* evict_prefix;  // [max_maps + 1], in 1024-voxel units
};

constexpr int kColTask = 32;       // columns per unit of the batched column pass (a bulk-copy chunk)
long long shift_units(const Geom& g, const int d[3], int whole);
long long tiles_of(const ExtractParams& p);
int tile_halo(const ExtractParams& p);
// evict: run the eviction kernel after the shifts; slots: some map of the
// step writes a ring slot.
// pow2: every map of the step has power-of-two extents.
cudaError_t launch_batch_update(const BatchTables& t, int max_maps, long long max_ray_blocks, const IngestArgs& shared,
                                const MarchShape& shape, bool evict, bool slots, bool pow2, cudaStream_t st);
// Whether every extent of the window is a power of two.
bool pow2_window(const Geom& g);
long long evict_units(const MapState& s);
// zmax > 0: every map's nz is a multiple of 4 and at most 256, zmax the
// largest (the bulk-copy column pass); 0: the vector/scalar column pass.
// px_smem: the pixel pass's shared memory per block, the largest
// slope_negative_smem of the step's maps.
cudaError_t launch_batch_extract(const BatchTables& t, int max_maps, size_t px_smem, int zmax, cudaStream_t st);
size_t slope_negative_smem(const ExtractParams& p);

// Lookup-table export (export.cu): blocks of the count / write kernels and
// the three launches (count, scan, write).
long long lut_blocks(long long V);
cudaError_t launch_export_lut(const MapState& s, const Geom& g, unsigned int* counts, long long* n_occupied,
                              long long* lut, uint32_t* dh, uint32_t* dp, float* dm, long long cap, cudaStream_t st);

// Raises a kernel's dynamic shared memory limit to at least `bytes` on the
// current device, calling the runtime only the first time a device needs a
// larger limit (cache: one slot per device ordinal, 64 devices at most).
cudaError_t allow_smem(const void* kernel, std::atomic<int>* cache, size_t bytes);

// Whether a configuration is within the documented limits (include/gvom.h).
bool valid_config(const gvom_config* c);

// Counts kernel launches (gvom_kernel_launches); graph replays add the
// number of kernels the graph holds.
void count_launch(long long n = 1);

// Launchers (return the CUDA error of the launch).
// Empties the map and, with a buffer, every ring slot.
cudaError_t launch_init_state(const MapState& s, long long V, cudaStream_t st);
// Empties the ring slots of `mask`, taking their counts out of the map and
// recomputing the lowest return where an emptied slot held it.
cudaError_t launch_evict(const MapState& s, unsigned long long mask, cudaStream_t st);
cudaError_t launch_shift(const MapState& s, const Geom& g_new, const long long d[3], cudaStream_t st);
// marker: a caller event recorded between the per-point pass and the walk (or null).
cudaError_t launch_ingest(const IngestArgs& a, const MarchShape& shape, cudaStream_t st,
                          cudaEvent_t marker = nullptr);
// Segments a ray of the given window can have at most, for segment length L.
long long max_segments_per_ray(const Geom& g, int seg_len);
cudaError_t launch_columns(const MapState& s, const ExtractParams& p, float* height, float* density,
                           uint8_t* flags, cudaStream_t st);
cudaError_t launch_slope_negative(const ExtractParams& p, const float* height, float* slope, float* rough,
                                  uint8_t* flags, cudaStream_t st);
cudaError_t launch_gather_voxels(const MapState& s, const Geom& g, uint32_t* hits, uint32_t* passes, float* minz,
                                 cudaStream_t st);
cudaError_t launch_scatter_voxels(const MapState& s, const Geom& g, const uint32_t* hits, const uint32_t* passes,
                                  const float* minz, cudaStream_t st);

__host__ __device__ inline long long floor_mod(long long a, long long n) {
    long long r = a % n;
    return r < 0 ? r + n : r;
}

}  // namespace gvom

// One map (include/gvom.h): configuration, window origin (host copy, updated
// in enqueue order), device state and per-scan scratch.
struct gvom_map {
    gvom_config cfg;
    long long origin[3];
    gvom::MapState s;
    gvom::RayScratch w;     // per-scan ray records and segment work list
    float* height_scratch;  // nx * ny, used when the caller asks for no height
    unsigned int* lut_counts;  // per-block counts of the lookup-table export
    struct gvom_batch* multi;  // tables for gvom_ingest_multi (created on first use)
    int buf_head;                    // ring slot of the next scan
    unsigned long long buf_occupied; // ring slots holding a scan
    gvom_tuning tune;
    cudaEvent_t walk_marker;         // gvom_set_walk_marker (null: none)
    unsigned int fused_epoch;        // tag of the last fused ingest's list entries
    long long scans;
    long long points_in;
    int device;
};

namespace gvom {
Geom geom_of(const gvom_map* m);
long long voxels(const gvom_map* m);
int cuda_status(cudaError_t e);
bool valid_origin(const int64_t o[3]);
ExtractParams extract_params(const gvom_map* m);
bool valid_pose(const double T[12]);
bool valid_tuning(const gvom_tuning* t);
// Takes the ring slots of the map's next k scans (k <= K): returns the
// occupied ones to empty first; slots[j] receives scan j's slot (-1 for a
// map without a buffer).
unsigned long long take_slots(gvom_map* m, int k, int* slots);
// gvom_ingest_multi after validation (batch.cu).
int ingest_multi(gvom_map* mp, int k, const float* const* pts_dev, const int64_t* n, int stride, const double* T_ws,
                 cudaStream_t st);
}  // namespace gvom
