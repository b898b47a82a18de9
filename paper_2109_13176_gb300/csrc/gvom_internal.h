// Internal declarations shared by the CUDA translation units of libgvom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gvom.h"

namespace gvom {

// Window geometry as the kernels see it. Voxel state is stored with
// toroidal addressing: the world voxel W lives at physical slot
// (W mod n) on every axis, so a window shift only rewrites the voxels that
// enter the window. A window-relative voxel c (0 <= c < n) is world voxel
// origin + c, i.e. physical slot (c + r) mod n with r = origin mod n.
struct Geom {
    int nx, ny, nz;
    int rx, ry, rz;
};

// Device state of one map.
struct MapState {
    uint32_t* hits;
    uint32_t* passes;
    float* minz;
    unsigned long long* counters;  // kCounters entries
};

enum Counter { kPointsIn = 0, kRaysValid = 1, kHitsInWindow = 2, kPassVisits = 3, kCounters = 4 };

// Per-scan scratch of the two-phase ingest, owned by the map: one record
// per point (quantised endpoint and its number of traversal segments), the
// segment work list, and its length.
struct RayScratch {
    int4* rays;               // cap_points entries: (qx, qy, qz, nseg)
    uint2* items;             // cap_items entries: (point index, segment index)
    unsigned long long* item_count; // one word
    long long cap_points;
    long long cap_items;
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
};

// Launch shape of the segment walk (tunable).
struct MarchShape {
    int block;                // threads per block
    int blocks_per_sm;        // 0: as many as fit
};

struct ExtractParams {
    Geom g;
    float res;
    float obs_min_h, obs_max_h;
    uint32_t hard_num, hard_den;
    int slope_n, slope_min_px;
    int neg_max_px;
    float neg_thresh;
};

// Whether a configuration is within the documented limits (include/gvom.h).
bool valid_config(const gvom_config* c);

// Counts kernel launches (gvom_kernel_launches).
void count_launch();

// Launchers (return the CUDA error of the launch).
cudaError_t launch_init_state(const MapState& s, long long V, cudaStream_t st);
cudaError_t launch_shift(const MapState& s, const Geom& g_new, const long long d[3], cudaStream_t st);
cudaError_t launch_ingest(const IngestArgs& a, const MarchShape& shape, cudaStream_t st);
// Segments a ray of the given window can have at most, for segment length L.
long long max_segments_per_ray(const Geom& g, int seg_len);
cudaError_t launch_columns(const MapState& s, const ExtractParams& p, float* height, float* density,
                           uint8_t* flags, cudaStream_t st);
cudaError_t launch_slope_negative(const ExtractParams& p, const float* height, float* slope, float* rough,
                                  uint8_t* flags, cudaStream_t st);
cudaError_t launch_gather_voxels(const MapState& s, const Geom& g, uint32_t* hits, uint32_t* passes, float* minz,
                                 cudaStream_t st);

__host__ __device__ inline long long floor_mod(long long a, long long n) {
    long long r = a % n;
    return r < 0 ? r + n : r;
}

}  // namespace gvom
