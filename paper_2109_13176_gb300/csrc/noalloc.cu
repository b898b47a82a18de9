// Allocation-free extraction of the 2D products (include/gvom.h,
// gvom_extract_maps_noalloc).
//
// Some callers cannot allocate device memory when they want the maps: a
// control loop that froze its memory after start-up, a host framework
// that owns every device buffer through its own pool, or code that must
// not call into the CUDA allocator at all. Such callers cannot create a
// gvom_map (gvom_create allocates). This entry point takes their own voxel
// grid and output buffers and allocates nothing. The one intermediate the
// extraction needs, the height map shared by the column pass and the
// plane-fit / cone-search pass, lives in a fixed file-scope device array
// when the caller does not ask for the height itself.
#include <mutex>

#include "gvom_internal.h"

namespace {

// Largest height map the static scratch holds: 512 x 512 pixels (1 MiB).
// Every GPU that loads the library keeps this array until the process ends.
constexpr long long kNoallocMaxPixels = 512LL * 512LL;
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_noalloc_height[kNoallocMaxPixels];

std::mutex g_mu;
float* g_height_ptr[kMaxDevices] = {};

// Device address of g_noalloc_height on the current device. Host code may
// not pass the symbol itself to a kernel (on the host it names a host-side
// shadow, not device memory), so the address is looked up once per device
// with that device current, and cached. The first look-up may load the
// library's device code, which must not happen while `stream` is being
// captured into a graph: that first call is refused then (GVOM_ERR_INVALID_ARG,
// nothing enqueued). A device reset (cudaDeviceReset) invalidates the cached
// address, as it invalidates every map; the library must not be used across one.
int noalloc_height_scratch(cudaStream_t stream, float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return GVOM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GVOM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_height_ptr[dev] == nullptr) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(stream, &cs);
        if (e != cudaSuccess) return GVOM_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return GVOM_ERR_INVALID_ARG;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_height);
        if (e != cudaSuccess) return GVOM_ERR_CUDA;
        g_height_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_height_ptr[dev];
    return GVOM_OK;
}

bool aligned(const void* p, uintptr_t a) { return (((uintptr_t)p) & (a - 1)) == 0; }

}  // namespace

extern "C" int gvom_extract_maps_noalloc(const gvom_config* cfg, const uint32_t* hits_dev, const uint32_t* passes_dev,
                                         const float* minz_dev, const gvom_maps_out* out, gvom_stream_t stream) {
    gvom::NvtxRange nvtx_range("gvom:extract_noalloc");
    if (!gvom::valid_config(cfg) || !hits_dev || !passes_dev || !minz_dev || !out) return GVOM_ERR_INVALID_ARG;
    if ((long long)cfg->nx * cfg->ny > kNoallocMaxPixels) return GVOM_ERR_INVALID_ARG;
    // The column pass reads a grid whose nz is a multiple of 4 with 16-byte
    // loads; other grids and the float outputs need their element alignment.
    const uintptr_t grid_align = (cfg->nz & 3) == 0 ? 16 : 4;
    if (!aligned(hits_dev, grid_align) || !aligned(passes_dev, grid_align) || !aligned(minz_dev, grid_align))
        return GVOM_ERR_INVALID_ARG;
    if (!aligned(out->height_dev, 4) || !aligned(out->density_dev, 4) || !aligned(out->slope_dev, 4) ||
        !aligned(out->roughness_dev, 4))
        return GVOM_ERR_INVALID_ARG;
    float* height = out->height_dev;
    if (height == nullptr) {
        const int rc = noalloc_height_scratch((cudaStream_t)stream, &height);
        if (rc != GVOM_OK) {
            cudaGetLastError();
            return rc;
        }
    }
    gvom::ExtractParams p;
    p.g.nx = cfg->nx;
    p.g.ny = cfg->ny;
    p.g.nz = cfg->nz;
    p.g.rx = p.g.ry = p.g.rz = 0;  // the caller's grid is in window order
    p.res = (float)cfg->res;
    p.obs_min_h = cfg->obs_min_h;
    p.obs_max_h = cfg->obs_max_h;
    p.hard_num = cfg->hard_num;
    p.hard_den = cfg->hard_den;
    p.slope_n = cfg->slope_n;
    p.slope_min_px = cfg->slope_min_px;
    p.neg_max_px = cfg->neg_max_px;
    p.neg_thresh = cfg->neg_thresh;
    p.px_tile = 0;  // built-in shapes
    p.col_shape = 0;
    gvom::MapState s = {};
    s.hits = const_cast<uint32_t*>(hits_dev);  // read only
    s.passes = const_cast<uint32_t*>(passes_dev);
    s.minz = const_cast<float*>(minz_dev);
    s.counters = nullptr;
    const cudaStream_t st = (cudaStream_t)stream;
    // The column pass writes every pixel of the height map, so nothing left
    // in the scratch by an earlier call is read.
    cudaError_t e = gvom::launch_columns(s, p, height, out->density_dev, out->flags_dev, st);
    if (e == cudaSuccess && (out->slope_dev || out->roughness_dev || out->flags_dev))
        e = gvom::launch_slope_negative(p, height, out->slope_dev, out->roughness_dev, out->flags_dev, st);
    return e == cudaSuccess ? GVOM_OK : GVOM_ERR_CUDA;
}
