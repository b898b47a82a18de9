// Asynchronous scan pipeline (include/gvom.h, gvom_pipeline_*): the paper's
// pointcloud processing and map processing run as independent stages
// (Sec. III: the pointcloud node and the map node), here three CUDA streams
// joined by events:
//
//   upload    host points -> a device staging slot            (copy engine)
//   map       window shift + ingest + column pass + plane-fit (SMs)
//             / cone pass into a product slot
//   download  the slot's products -> host                     (copy engine)
//
// Scan t's upload and scan t-1's download overlap scan t's compute. The
// compute of consecutive scans stays on one stream: the ingest and column
// kernels are persistent grids sized to fill every SM, and running another
// scan's pixel pass beside them only delays their resident blocks. Only the
// map stream touches the voxel state, so the map sees its scans strictly in
// order. kDepth slots of staging and products let up to kDepth scans be in
// flight; a submit waits on the host for the scan that last used its slot.
#include <math.h>

#include <new>

#include "gvom_internal.h"

namespace {

constexpr int kDepth = 3;

}  // namespace

struct gvom_pipeline {
    gvom_map* map;
    long long max_points;
    cudaStream_t up, mp, out;
    float* pts[kDepth];
    float* height[kDepth];
    float* density[kDepth];
    float* slope[kDepth];
    float* rough[kDepth];
    uint8_t* flags[kDepth];
    cudaEvent_t uploaded[kDepth], computed[kDepth], done[kDepth];
    long long ticket_of[kDepth];
    long long submitted;
};

extern "C" {

void gvom_pipeline_destroy(gvom_pipeline* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (int k = 0; k < kDepth; ++k) {
        cudaFree(p->pts[k]);
        cudaFree(p->height[k]);
        cudaFree(p->density[k]);
        cudaFree(p->slope[k]);
        cudaFree(p->rough[k]);
        cudaFree(p->flags[k]);
        if (p->uploaded[k]) cudaEventDestroy(p->uploaded[k]);
        if (p->computed[k]) cudaEventDestroy(p->computed[k]);
        if (p->done[k]) cudaEventDestroy(p->done[k]);
    }
    if (p->up) cudaStreamDestroy(p->up);
    if (p->mp) cudaStreamDestroy(p->mp);
    if (p->out) cudaStreamDestroy(p->out);
    delete p;
}

int gvom_pipeline_create(gvom_map* map, int64_t max_points, gvom_pipeline** out) {
    if (!out) return GVOM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!map || max_points < 1 || max_points > GVOM_MAX_SCAN_POINTS / 4) return GVOM_ERR_INVALID_ARG;
    gvom_pipeline* p = new (std::nothrow) gvom_pipeline();
    if (!p) return GVOM_ERR_OUT_OF_MEMORY;
    p->map = map;
    p->max_points = max_points;
    const size_t px = (size_t)map->cfg.nx * map->cfg.ny;
    cudaError_t e = cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->mp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking);
    for (int k = 0; k < kDepth && e == cudaSuccess; ++k) {
        e = cudaMalloc(&p->pts[k], sizeof(float) * 4 * (size_t)max_points);
        if (e == cudaSuccess) e = cudaMalloc(&p->height[k], sizeof(float) * px);
        if (e == cudaSuccess) e = cudaMalloc(&p->density[k], sizeof(float) * px);
        if (e == cudaSuccess) e = cudaMalloc(&p->slope[k], sizeof(float) * px);
        if (e == cudaSuccess) e = cudaMalloc(&p->rough[k], sizeof(float) * px);
        if (e == cudaSuccess) e = cudaMalloc(&p->flags[k], px);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->uploaded[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->computed[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming);
    }
    int rc = gvom::cuda_status(e);
    // the map's per-scan scratch sized once, so no submit grows it
    if (rc == GVOM_OK) rc = gvom_reserve(map, max_points, p->mp);
    if (rc == GVOM_OK) rc = gvom::cuda_status(cudaStreamSynchronize(p->mp));
    if (rc != GVOM_OK) {
        gvom_pipeline_destroy(p);
        cudaGetLastError();
        return rc;
    }
    *out = p;
    return GVOM_OK;
}

int gvom_pipeline_submit(gvom_pipeline* p, const double vehicle_xyz[3], const float* pts_host, int64_t n,
                         int32_t stride, const double T_ws[12], const gvom_maps_out* out_host, int64_t* ticket) {
    gvom::NvtxRange nvtx_range("gvom:pipeline_submit");
    if (!p || !vehicle_xyz || !T_ws || !ticket || n < 0 || n > p->max_points || (stride != 3 && stride != 4) ||
        (n > 0 && !pts_host))
        return GVOM_ERR_INVALID_ARG;
    if (!gvom::valid_pose(T_ws)) return GVOM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(vehicle_xyz[k])) return GVOM_ERR_INVALID_ARG;
    const long long t = p->submitted + 1;
    const int k = (int)(t % kDepth);
    // the scan that last used this slot has finished every stage
    cudaError_t e = p->ticket_of[k] ? cudaEventSynchronize(p->done[k]) : cudaSuccess;
    if (e != cudaSuccess) return gvom::cuda_status(e);

    // upload
    if (n > 0)
        e = cudaMemcpyAsync(p->pts[k], pts_host, sizeof(float) * (size_t)stride * (size_t)n, cudaMemcpyHostToDevice,
                            p->up);
    if (e == cudaSuccess) e = cudaEventRecord(p->uploaded[k], p->up);
    // map stage
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->mp, p->uploaded[k], 0);
    if (e != cudaSuccess) return gvom::cuda_status(e);
    int rc = gvom_update(p->map, vehicle_xyz, p->pts[k], n, stride, T_ws, p->mp);
    if (rc != GVOM_OK) return rc;
    const gvom::ExtractParams ep = gvom::extract_params(p->map);
    e = gvom::launch_columns(p->map->s, ep, p->height[k], p->density[k], p->flags[k], p->mp);
    if (e == cudaSuccess) e = gvom::launch_slope_negative(ep, p->height[k], p->slope[k], p->rough[k], p->flags[k], p->mp);
    if (e == cudaSuccess) e = cudaEventRecord(p->computed[k], p->mp);
    // download stage
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->out, p->computed[k], 0);
    const size_t px = (size_t)p->map->cfg.nx * p->map->cfg.ny;
    if (out_host) {
        const struct {
            void* dst;
            const void* src;
            size_t bytes;
        } copies[5] = {{out_host->height_dev, p->height[k], sizeof(float) * px},
                       {out_host->density_dev, p->density[k], sizeof(float) * px},
                       {out_host->flags_dev, p->flags[k], px},
                       {out_host->slope_dev, p->slope[k], sizeof(float) * px},
                       {out_host->roughness_dev, p->rough[k], sizeof(float) * px}};
        for (int c = 0; c < 5 && e == cudaSuccess; ++c)
            if (copies[c].dst) e = cudaMemcpyAsync(copies[c].dst, copies[c].src, copies[c].bytes, cudaMemcpyDeviceToHost, p->out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->done[k], p->out);
    if (e != cudaSuccess) return gvom::cuda_status(e);
    p->ticket_of[k] = t;
    p->submitted = t;
    *ticket = t;
    return GVOM_OK;
}

// A ticket whose slot has since been taken by a newer scan finished before
// that scan was submitted.
static int pipeline_ticket(gvom_pipeline* p, int64_t ticket, bool block) {
    if (!p || ticket < 1 || ticket > p->submitted) return GVOM_ERR_INVALID_ARG;
    const int k = (int)(ticket % kDepth);
    if (p->ticket_of[k] != ticket) return GVOM_OK;
    const cudaError_t e = block ? cudaEventSynchronize(p->done[k]) : cudaEventQuery(p->done[k]);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return GVOM_NOT_READY;
    }
    return gvom::cuda_status(e);
}

int gvom_pipeline_query(gvom_pipeline* p, int64_t ticket) { return pipeline_ticket(p, ticket, false); }

int gvom_pipeline_wait(gvom_pipeline* p, int64_t ticket) { return pipeline_ticket(p, ticket, true); }

int gvom_pipeline_products(gvom_pipeline* p, int64_t ticket, gvom_maps_out* out_dev) {
    if (!p || !out_dev || ticket < 1 || ticket > p->submitted) return GVOM_ERR_INVALID_ARG;
    const int k = (int)(ticket % kDepth);
    if (p->ticket_of[k] != ticket) return GVOM_ERR_INVALID_ARG;
    out_dev->height_dev = p->height[k];
    out_dev->density_dev = p->density[k];
    out_dev->flags_dev = p->flags[k];
    out_dev->slope_dev = p->slope[k];
    out_dev->roughness_dev = p->rough[k];
    return GVOM_OK;
}

}  // extern "C"
