"""GB300 voxel map update (G-VOM, arXiv 2109.13176) -- Python binding.

A thin ctypes layer over libgvom.so (include/gvom.h). Every step of the map
update runs in the library's CUDA kernels; this module only marshals
arguments. PyTorch supplies device memory (tensors) and streams. There is no
CPU fallback: if the library is not built, or no CUDA device is present,
the calls raise.

Low-level names match the C ABI (gvom_create, gvom_ingest_scan, ...);
`VoxelMap` wraps one map for convenience.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# GVOM_CHECKED=1 in the environment selects the range-checked debug build
# (build.build(checked=True)): same ABI, every kernel index checked.
CHECKED = os.environ.get("GVOM_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "_build", "checked", "libgvom_checked.so") if CHECKED else \
    os.path.join(HERE, "_build", "libgvom.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

GVOM_OK = 0
GVOM_NOT_READY = 1
GVOM_ERR_INVALID_ARG = -1
GVOM_ERR_OUT_OF_MEMORY = -2
GVOM_ERR_CUDA = -3
GVOM_ERR_TIMEOUT = -4
GVOM_ERR_BOUNDS = -5
GVOM_BATCH_GRAPH = 1


class GvomError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class gvom_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("scan_buffer", ctypes.c_int32),
        ("res", ctypes.c_double), ("max_range", ctypes.c_double),
        ("obs_min_h", ctypes.c_float), ("obs_max_h", ctypes.c_float),
        ("hard_num", ctypes.c_uint32), ("hard_den", ctypes.c_uint32),
        ("slope_n", ctypes.c_int32), ("slope_min_px", ctypes.c_int32),
        ("neg_max_px", ctypes.c_int32), ("neg_thresh", ctypes.c_float),
    ]


class gvom_maps_out(ctypes.Structure):
    _fields_ = [("height_dev", ctypes.c_void_p), ("density_dev", ctypes.c_void_p),
                ("flags_dev", ctypes.c_void_p), ("slope_dev", ctypes.c_void_p),
                ("roughness_dev", ctypes.c_void_p)]


class gvom_tuning(ctypes.Structure):
    _fields_ = [("seg_len", ctypes.c_int32), ("march_block", ctypes.c_int32),
                ("march_blocks_per_sm", ctypes.c_int32), ("px_tile", ctypes.c_int32),
                ("col_shape", ctypes.c_int32), ("fused_ingest", ctypes.c_int32)]


class gvom_stats(ctypes.Structure):
    _fields_ = [("scans", ctypes.c_int64), ("points_in", ctypes.c_int64),
                ("rays_valid", ctypes.c_int64), ("hits_in_window", ctypes.c_int64),
                ("pass_visits", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def header_functions() -> list[str]:
    """Names of the entry points the headers under include/ declare."""
    import glob
    names = []
    for h in sorted(glob.glob(os.path.join(INCLUDE, "*.h"))):
        with open(h) as fh:
            text = fh.read()
        names += re.findall(r"^GVOM_API\s+[\w\s\*]+?\b(gvom_\w+)\s*\(", text, flags=re.M)
    return names


def load_library():
    """Loads libgvom.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"the library is not built ({LIB_PATH}); run paper_2109_13176_gb300.build.build("
                               f"checked={CHECKED})")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        d3 = P(ctypes.c_double)
        o3 = P(ctypes.c_int64)
        sig = {
            "gvom_config_default": ([P(gvom_config)], ctypes.c_int),
            "gvom_create": ([P(gvom_config), P(vp)], ctypes.c_int),
            "gvom_destroy": ([vp], None),
            "gvom_get_config": ([vp, P(gvom_config)], ctypes.c_int),
            "gvom_origin_for_pose": ([vp, d3, o3], ctypes.c_int),
            "gvom_get_origin": ([vp, o3], ctypes.c_int),
            "gvom_reset": ([vp, o3, vp], ctypes.c_int),
            "gvom_shift": ([vp, o3, vp], ctypes.c_int),
            "gvom_ingest_scan": ([vp, vp, i64, i32, d3, vp], ctypes.c_int),
            "gvom_update": ([vp, d3, vp, i64, i32, d3, vp], ctypes.c_int),
            "gvom_extract_maps": ([vp, P(gvom_maps_out), vp], ctypes.c_int),
            "gvom_extract_voxels": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "gvom_get_stats": ([vp, P(gvom_stats)], ctypes.c_int),
            "gvom_reset_stats": ([vp, vp], ctypes.c_int),
            "gvom_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "gvom_tuning_default": ([P(gvom_tuning)], ctypes.c_int),
            "gvom_set_tuning": ([vp, P(gvom_tuning)], ctypes.c_int),
            "gvom_get_tuning": ([vp, P(gvom_tuning)], ctypes.c_int),
            "gvom_reserve": ([vp, i64, vp], ctypes.c_int),
            "gvom_batch_create": ([i32, i64, i32, P(vp)], ctypes.c_int),
            "gvom_batch_destroy": ([vp], None),
            "gvom_batch_set_tuning": ([vp, P(gvom_tuning)], ctypes.c_int),
            "gvom_batch_step": ([vp, P(vp), i32, P(ctypes.c_double), P(vp), P(i64), i32, P(ctypes.c_double),
                                 P(gvom_maps_out), vp], ctypes.c_int),
            "gvom_microbench_red": ([vp, i64, i64, ctypes.c_uint32, vp], ctypes.c_int),
            "gvom_microbench_red_coalesced": ([vp, i64, i64, ctypes.c_uint32, vp], ctypes.c_int),
            "gvom_set_walk_marker": ([vp, vp], ctypes.c_int),
            "gvom_extract_maps_noalloc": ([P(gvom_config), vp, vp, vp, P(gvom_maps_out), vp], ctypes.c_int),
            "gvom_kernel_launches": ([], ctypes.c_int64),
            "gvom_ingest_multi": ([vp, i32, P(vp), P(i64), i32, P(ctypes.c_double), vp], ctypes.c_int),
            "gvom_update_extract": ([vp, d3, vp, i64, i32, d3, P(gvom_maps_out), vp], ctypes.c_int),
            "gvom_export_lut": ([vp, vp, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "gvom_pipeline_create": ([vp, i64, P(vp)], ctypes.c_int),
            "gvom_pipeline_destroy": ([vp], None),
            "gvom_pipeline_submit": ([vp, d3, vp, i64, i32, d3, P(gvom_maps_out), P(i64)], ctypes.c_int),
            "gvom_pipeline_query": ([vp, i64], ctypes.c_int),
            "gvom_pipeline_wait": ([vp, i64], ctypes.c_int),
            "gvom_pipeline_products": ([vp, i64, P(gvom_maps_out)], ctypes.c_int),
            "gvom_checked_build": ([], ctypes.c_int),
            "gvom_import_state": ([vp, o3, vp, vp, vp, vp], ctypes.c_int),
            "gvom_selftest_wait_timeout": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
            "gvom_selftest_bounds": ([vp, vp], ctypes.c_int),
            "gvom_selftest_conversions": ([vp, i64, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load_library().gvom_status_string(int(status)).decode()
    except RuntimeError:
        return "library not loaded"


def _check(status: int, what: str) -> None:
    if status != GVOM_OK:
        raise GvomError(status, what)


def _d(vals, n):
    import numpy as np
    a = np.ascontiguousarray(vals, dtype=np.float64).reshape(n)
    return (ctypes.c_double * n).from_buffer_copy(a)


def _i64(vals):
    return (ctypes.c_int64 * 3)(*[int(v) for v in vals])


def _T(T_ws):
    import numpy as np
    t = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(12)
    return (ctypes.c_double * 12).from_buffer_copy(t)


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


# --- C ABI, same names --------------------------------------------------------
def gvom_config_default() -> gvom_config:
    c = gvom_config()
    _check(load_library().gvom_config_default(ctypes.byref(c)), "gvom_config_default")
    return c


def gvom_create(cfg: gvom_config) -> int:
    h = ctypes.c_void_p()
    _check(load_library().gvom_create(ctypes.byref(cfg), ctypes.byref(h)), "gvom_create")
    return h.value


def gvom_destroy(handle: int) -> None:
    load_library().gvom_destroy(handle)


def gvom_get_config(handle: int) -> gvom_config:
    c = gvom_config()
    _check(load_library().gvom_get_config(handle, ctypes.byref(c)), "gvom_get_config")
    return c


def gvom_status_string(status: int) -> str:
    return status_string(status)


def gvom_tuning_default() -> gvom_tuning:
    t = gvom_tuning()
    _check(load_library().gvom_tuning_default(ctypes.byref(t)), "gvom_tuning_default")
    return t


def gvom_set_tuning(handle: int, tuning: gvom_tuning) -> None:
    _check(load_library().gvom_set_tuning(handle, ctypes.byref(tuning)), "gvom_set_tuning")


def gvom_get_tuning(handle: int) -> gvom_tuning:
    t = gvom_tuning()
    _check(load_library().gvom_get_tuning(handle, ctypes.byref(t)), "gvom_get_tuning")
    return t


def gvom_reserve(handle: int, max_points: int, stream=None) -> None:
    _check(load_library().gvom_reserve(handle, int(max_points), _stream_handle(stream)), "gvom_reserve")


def gvom_origin_for_pose(handle: int, vehicle_xyz) -> tuple:
    out = (ctypes.c_int64 * 3)()
    _check(load_library().gvom_origin_for_pose(handle, _d(vehicle_xyz, 3), out), "gvom_origin_for_pose")
    return tuple(out)


def gvom_get_origin(handle: int) -> tuple:
    out = (ctypes.c_int64 * 3)()
    _check(load_library().gvom_get_origin(handle, out), "gvom_get_origin")
    return tuple(out)


def gvom_reset(handle: int, origin, stream=None) -> None:
    _check(load_library().gvom_reset(handle, _i64(origin), _stream_handle(stream)), "gvom_reset")


def gvom_shift(handle: int, new_origin, stream=None) -> None:
    _check(load_library().gvom_shift(handle, _i64(new_origin), _stream_handle(stream)), "gvom_shift")


def _points_args(points):
    import torch
    if not isinstance(points, torch.Tensor) or not points.is_cuda or points.dtype != torch.float32:
        raise TypeError("points must be a CUDA float32 tensor of shape (n, 3) or (n, 4)")
    if points.dim() != 2 or points.shape[1] not in (3, 4) or not points.is_contiguous():
        raise ValueError("points must be contiguous with shape (n, 3) or (n, 4)")
    return points.data_ptr() if points.numel() else None, points.shape[0], points.shape[1]


def gvom_ingest_scan(handle: int, points, T_ws, stream=None) -> None:
    ptr, n, stride = _points_args(points)
    _check(load_library().gvom_ingest_scan(handle, ptr, n, stride, _T(T_ws), _stream_handle(stream)),
           "gvom_ingest_scan")


def gvom_update(handle: int, vehicle_xyz, points, T_ws, stream=None) -> None:
    ptr, n, stride = _points_args(points)
    _check(load_library().gvom_update(handle, _d(vehicle_xyz, 3), ptr, n, stride, _T(T_ws), _stream_handle(stream)),
           "gvom_update")


def gvom_update_extract(handle: int, vehicle_xyz, points, T_ws, outs: dict, stream=None) -> None:
    """Update with one scan (device points) and extract every product into
    outs (dict of device tensors, see VoxelMap.alloc_maps), in one call."""
    ptr, n, stride = _points_args(points)
    o = gvom_maps_out(*(outs[k].data_ptr() if outs.get(k) is not None else None
                        for k in ("height", "density", "flags", "slope", "roughness")))
    _check(load_library().gvom_update_extract(handle, _d(vehicle_xyz, 3), ptr, n, stride, _T(T_ws), ctypes.byref(o),
                                              _stream_handle(stream)), "gvom_update_extract")


def gvom_extract_maps(handle: int, height=None, density=None, flags=None, slope=None, roughness=None,
                      stream=None) -> None:
    out = gvom_maps_out(*(t.data_ptr() if t is not None else None
                          for t in (height, density, flags, slope, roughness)))
    _check(load_library().gvom_extract_maps(handle, ctypes.byref(out), _stream_handle(stream)), "gvom_extract_maps")


def gvom_extract_maps_noalloc(cfg: gvom_config, hits, passes, minz, height=None, density=None, flags=None,
                              slope=None, roughness=None, stream=None) -> None:
    """Allocation-free extraction from a caller-owned voxel grid in window
    order (see include/gvom.h); the height intermediate uses the library's
    fixed device array when `height` is None."""
    out = gvom_maps_out(*(t.data_ptr() if t is not None else None
                          for t in (height, density, flags, slope, roughness)))
    _check(load_library().gvom_extract_maps_noalloc(ctypes.byref(cfg), hits.data_ptr(), passes.data_ptr(),
                                                    minz.data_ptr(), ctypes.byref(out), _stream_handle(stream)),
           "gvom_extract_maps_noalloc")


def gvom_ingest_multi(handle: int, points, T_ws, stream=None) -> None:
    """points: list of k device float32 (n_j, 3|4) tensors; T_ws: k poses."""
    import numpy as np
    k = len(points)
    if k != len(T_ws) or k < 1:
        raise ValueError("one pose per scan, at least one scan")
    stride = int(points[0].shape[1])
    ptrs = (ctypes.c_void_p * k)()
    ns = (ctypes.c_int64 * k)()
    for j, p in enumerate(points):
        if p.dim() != 2 or int(p.shape[1]) != stride:
            raise ValueError("all scans must be (n, 3) or all (n, 4)")
        if p.element_size() != 4 or not p.dtype.is_floating_point or not p.is_contiguous():
            raise ValueError("points must be contiguous float32")
        n = int(p.shape[0])
        ptrs[j] = p.data_ptr() if n else None
        ns[j] = n
    T = np.empty((k, 12), dtype=np.float64)
    for j, t in enumerate(T_ws):
        T[j] = np.asarray(t, dtype=np.float64).reshape(12)
    Tc = (ctypes.c_double * (12 * k)).from_buffer_copy(T)
    _check(load_library().gvom_ingest_multi(handle, k, ptrs, ns, stride, Tc, _stream_handle(stream)),
           "gvom_ingest_multi")


def gvom_export_lut(handle: int, lut, data_hits, data_passes, data_minz, data_capacity: int, n_occupied,
                    stream=None) -> None:
    ptrs = [t.data_ptr() if t is not None else None for t in (lut, data_hits, data_passes, data_minz)]
    _check(load_library().gvom_export_lut(handle, *ptrs, int(data_capacity), n_occupied.data_ptr(),
                                          _stream_handle(stream)), "gvom_export_lut")


def gvom_extract_voxels(handle: int, hits=None, passes=None, minz=None, stream=None) -> None:
    ptrs = [t.data_ptr() if t is not None else None for t in (hits, passes, minz)]
    _check(load_library().gvom_extract_voxels(handle, *ptrs, _stream_handle(stream)), "gvom_extract_voxels")


def gvom_import_state(handle: int, origin, hits, passes, minz, stream=None) -> None:
    """Restores a checkpoint (origin + logical voxel arrays) into a map
    without a scan buffer (see include/gvom.h)."""
    _check(load_library().gvom_import_state(handle, _i64(origin), hits.data_ptr(), passes.data_ptr(), minz.data_ptr(),
                                            _stream_handle(stream)), "gvom_import_state")


def gvom_get_stats(handle: int) -> dict:
    st = gvom_stats()
    _check(load_library().gvom_get_stats(handle, ctypes.byref(st)), "gvom_get_stats")
    return {f: getattr(st, f) for f, _ in gvom_stats._fields_}


def gvom_reset_stats(handle: int, stream=None) -> None:
    _check(load_library().gvom_reset_stats(handle, _stream_handle(stream)), "gvom_reset_stats")


def gvom_batch_create(max_maps: int, max_points: int, flags: int = GVOM_BATCH_GRAPH) -> int:
    h = ctypes.c_void_p()
    _check(load_library().gvom_batch_create(int(max_maps), int(max_points), int(flags), ctypes.byref(h)),
           "gvom_batch_create")
    return h.value


def gvom_batch_destroy(handle: int) -> None:
    load_library().gvom_batch_destroy(handle)


def gvom_batch_set_tuning(handle: int, tuning: gvom_tuning) -> None:
    _check(load_library().gvom_batch_set_tuning(handle, ctypes.byref(tuning)), "gvom_batch_set_tuning")


def gvom_batch_step(handle: int, map_handles, vehicle_xyz, points, T_ws, outs=None, stream=None) -> None:
    """One batched step: map_handles[m] takes the scan points[m] (CUDA float32
    (n, 3|4) tensors, all the same stride) with pose T_ws[m] at vehicle_xyz[m];
    outs: None or a list of dicts of output tensors (see VoxelMap.alloc_maps)."""
    import numpy as np
    B = len(map_handles)
    strides = {p.shape[1] for p in points}
    if len(strides) != 1:
        raise ValueError("all scans of a step must have the same stride")
    maps = (ctypes.c_void_p * B)(*map_handles)
    ptrs, ns = [], []
    for p in points:
        ptr, n, _ = _points_args(p)
        ptrs.append(ptr)
        ns.append(n)
    vx = np.ascontiguousarray(vehicle_xyz, dtype=np.float64).reshape(B * 3)
    T = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(B * 12)
    c_out = None
    if outs is not None:
        c_out = (gvom_maps_out * B)(*[gvom_maps_out(*(o[k].data_ptr() if o.get(k) is not None else None
                                                        for k in ("height", "density", "flags", "slope", "roughness")))
                                      for o in outs])
    _check(load_library().gvom_batch_step(
        handle, maps, B, (ctypes.c_double * (3 * B))(*vx.tolist()), (ctypes.c_void_p * B)(*ptrs),
        (ctypes.c_int64 * B)(*ns), strides.pop(), (ctypes.c_double * (12 * B))(*T.tolist()),
        c_out, _stream_handle(stream)), "gvom_batch_step")


def gvom_pipeline_create(map_handle: int, max_points: int) -> int:
    h = ctypes.c_void_p()
    _check(load_library().gvom_pipeline_create(map_handle, int(max_points), ctypes.byref(h)), "gvom_pipeline_create")
    return h.value


def gvom_pipeline_destroy(handle: int) -> None:
    load_library().gvom_pipeline_destroy(handle)


def _host_outs(outs):
    if outs is None:
        return None
    return gvom_maps_out(*(outs[k].data_ptr() if outs.get(k) is not None else None
                           for k in ("height", "density", "flags", "slope", "roughness")))


def gvom_pipeline_submit(handle: int, vehicle_xyz, points, T_ws, outs=None) -> int:
    """points: CPU float32 (n, 3|4) tensor (pinned for overlap); outs: None or a
    dict of CPU tensors (pinned for overlap) for the products."""
    if points.device.type != "cpu" or points.dtype.itemsize != 4 or not points.is_contiguous():
        raise ValueError("points must be a contiguous float32 CPU tensor")
    n, stride = int(points.shape[0]), int(points.shape[1])
    t = ctypes.c_int64()
    o = _host_outs(outs)
    _check(load_library().gvom_pipeline_submit(handle, _d(vehicle_xyz, 3), points.data_ptr() if n else None, n,
                                               stride, _T(T_ws), ctypes.byref(o) if o is not None else None,
                                               ctypes.byref(t)), "gvom_pipeline_submit")
    return t.value


def gvom_pipeline_query(handle: int, ticket: int) -> bool:
    rc = load_library().gvom_pipeline_query(handle, int(ticket))
    if rc == GVOM_NOT_READY:
        return False
    _check(rc, "gvom_pipeline_query")
    return True


def gvom_pipeline_wait(handle: int, ticket: int) -> None:
    _check(load_library().gvom_pipeline_wait(handle, int(ticket)), "gvom_pipeline_wait")


def gvom_pipeline_products(handle: int, ticket: int) -> dict:
    """Device pointers (ints) of a finished scan's products."""
    o = gvom_maps_out()
    _check(load_library().gvom_pipeline_products(handle, int(ticket), ctypes.byref(o)), "gvom_pipeline_products")
    return {"height": o.height_dev, "density": o.density_dev, "flags": o.flags_dev, "slope": o.slope_dev,
            "roughness": o.roughness_dev}


class Pipeline:
    """Asynchronous scan pipeline over one VoxelMap (see gvom_pipeline_*)."""

    def __init__(self, vmap, max_points: int):
        self.map = vmap
        self.handle = gvom_pipeline_create(vmap.handle, max_points)

    def alloc_host_outs(self):
        import torch
        nx, ny = self.map.shape[:2]
        outs = {k: torch.empty((nx, ny), dtype=torch.float32, pin_memory=True)
                for k in ("height", "density", "slope", "roughness")}
        outs["flags"] = torch.empty((nx, ny), dtype=torch.uint8, pin_memory=True)
        return outs

    def submit(self, vehicle_xyz, points, T_ws, outs=None) -> int:
        return gvom_pipeline_submit(self.handle, vehicle_xyz, points, T_ws, outs)

    def query(self, ticket: int) -> bool:
        return gvom_pipeline_query(self.handle, ticket)

    def wait(self, ticket: int) -> None:
        gvom_pipeline_wait(self.handle, ticket)

    def close(self):
        if getattr(self, "handle", None):
            gvom_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MapBatch:
    """A batch context: steps many VoxelMaps together (see gvom_batch_step)."""

    def __init__(self, max_maps: int, max_points: int, graph: bool = True):
        self.handle = gvom_batch_create(max_maps, max_points, GVOM_BATCH_GRAPH if graph else 0)

    def set_tuning(self, seg_len=16, march_block=256, march_blocks_per_sm=0):
        gvom_batch_set_tuning(self.handle, gvom_tuning(seg_len, march_block, march_blocks_per_sm, 0, 0, 0))

    def step(self, maps, vehicle_xyz, points, T_ws, outs=None, stream=None):
        gvom_batch_step(self.handle, [m.handle for m in maps], vehicle_xyz, points, T_ws, outs, stream)

    def close(self):
        if getattr(self, "handle", None):
            gvom_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gvom_microbench_red(buf, ops: int, seed: int = 1, stream=None) -> None:
    _check(load_library().gvom_microbench_red(buf.data_ptr(), buf.numel(), int(ops), seed & 0xffffffff,
                                              _stream_handle(stream)), "gvom_microbench_red")


def gvom_microbench_red_coalesced(buf, ops: int, seed: int = 1, stream=None) -> None:
    _check(load_library().gvom_microbench_red_coalesced(buf.data_ptr(), buf.numel(), int(ops), seed & 0xffffffff,
                                                        _stream_handle(stream)), "gvom_microbench_red_coalesced")


def gvom_set_walk_marker(handle: int, event=None) -> None:
    """event: a torch.cuda.Event (or None to turn the marker off); see
    include/gvom_microbench.h."""
    ptr = None if event is None else ctypes.c_void_p(int(event.cuda_event))
    _check(load_library().gvom_set_walk_marker(handle, ptr), "gvom_set_walk_marker")


def gvom_kernel_launches() -> int:
    return int(load_library().gvom_kernel_launches())


def gvom_checked_build() -> bool:
    """Whether the loaded library is the range-checked build."""
    return bool(load_library().gvom_checked_build())


def gvom_selftest_wait_timeout(handle: int, spin_limit: int = 1000, stream=None) -> None:
    """Makes a bounded device wait give up (see include/gvom_selftest.h);
    the next gvom_get_stats reports GVOM_ERR_TIMEOUT."""
    _check(load_library().gvom_selftest_wait_timeout(handle, int(spin_limit), _stream_handle(stream)),
           "gvom_selftest_wait_timeout")


def gvom_selftest_conversions(bits, mismatches, stream=None) -> None:
    """bits: device int64 tensor of bit patterns; mismatches: device int64
    tensor of one element (zeroed by the caller); see include/gvom_selftest.h."""
    _check(load_library().gvom_selftest_conversions(bits.data_ptr(), bits.numel(), mismatches.data_ptr(),
                                                    _stream_handle(stream)), "gvom_selftest_conversions")


def gvom_selftest_bounds(handle: int, stream=None) -> None:
    """Checked builds only: sends an out-of-range index through the range
    check; the next gvom_get_stats reports GVOM_ERR_BOUNDS."""
    _check(load_library().gvom_selftest_bounds(handle, _stream_handle(stream)), "gvom_selftest_bounds")


# --- convenience --------------------------------------------------------------
def make_config(nx=128, ny=128, nz=32, res=0.2, **kw) -> gvom_config:
    c = gvom_config_default()
    c.nx, c.ny, c.nz, c.res = nx, ny, nz, res
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class VoxelMap:
    """One device-resident map. Device buffers are torch tensors."""

    def __init__(self, cfg: gvom_config | None = None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("VoxelMap needs a CUDA device")
        self.cfg = cfg if cfg is not None else make_config(**kw)
        self.handle = gvom_create(self.cfg)

    def close(self):
        if getattr(self, "handle", None):
            gvom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.cfg.nx, self.cfg.ny, self.cfg.nz)

    @property
    def origin(self):
        return gvom_get_origin(self.handle)

    def origin_for_pose(self, vehicle_xyz):
        return gvom_origin_for_pose(self.handle, vehicle_xyz)

    def reset(self, origin=(0, 0, 0), stream=None):
        gvom_reset(self.handle, origin, stream)

    def shift(self, new_origin, stream=None):
        gvom_shift(self.handle, new_origin, stream)

    def set_tuning(self, seg_len=16, march_block=256, march_blocks_per_sm=0, px_tile=None, col_shape=None,
                   fused_ingest=None):
        """Walk shape; px_tile / col_shape (extraction shapes) and fused_ingest
        (one kernel lists and walks) keep their current values when not given."""
        cur = gvom_get_tuning(self.handle)
        px = cur.px_tile if px_tile is None else px_tile
        cs = cur.col_shape if col_shape is None else col_shape
        fu = cur.fused_ingest if fused_ingest is None else int(bool(fused_ingest))
        gvom_set_tuning(self.handle, gvom_tuning(seg_len, march_block, march_blocks_per_sm, px, cs, fu))

    def set_extract_tuning(self, px_tile=0, col_shape=0):
        """Extraction shapes only (see gvom_tuning); the walk's stay."""
        cur = gvom_get_tuning(self.handle)
        gvom_set_tuning(self.handle, gvom_tuning(cur.seg_len, cur.march_block, cur.march_blocks_per_sm, px_tile,
                                                 col_shape, cur.fused_ingest))

    def set_fused_ingest(self, on=True):
        """One persistent kernel lists and walks each scan (see gvom_tuning)."""
        cur = gvom_get_tuning(self.handle)
        gvom_set_tuning(self.handle, gvom_tuning(cur.seg_len, cur.march_block, cur.march_blocks_per_sm, cur.px_tile,
                                                 cur.col_shape, int(bool(on))))

    def reserve(self, max_points, stream=None):
        gvom_reserve(self.handle, max_points, stream)

    def ingest(self, points, T_ws, stream=None):
        gvom_ingest_scan(self.handle, points, T_ws, stream)

    def update(self, vehicle_xyz, points, T_ws, stream=None):
        gvom_update(self.handle, vehicle_xyz, points, T_ws, stream)

    def alloc_maps(self, device=None):
        import torch
        dev = device or torch.device("cuda")
        n2 = (self.cfg.nx, self.cfg.ny)
        return {"height": torch.empty(n2, dtype=torch.float32, device=dev),
                "density": torch.empty(n2, dtype=torch.float32, device=dev),
                "flags": torch.empty(n2, dtype=torch.uint8, device=dev),
                "slope": torch.empty(n2, dtype=torch.float32, device=dev),
                "roughness": torch.empty(n2, dtype=torch.float32, device=dev)}

    def alloc_maps_packed(self, device=None, pin_memory=False):
        """The five products as views into one contiguous byte buffer (each
        product 256-byte aligned), so that one copy moves them all. Returns
        (buffer, dict of views). On the CPU, pin_memory gives page-locked
        memory."""
        import torch
        dev = device or torch.device("cuda")
        nx, ny = self.cfg.nx, self.cfg.ny
        layout = [("height", torch.float32, 4), ("density", torch.float32, 4), ("slope", torch.float32, 4),
                  ("roughness", torch.float32, 4), ("flags", torch.uint8, 1)]
        offs, o = [], 0
        for _, _, sz in layout:
            offs.append(o)
            o += (nx * ny * sz + 255) // 256 * 256
        buf = torch.empty(o, dtype=torch.uint8, device=dev, pin_memory=pin_memory and str(dev) == "cpu")
        views = {name: buf[off:off + nx * ny * sz].view(dt).view(nx, ny)
                 for (name, dt, sz), off in zip(layout, offs)}
        return buf, views

    def extract_maps(self, out=None, stream=None):
        out = out if out is not None else self.alloc_maps()
        gvom_extract_maps(self.handle, out.get("height"), out.get("density"), out.get("flags"),
                          out.get("slope"), out.get("roughness"), stream)
        return out

    def extract_voxels(self, stream=None):
        import torch
        shp = self.shape
        hits = torch.empty(shp, dtype=torch.int32, device="cuda")
        passes = torch.empty(shp, dtype=torch.int32, device="cuda")
        minz = torch.empty(shp, dtype=torch.float32, device="cuda")
        gvom_extract_voxels(self.handle, hits, passes, minz, stream)
        return hits, passes, minz

    def update_extract(self, vehicle_xyz, points, T_ws, out, stream=None):
        gvom_update_extract(self.handle, vehicle_xyz, points, T_ws, out, stream)
        return out

    def checkpoint(self, stream=None):
        """(origin, hits, passes, minz): the map's window and its voxels in
        logical order (device tensors); gvom_import_state restores it."""
        return (tuple(self.origin),) + tuple(self.extract_voxels(stream))

    def restore(self, checkpoint, stream=None):
        origin, hits, passes, minz = checkpoint
        gvom_import_state(self.handle, origin, hits, passes, minz, stream)

    def ingest_multi(self, points, T_ws, stream=None):
        gvom_ingest_multi(self.handle, points, T_ws, stream)

    def export_lut(self, capacity=None, stream=None):
        """The lookup table (int64, window shape) and the occupied voxels'
        data (hits, passes, minz) in the paper's storage format. With no
        capacity given, the data arrays are sized from a first counting call."""
        import torch
        lut = torch.empty(self.shape, dtype=torch.int64, device="cuda")
        n_occ = torch.zeros(1, dtype=torch.int64, device="cuda")
        if capacity is None:
            gvom_export_lut(self.handle, lut, None, None, None, 0, n_occ, stream)
            torch.cuda.synchronize()
            capacity = int(n_occ.item())
        dh = torch.empty(capacity, dtype=torch.int32, device="cuda")
        dp = torch.empty(capacity, dtype=torch.int32, device="cuda")
        dm = torch.empty(capacity, dtype=torch.float32, device="cuda")
        gvom_export_lut(self.handle, lut, dh if capacity else None, dp if capacity else None,
                        dm if capacity else None, capacity, n_occ, stream)
        return lut, n_occ, {"hits": dh, "passes": dp, "minz": dm}

    def stats(self):
        return gvom_get_stats(self.handle)

    def reset_stats(self, stream=None):
        gvom_reset_stats(self.handle, stream)
