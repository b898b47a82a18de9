"""CPU oracle for the G-VOM per-scan map update -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 C statement of the method (G-VOM,
arXiv 2109.13176, Sec. III), loaded here through ctypes. Only the tests, the
smoke check and the CPU-baseline leg of the benchmark use it; the CUDA
library never imports, links or calls anything in this package, and this
package imports nothing from the CUDA side.

`OracleMap` holds a map in logical (window-relative, un-rotated) order:
hits/passes u32 and minz f32 of shape (nx, ny, nz), and the int64 origin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gvom_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: every FP64 operation is rounded on its own, as written
# (GCC contracts a*b+c into a fused multiply-add on Arm unless told not to).
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("res", ctypes.c_double), ("max_range", ctypes.c_double),
        ("obs_min_h", ctypes.c_float), ("obs_max_h", ctypes.c_float),
        ("hard_num", ctypes.c_uint32), ("hard_den", ctypes.c_uint32),
        ("slope_n", ctypes.c_int32), ("slope_min_px", ctypes.c_int32),
        ("neg_max_px", ctypes.c_int32), ("neg_thresh", ctypes.c_float),
    ]


class OrStats(ctypes.Structure):
    _fields_ = [("points_in", ctypes.c_int64), ("rays_valid", ctypes.c_int64),
                ("hits_in_window", ctypes.c_int64), ("pass_visits", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i64p = P(ctypes.c_int64)
            u32p = P(ctypes.c_uint32)
            f32p = P(ctypes.c_float)
            f64p = P(ctypes.c_double)
            u8p = P(ctypes.c_uint8)
            lib.or_origin_for_pose.argtypes = [P(OrParams), f64p, i64p]
            lib.or_clear.argtypes = [P(OrParams), u32p, u32p, f32p]
            lib.or_shift.argtypes = [P(OrParams), i64p, i64p, u32p, u32p, f32p]
            lib.or_traverse_cells.argtypes = [i64p, i64p, i64p, ctypes.c_int64]
            lib.or_traverse_cells.restype = ctypes.c_int64
            lib.or_ingest.argtypes = [P(OrParams), i64p, u32p, u32p, f32p, f32p, ctypes.c_int64,
                                      ctypes.c_int32, f64p, P(OrStats)]
            lib.or_columns.argtypes = [P(OrParams), u32p, u32p, f32p, f32p, f32p, u8p]
            lib.or_slope.argtypes = [P(OrParams), f32p, f32p, f32p]
            lib.or_negative.argtypes = [P(OrParams), f32p, u8p]
            lib.or_extract.argtypes = [P(OrParams), u32p, u32p, f32p, f32p, f32p, u8p, f32p, f32p]
            lib.or_lut.argtypes = [P(OrParams), u32p, u32p, f32p, i64p, u32p, u32p, f32p, ctypes.c_int64]
            lib.or_lut.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class OracleParams:
    """Map parameters; defaults are the readings used for the paper's unnamed
    constants (Sec. III-D)."""
    nx: int = 128
    ny: int = 128
    nz: int = 32
    res: float = 0.2
    max_range: float = 100.0
    obs_min_h: float = 0.3
    obs_max_h: float = 2.0
    hard_num: int = 1
    hard_den: int = 2
    slope_n: int = 5
    slope_min_px: int = 3
    neg_max_px: int = 10
    neg_thresh: float = 0.3

    def c(self) -> OrParams:
        return OrParams(self.nx, self.ny, self.nz, self.res, self.max_range, self.obs_min_h,
                        self.obs_max_h, self.hard_num, self.hard_den, self.slope_n,
                        self.slope_min_px, self.neg_max_px, self.neg_thresh)


def traverse_cells(A, B) -> np.ndarray:
    """Cells met by the segment A->B (1/256-voxel integer endpoints), in order."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.int64)
    b = np.ascontiguousarray(B, dtype=np.int64)
    cap = 64
    while True:
        out = np.zeros((cap, 3), dtype=np.int64)
        n = lib.or_traverse_cells(_ptr(a, ctypes.c_int64), _ptr(b, ctypes.c_int64),
                                  _ptr(out, ctypes.c_int64), cap)
        if n <= cap:
            return out[:n]
        cap = int(n)


def origin_for_pose(params: OracleParams, vehicle_xyz) -> np.ndarray:
    lib = _load()
    pc = params.c()
    v = np.ascontiguousarray(vehicle_xyz, dtype=np.float64)
    out = np.zeros(3, dtype=np.int64)
    lib.or_origin_for_pose(ctypes.byref(pc), _ptr(v, ctypes.c_double), _ptr(out, ctypes.c_int64))
    return out


class OracleMap:
    """A map held in logical order, updated by the C oracle."""

    def __init__(self, params: OracleParams, origin=(0, 0, 0)):
        self.params = params
        self._pc = params.c()
        shape = (params.nx, params.ny, params.nz)
        self.hits = np.zeros(shape, dtype=np.uint32)
        self.passes = np.zeros(shape, dtype=np.uint32)
        self.minz = np.full(shape, np.inf, dtype=np.float32)
        self.origin = np.array(origin, dtype=np.int64)
        self.stats = OrStats()

    def copy(self) -> "OracleMap":
        m = OracleMap(self.params, self.origin)
        m.hits[...] = self.hits
        m.passes[...] = self.passes
        m.minz[...] = self.minz
        return m

    def shift_to(self, new_origin) -> None:
        lib = _load()
        new_o = np.ascontiguousarray(new_origin, dtype=np.int64)
        lib.or_shift(ctypes.byref(self._pc), _ptr(self.origin, ctypes.c_int64),
                     _ptr(new_o, ctypes.c_int64), _ptr(self.hits, ctypes.c_uint32),
                     _ptr(self.passes, ctypes.c_uint32), _ptr(self.minz, ctypes.c_float))
        self.origin = new_o.copy()

    def shift_for_pose(self, vehicle_xyz) -> None:
        self.shift_to(origin_for_pose(self.params, vehicle_xyz))

    def ingest(self, points: np.ndarray, T_ws: np.ndarray) -> OrStats:
        """points: float32 (n, 3) or (n, 4); T_ws: float64 (3, 4) world<-sensor."""
        lib = _load()
        pts = np.ascontiguousarray(points, dtype=np.float32)
        if pts.ndim != 2 or pts.shape[1] not in (3, 4):
            raise ValueError("points must be (n, 3) or (n, 4)")
        T = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(12)
        st = OrStats()
        lib.or_ingest(ctypes.byref(self._pc), _ptr(self.origin, ctypes.c_int64),
                      _ptr(self.hits, ctypes.c_uint32), _ptr(self.passes, ctypes.c_uint32),
                      _ptr(self.minz, ctypes.c_float), _ptr(pts, ctypes.c_float),
                      pts.shape[0], pts.shape[1], _ptr(T, ctypes.c_double), ctypes.byref(st))
        for f, _ in OrStats._fields_:
            setattr(self.stats, f, getattr(self.stats, f) + getattr(st, f))
        return st

    def extract(self) -> dict:
        p = self.params
        return extract(p, self.hits, self.passes, self.minz)


class BufferedOracleMap:
    """The map buffer of Sec. III-A/III-B: the last K per-scan maps. Each
    per-scan map is one scan folded into an empty map at the window of its
    moment, and moves with every later window shift (voxels that leave are
    lost, voxels that enter are empty). The map the products come from
    combines the buffer: hits and passes summed (mod 2^32, like the uint32
    counts), lowest return the minimum."""

    def __init__(self, params: OracleParams, K: int, origin=(0, 0, 0)):
        if K < 1:
            raise ValueError("K >= 1")
        self.params = params
        self.K = K
        self.origin = np.array(origin, dtype=np.int64)
        self.scans: list[OracleMap] = []
        self.stats = OrStats()

    def shift_to(self, new_origin) -> None:
        for m in self.scans:
            m.shift_to(new_origin)
        self.origin = np.array(new_origin, dtype=np.int64)

    def shift_for_pose(self, vehicle_xyz) -> None:
        self.shift_to(origin_for_pose(self.params, vehicle_xyz))

    def ingest(self, points: np.ndarray, T_ws: np.ndarray) -> OrStats:
        m = OracleMap(self.params, self.origin)
        st = m.ingest(points, T_ws)
        self.scans.append(m)
        if len(self.scans) > self.K:
            self.scans.pop(0)
        for f, _ in OrStats._fields_:
            setattr(self.stats, f, getattr(self.stats, f) + getattr(st, f))
        return st

    def _combine(self):
        p = self.params
        shape = (p.nx, p.ny, p.nz)
        h = np.zeros(shape, dtype=np.uint64)
        ps = np.zeros(shape, dtype=np.uint64)
        mz = np.full(shape, np.inf, dtype=np.float32)
        for m in self.scans:
            h += m.hits
            ps += m.passes
            mz = np.minimum(mz, m.minz)
        return h.astype(np.uint32), ps.astype(np.uint32), mz

    @property
    def hits(self):
        return self._combine()[0]

    @property
    def passes(self):
        return self._combine()[1]

    @property
    def minz(self):
        return self._combine()[2]

    def extract(self) -> dict:
        return extract(self.params, *self._combine())


def extract(params: OracleParams, hits, passes, minz) -> dict:
    """All 2D products: height, density, flags, slope, roughness, shape (nx, ny)."""
    lib = _load()
    pc = params.c()
    shape2 = (params.nx, params.ny)
    out = {k: np.zeros(shape2, dtype=np.float32) for k in ("height", "density", "slope", "roughness")}
    out["flags"] = np.zeros(shape2, dtype=np.uint8)
    h = np.ascontiguousarray(hits, dtype=np.uint32)
    ps = np.ascontiguousarray(passes, dtype=np.uint32)
    m = np.ascontiguousarray(minz, dtype=np.float32)
    lib.or_extract(ctypes.byref(pc), _ptr(h, ctypes.c_uint32), _ptr(ps, ctypes.c_uint32),
                   _ptr(m, ctypes.c_float), _ptr(out["height"], ctypes.c_float),
                   _ptr(out["density"], ctypes.c_float), _ptr(out["flags"], ctypes.c_uint8),
                   _ptr(out["slope"], ctypes.c_float), _ptr(out["roughness"], ctypes.c_float))
    return out


def lut(params: OracleParams, hits, passes, minz):
    """Lookup-table encoding (Sec. III-A): (lut int64 (nx,ny,nz), data dict of
    occupied-voxel arrays in linear order)."""
    lib = _load()
    pc = params.c()
    h = np.ascontiguousarray(hits, dtype=np.uint32)
    ps = np.ascontiguousarray(passes, dtype=np.uint32)
    m = np.ascontiguousarray(minz, dtype=np.float32)
    table = np.zeros(h.shape, dtype=np.int64)
    cap = int(np.count_nonzero(h))
    dh = np.zeros(max(cap, 1), np.uint32)
    dp = np.zeros(max(cap, 1), np.uint32)
    dm = np.zeros(max(cap, 1), np.float32)
    n = lib.or_lut(ctypes.byref(pc), _ptr(h, ctypes.c_uint32), _ptr(ps, ctypes.c_uint32), _ptr(m, ctypes.c_float),
                   _ptr(table, ctypes.c_int64), _ptr(dh, ctypes.c_uint32), _ptr(dp, ctypes.c_uint32),
                   _ptr(dm, ctypes.c_float), cap)
    return table, {"hits": dh[:n], "passes": dp[:n], "minz": dm[:n]}


def slope_roughness(params: OracleParams, height: np.ndarray):
    lib = _load()
    pc = params.c()
    h = np.ascontiguousarray(height, dtype=np.float32)
    s = np.zeros_like(h)
    r = np.zeros_like(h)
    lib.or_slope(ctypes.byref(pc), _ptr(h, ctypes.c_float), _ptr(s, ctypes.c_float),
                 _ptr(r, ctypes.c_float))
    return s, r


def negative(params: OracleParams, height: np.ndarray, flags: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    pc = params.c()
    h = np.ascontiguousarray(height, dtype=np.float32)
    f = np.zeros(h.shape, dtype=np.uint8) if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).copy()
    lib.or_negative(ctypes.byref(pc), _ptr(h, ctypes.c_float), _ptr(f, ctypes.c_uint8))
    return f


def columns(params: OracleParams, hits, passes, minz) -> dict:
    lib = _load()
    pc = params.c()
    shape2 = (params.nx, params.ny)
    out = {"height": np.zeros(shape2, np.float32), "density": np.zeros(shape2, np.float32),
           "flags": np.zeros(shape2, np.uint8)}
    h = np.ascontiguousarray(hits, dtype=np.uint32)
    ps = np.ascontiguousarray(passes, dtype=np.uint32)
    m = np.ascontiguousarray(minz, dtype=np.float32)
    lib.or_columns(ctypes.byref(pc), _ptr(h, ctypes.c_uint32), _ptr(ps, ctypes.c_uint32),
                   _ptr(m, ctypes.c_float), _ptr(out["height"], ctypes.c_float),
                   _ptr(out["density"], ctypes.c_float), _ptr(out["flags"], ctypes.c_uint8))
    return out
