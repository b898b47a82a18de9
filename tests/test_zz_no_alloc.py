"""The allocation-free extraction entry point (gvom_extract_maps_noalloc).

It serves callers that cannot allocate device memory when they want the maps
(memory fixed at start-up, or owned by their own pool) and so cannot hold a
gvom_map. It must give the same 2D products as gvom_extract_maps on the
same voxel grid, with the height intermediate in the library's fixed device
array, call after call. This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tolerances of the parity tests: exact for height/flags/density,
# 1e-3 rad slope, 1e-4 m^2 roughness
SLOPE_TOL = 1e-3
ROUGH_TOL = 1e-4


@pytest.fixture(scope="module")
def gv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_13176_gb300 import build
    build.build()
    import paper_2109_13176_gb300 as m
    return m


def _compare(a, b):
    np.testing.assert_array_equal(a["flags"], b["flags"])
    np.testing.assert_array_equal(a["density"], b["density"])
    for k, tol in (("slope", SLOPE_TOL), ("roughness", ROUGH_TOL)):
        np.testing.assert_array_equal(np.isnan(a[k]), np.isnan(b[k]))
        m = ~np.isnan(b[k])
        if m.any():
            assert np.max(np.abs(a[k][m] - b[k][m])) <= tol


def _noalloc_maps(gv, cfg, hits, passes, minz):
    n2 = (cfg.nx, cfg.ny)
    out = {"density": torch.full(n2, -1.0, device="cuda"),
           "flags": torch.full(n2, 255, dtype=torch.uint8, device="cuda"),
           "slope": torch.full(n2, -1.0, device="cuda"),
           "roughness": torch.full(n2, -1.0, device="cuda")}
    gv.gvom_extract_maps_noalloc(cfg, hits, passes, minz, height=None, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_extract_maps_on_consecutive_calls(gv):
    # two different maps in a row: the second call reuses the fixed scratch
    scans = [synth.single_scan()]
    cfg_seq, seq = synth.sequence_scans("sequence", n_scans=1)
    scans.append(seq[0])
    specs = [synth.WORKLOADS["single_scan"]["map"], cfg_seq.map]
    for ms, s in zip(specs, scans):
        cfg = gv.make_config(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
        m = gv.VoxelMap(cfg)
        m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
        ref = {k: v.cpu().numpy() for k, v in m.extract_maps().items()}
        hits, passes, minz = m.extract_voxels()
        got = _noalloc_maps(gv, cfg, hits, passes, minz)
        _compare(got, ref)
        # and the same again, with the caller's own height buffer
        h = torch.empty((ms.nx, ms.ny), device="cuda")
        gv.gvom_extract_maps_noalloc(cfg, hits, passes, minz, height=h)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(h.cpu().numpy(), ref["height"])
        m.close()


@pytest.mark.parametrize("nz", [30, 128])
def test_noalloc_matches_extract_maps_on_other_column_paths(gv, nz):
    # nz not a multiple of 4 (the scalar column pass) and nz = 128 (the
    # 32-lane vector pass): the single-scan cloud on a 64 x 64 window
    s = synth.single_scan()
    cfg = gv.make_config(nx=64, ny=64, nz=nz, res=0.2, neg_max_px=10)
    m = gv.VoxelMap(cfg)
    m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    ref = {k: v.cpu().numpy() for k, v in m.extract_maps().items()}
    hits, passes, minz = m.extract_voxels()
    for _ in range(2):
        _compare(_noalloc_maps(gv, cfg, hits, passes, minz), ref)
    assert (ref["flags"] & 1).any() and np.isfinite(ref["slope"]).any()
    m.close()


_CAPTURE_PROBE = r"""
import ctypes, sys, torch
import paper_2109_13176_gb300 as gv
lib = gv.load_library()
cfg = gv.make_config(nx=32, ny=32, nz=8, res=0.2)
hits = torch.zeros(32 * 32 * 8, dtype=torch.int32, device="cuda")
minz = torch.full((32 * 32 * 8,), float("inf"), device="cuda")
flags = torch.empty((32, 32), dtype=torch.uint8, device="cuda")
out = gv.gvom_maps_out(None, None, flags.data_ptr(), None, None)
st = torch.cuda.Stream()
torch.cuda.synchronize()
rc = []
# the first call on this device, made while the stream captures: refused,
# nothing enqueued (the capture ends empty)
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=st):
    rc.append(lib.gvom_extract_maps_noalloc(ctypes.byref(cfg), hits.data_ptr(), hits.data_ptr(), minz.data_ptr(),
                                            ctypes.byref(out), ctypes.c_void_p(st.cuda_stream)))
# outside a capture the same call sets up and runs
rc.append(lib.gvom_extract_maps_noalloc(ctypes.byref(cfg), hits.data_ptr(), hits.data_ptr(), minz.data_ptr(),
                                        ctypes.byref(out), ctypes.c_void_p(st.cuda_stream)))
torch.cuda.synchronize()
print("RC", rc[0], rc[1], int((flags == 0).all()))
"""


def test_noalloc_first_call_during_capture_is_refused(gv, tmp_path):
    # a fresh process, so that this is the first call on the device
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CAPTURE_PROBE], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RC")][-1].split()
    assert int(line[1]) == gv.GVOM_ERR_INVALID_ARG
    assert int(line[2]) == gv.GVOM_OK and int(line[3]) == 1


def test_noalloc_rejects_oversized_maps(gv):
    lib = gv.load_library()
    cfg = gv.make_config(nx=1024, ny=512, nz=8)
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = gv.gvom_maps_out()
    rc = lib.gvom_extract_maps_noalloc(ctypes.byref(cfg), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                       ctypes.byref(out), None)
    assert rc == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_extract_maps_noalloc(ctypes.byref(cfg), None, None, None, ctypes.byref(out), None) == \
        gv.GVOM_ERR_INVALID_ARG
