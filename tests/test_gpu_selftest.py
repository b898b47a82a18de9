"""Failure detection on the GPU without a fault (the paper has none of it):

- a bounded device wait that nothing completes gives up after its
  iteration limit, gvom_get_stats reports GVOM_ERR_TIMEOUT, and after
  gvom_reset_stats the same map updates exactly like the oracle again;
- the range-checked build (GVOM_CHECKED) runs the path on small maps with
  no violation and results equal to the oracle's, and an index one past the
  map sent through its range check is reported as GVOM_ERR_BOUNDS with the
  access skipped.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_13176_gb300 import build
    build.build()
    import paper_2109_13176_gb300 as m
    return m


def stats_status(gv, m):
    st = gv.gvom_stats()
    return gv.load_library().gvom_get_stats(m.handle, ctypes.byref(st))


def test_bounded_wait_gives_up_and_the_map_stays_usable(gv):
    s = synth.single_scan()
    ms = synth.WORKLOADS["single_scan"]["map"]
    m = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    assert gv.load_library().gvom_selftest_wait_timeout(m.handle, 0, None) == gv.GVOM_ERR_INVALID_ARG
    gv.gvom_selftest_wait_timeout(m.handle, 2000)
    torch.cuda.synchronize()
    assert stats_status(gv, m) == gv.GVOM_ERR_TIMEOUT
    m.reset_stats()
    assert stats_status(gv, m) == gv.GVOM_OK
    # the context and the map work as before
    om = oracle.OracleMap(oracle.OracleParams(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res))
    om.shift_for_pose(s.vehicle_xyz)
    om.ingest(s.points, s.T_ws)
    m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    hits, passes, minz = (t.cpu().numpy() for t in m.extract_voxels())
    np.testing.assert_array_equal(hits.view(np.uint32), om.hits)
    np.testing.assert_array_equal(passes.view(np.uint32), om.passes)
    assert stats_status(gv, m) == gv.GVOM_OK
    m.close()


def test_unchecked_build_refuses_the_bounds_selftest(gv):
    if gv.gvom_checked_build():
        pytest.skip("this process loaded the checked build")
    m = gv.VoxelMap(nx=16, ny=16, nz=8, res=0.2)
    assert gv.load_library().gvom_selftest_bounds(m.handle, None) == gv.GVOM_ERR_INVALID_ARG
    assert stats_status(gv, m) == gv.GVOM_OK
    m.close()


_CHECKED_RUN = r"""
import ctypes, math, sys
import numpy as np, torch
import oracle, synth
from paper_2109_13176_gb300 import build
build.build(checked=True)
import paper_2109_13176_gb300 as gv
assert gv.gvom_checked_build()
lib = gv.load_library()

def status(m):
    st = gv.gvom_stats()
    return lib.gvom_get_stats(m.handle, ctypes.byref(st))

def same_as_oracle(m, om):
    h, p, z = (t.cpu().numpy() for t in m.extract_voxels())
    assert np.array_equal(h.view(np.uint32), om.hits) and np.array_equal(p.view(np.uint32), om.passes)
    assert np.array_equal(z, om.minz)
    out = {k: v.cpu().numpy() for k, v in m.extract_maps().items()}
    ref = om.extract()
    assert np.array_equal(out["flags"], ref["flags"]) and np.array_equal(out["height"], ref["height"], equal_nan=True)

scan = synth.single_scan()
cfg, seq = synth.sequence_scans("sequence", n_scans=2, stride=4)
checked = 0
# a power-of-two window and an odd-sized one (both walk variants, all column passes)
for dims, buf in (((128, 128, 32), 0), ((100, 90, 30), 0), ((96, 96, 32), 2)):
    p = oracle.OracleParams(nx=dims[0], ny=dims[1], nz=dims[2], res=0.2)
    om = oracle.BufferedOracleMap(p, 2) if buf else oracle.OracleMap(p)
    m = gv.VoxelMap(nx=dims[0], ny=dims[1], nz=dims[2], res=0.2, scan_buffer=buf)
    for s in [scan] + seq:
        om.shift_for_pose(s.vehicle_xyz)
        om.ingest(s.points, s.T_ws)
        m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
        same_as_oracle(m, om)
    V = dims[0] * dims[1] * dims[2]
    lut = torch.empty(V, dtype=torch.int64, device="cuda")
    d = [torch.empty(V, dtype=t, device="cuda") for t in (torch.int32, torch.int32, torch.float32)]
    n_occ = torch.zeros(1, dtype=torch.int64, device="cuda")
    gv.gvom_export_lut(m.handle, lut, d[0], d[1], d[2], V, n_occ)
    torch.cuda.synchronize()
    assert status(m) == gv.GVOM_OK, status(m)
    checked += 1
    m.close()
# a batch step of three maps
maps = [gv.VoxelMap(nx=64, ny=64, nz=32, res=0.2) for _ in range(3)]
batch = gv.MapBatch(3, 3 * len(scan.points), graph=True)
pts = [torch.from_numpy(scan.points).cuda()] * 3
outs = [mm.alloc_maps() for mm in maps]
batch.step(maps, [scan.vehicle_xyz] * 3, pts, [scan.T_ws] * 3, outs=outs)
torch.cuda.synchronize()
assert all(status(mm) == gv.GVOM_OK for mm in maps)
# the range check itself: one past the last voxel is caught, nothing is written
mm = maps[0]
before = [t.clone() for t in mm.extract_voxels()]
gv.gvom_selftest_bounds(mm.handle)
torch.cuda.synchronize()
assert status(mm) == gv.GVOM_ERR_BOUNDS
assert all(torch.equal(a, b) for a, b in zip(before, mm.extract_voxels()))
mm.reset_stats()
assert status(mm) == gv.GVOM_OK
batch.close()
for mm in maps:
    mm.close()
print("CHECKED_OK", checked)
"""


def test_checked_build_runs_clean_and_catches_an_out_of_range_index(gv):
    env = dict(os.environ, GVOM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", _CHECKED_RUN], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-3000:])
    assert "CHECKED_OK 3" in r.stdout


def test_checkpoint_restore_continues_like_the_original(gv):
    # a map checkpointed after two scans and restored into a fresh map
    # (another window origin first) continues bit for bit like the original
    cfg, scans = synth.sequence_scans("sequence", n_scans=4, stride=3)
    ms = cfg.map
    kw = dict(nx=96, ny=80, nz=32, res=ms.res)
    a = gv.VoxelMap(**kw)
    for s in scans[:2]:
        a.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    ck = a.checkpoint()
    b = gv.VoxelMap(**kw)
    b.shift((7, -3, 2))
    b.restore(ck)
    assert tuple(b.origin) == tuple(a.origin)
    for s in scans[2:]:
        for m in (a, b):
            m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    for x, y in zip(a.extract_voxels(), b.extract_voxels()):
        assert torch.equal(x, y)
    oa, ob = a.extract_maps(), b.extract_maps()
    for k in oa:
        np.testing.assert_array_equal(oa[k].cpu().numpy(), ob[k].cpu().numpy())
    # a map with a scan buffer cannot be restored from a plain checkpoint
    c = gv.VoxelMap(scan_buffer=2, **kw)
    o = (ctypes.c_int64 * 3)(*ck[0])
    assert gv.load_library().gvom_import_state(c.handle, o, ck[1].data_ptr(), ck[2].data_ptr(), ck[3].data_ptr(),
                                               None) == gv.GVOM_ERR_INVALID_ARG
    for m in (a, b, c):
        m.close()


def test_integer_pipe_conversions_match_cuda(gv):
    # the per-point pass's float -> double, double -> int and double -> float
    # conversions (bit-field arithmetic, round to nearest, ties to even)
    # against CUDA's own conversions: random bit patterns and the edges
    rng = np.random.default_rng(2109)
    parts = [rng.integers(0, 2 ** 63, size=200_000, dtype=np.int64),
             -rng.integers(0, 2 ** 63, size=200_000, dtype=np.int64)]
    # ties and near-ties of the integer rounding: k + 0.5, k + 0.5 +- 1 ulp, |k| < 2^30
    k = rng.integers(-(2 ** 30) + 2, 2 ** 30 - 2, size=50_000).astype(np.float64)
    for v in (k + 0.5, np.nextafter(k + 0.5, np.inf), np.nextafter(k + 0.5, -np.inf), k, -k - 0.5,
              np.array([0.5, -0.5, 1.5, -1.5, 2.5, 0.49999999999999994, -0.0, 0.0, 2 ** 30 - 0.5,
                        -(2 ** 30) + 0.5])):
        parts.append(np.asarray(v, dtype=np.float64).view(np.int64))
    # ties of the float rounding: a float plus half its ulp, and neighbours
    f = rng.uniform(-1e6, 1e6, size=50_000).astype(np.float32)
    f64 = f.astype(np.float64)
    ulp = np.abs(np.nextafter(f, np.float32(np.inf)).astype(np.float64) - f64)
    for v in (f64 + ulp / 2, np.nextafter(f64 + ulp / 2, np.inf), np.nextafter(f64 + ulp / 2, -np.inf)):
        parts.append(v.view(np.int64))
    # extremes of the float range and subnormals, as doubles and as floats
    ext = np.array([3.4028234663852886e38, 3.4028235677973366e38, 3.4028236e38, 1.1754943508222875e-38,
                    1.1754942e-38, 1e-45, 7e-46, 1e-300, 1e300, 65504.0, 1.0, -1.0], dtype=np.float64)
    parts.append(ext.view(np.int64))
    fl = np.array([1e-45, 1e-40, 1.1754942e-38, 1.1754944e-38, 3.4e38, -0.0, 0.0, 1.0], dtype=np.float32)
    parts.append(fl.view(np.uint32).astype(np.int64))
    bits = torch.from_numpy(np.concatenate(parts)).cuda()
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    gv.gvom_selftest_conversions(bits, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 0
