"""GPU parity of the scan buffer (Sec. III-A / III-B: the map is the
combination of its last K scans) against the oracle's buffer of per-scan
maps, on the plain path, the several-sensor path and the batched path.
Counts and lowest returns bit-exact; products as in the plain parity tests."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def gpu_config(gv, p, K):
    return gv.make_config(nx=p.nx, ny=p.ny, nz=p.nz, res=p.res, max_range=p.max_range, obs_min_h=p.obs_min_h,
                          obs_max_h=p.obs_max_h, hard_num=p.hard_num, hard_den=p.hard_den, slope_n=p.slope_n,
                          slope_min_px=p.slope_min_px, neg_max_px=p.neg_max_px, neg_thresh=p.neg_thresh,
                          scan_buffer=K)


def to_dev(points):
    return torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()


def compare_voxels(gm, om):
    hits, passes, minz = gm.extract_voxels()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hits.cpu().numpy().view(np.uint32), om.hits)
    np.testing.assert_array_equal(passes.cpu().numpy().view(np.uint32), om.passes)
    np.testing.assert_array_equal(minz.cpu().numpy(), om.minz)


def compare_products(gm, om):
    out = {k: v.cpu().numpy() for k, v in gm.extract_maps().items()}
    ref = om.extract()
    np.testing.assert_array_equal(out["height"], ref["height"])
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    np.testing.assert_allclose(out["density"], ref["density"], rtol=1e-6, atol=0)
    for k, tol in (("slope", SLOPE_TOL), ("roughness", ROUGH_TOL)):
        a, b = out[k], ref[k]
        np.testing.assert_array_equal(np.isnan(a), np.isnan(b), err_msg=k)
        m = ~np.isnan(b)
        if m.any():
            assert np.max(np.abs(a[m] - b[m])) <= tol, k


def pose(th, t):
    c, s = math.cos(th), math.sin(th)
    return np.array([[c, -s, 0.0, t[0]], [s, c, 0.0, t[1]], [0.0, 0.0, 1.0, t[2]]])


def rough_scan(rng, n, centre):
    pts = np.concatenate([rng.normal(scale=[4, 4, 0.6], size=(n, 3)),
                          rng.uniform(-6, 6, size=(n // 6, 3))]).astype(np.float32)
    return pts, pose(rng.uniform(0, 2 * np.pi), centre)


def test_buffer_full_size_sequence(gv):
    # the 256 x 256 x 64 map, shifting every scan, buffer of 3 scans
    cfg, scans = synth.sequence_scans("sequence", n_scans=6)
    params = oracle.OracleParams(nx=cfg.map.nx, ny=cfg.map.ny, nz=cfg.map.nz, res=cfg.map.res,
                                 neg_max_px=int(math.ceil(2.0 / cfg.map.res)))
    om = oracle.BufferedOracleMap(params, K=3)
    gm = gv.VoxelMap(gpu_config(gv, params, 3))
    for s in scans:
        om.shift_for_pose(s.vehicle_xyz)
        om.ingest(s.points, s.T_ws)
        gm.update(s.vehicle_xyz, to_dev(s.points), s.T_ws)
        compare_voxels(gm, om)
    compare_products(gm, om)
    gm.close()


@pytest.mark.parametrize("K", [1, 2, 5, 64])
def test_buffer_sequences_with_shifts_and_empty_scans(gv, K):
    rng = np.random.default_rng(100 + K)
    params = oracle.OracleParams(nx=72, ny=64, nz=24, res=0.2, neg_max_px=6)
    om = oracle.BufferedOracleMap(params, K=K)
    gm = gv.VoxelMap(gpu_config(gv, params, K))
    vehicle = np.zeros(3)
    for step in range(9):
        vehicle = vehicle + rng.uniform(-0.7, 0.7, 3) * np.array([1, 1, 0.2])
        if step == 6:
            vehicle = vehicle + np.array([30.0, 0, 0])   # past the window: every slot empties
        n = 0 if step == 4 else int(rng.integers(500, 6000))
        pts, T = rough_scan(rng, n, vehicle + np.array([0, 0, 1.0]))
        om.shift_for_pose(vehicle)
        om.ingest(pts, T)
        gm.update(vehicle, to_dev(pts), T)
        compare_voxels(gm, om)
    compare_products(gm, om)
    gm.close()


def test_buffer_reset_and_plain_shift(gv):
    rng = np.random.default_rng(7)
    params = oracle.OracleParams(nx=40, ny=40, nz=20, res=0.25)
    gm = gv.VoxelMap(gpu_config(gv, params, 2))
    for _ in range(3):
        pts, T = rough_scan(rng, 2000, (0.0, 0.0, 1.0))
        gm.ingest(to_dev(pts), T)
    gm.reset((-20, -20, -10))
    om = oracle.BufferedOracleMap(params, K=2, origin=(-20, -20, -10))
    for step in range(4):
        pts, T = rough_scan(rng, 1500, (0.3 * step, 0.0, 1.0))
        om.ingest(pts, T)
        gm.ingest(to_dev(pts), T)
        o = (-20 + step, -20 - step, -10 + (step % 2))
        om.shift_to(o)
        gm.shift(o)
        compare_voxels(gm, om)
    gm.close()


def test_buffer_with_several_sensors(gv):
    # two sensors per call, K = 5: the slots wrap in the middle of a call
    rng = np.random.default_rng(21)
    params = oracle.OracleParams(nx=64, ny=64, nz=24, res=0.2)
    om = oracle.BufferedOracleMap(params, K=5)
    gm = gv.VoxelMap(gpu_config(gv, params, 5))
    vehicle = np.zeros(3)
    for step in range(6):
        vehicle = vehicle + rng.uniform(-0.5, 0.5, 3) * np.array([1, 1, 0.1])
        om.shift_for_pose(vehicle)
        gm.shift(om.origin)
        pts, Ts = [], []
        for j in range(2):
            p, T = rough_scan(rng, int(rng.integers(0, 5000)), vehicle + np.array([0.5 * j, 0, 1.0]))
            pts.append(p)
            Ts.append(T)
            om.ingest(p, T)
        gm.ingest_multi([to_dev(p) for p in pts], Ts)
        compare_voxels(gm, om)
    with pytest.raises(gv.GvomError):
        gm.ingest_multi([to_dev(pts[0])] * 6, Ts[:1] * 6)   # more scans than the buffer holds
    gm.close()


@pytest.mark.parametrize("graph", [True, False])
def test_buffer_in_batch_steps(gv, graph):
    # a batch of buffered and unbuffered maps equals the same maps updated
    # one by one, over more steps than the buffers hold
    rng = np.random.default_rng(33)
    specs = [(48, 40, 24, 0.2, 2), (64, 64, 32, 0.25, 0), (40, 44, 20, 0.2, 3), (32, 32, 16, 0.3, 1)]
    batch_maps, solo_maps = [], []
    for nx, ny, nz, res, K in specs:
        kw = dict(nx=nx, ny=ny, nz=nz, res=res, neg_max_px=int(math.ceil(2.0 / res)), scan_buffer=K)
        batch_maps.append(gv.VoxelMap(**kw))
        solo_maps.append(gv.VoxelMap(**kw))
    mb = gv.MapBatch(len(specs), 40000, graph=graph)
    outs = [m.alloc_maps() for m in batch_maps]
    centres = [np.zeros(3) for _ in specs]
    for step in range(6):
        vxyz, pts, Ts = [], [], []
        for i in range(len(specs)):
            centres[i] = centres[i] + rng.uniform(-0.5, 0.5, 3) * np.array([1, 1, 0.1])
            p, T = rough_scan(rng, int(rng.integers(0, 8000)), centres[i] + np.array([0, 0, 1.0]))
            vxyz.append(centres[i].copy())
            pts.append(to_dev(p))
            Ts.append(T)
        mb.step(batch_maps, vxyz, pts, Ts, outs=outs)
        for i, m in enumerate(solo_maps):
            m.update(vxyz[i], pts[i], Ts[i])
        torch.cuda.synchronize()
        for a, b in zip(batch_maps, solo_maps):
            for x, y in zip(a.extract_voxels(), b.extract_voxels()):
                np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    for i, m in enumerate(solo_maps):
        ref = m.extract_maps()
        for k in ref:
            np.testing.assert_array_equal(outs[i][k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=k)
    mb.close()
    for m in batch_maps + solo_maps:
        m.close()
