"""GPU parity of the lookup-table export (the paper's storage format,
Sec. III-A) and of the several-sensors-one-map ingest (Sec. III: many
pointclouds feed one map), against the CPU oracle on the same seeded inputs.
Both are integer / exact work: bit-exact."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_13176_gb300 import build
    build.build()
    import paper_2109_13176_gb300 as m
    return m


def gpu_config(gv, p):
    return gv.make_config(nx=p.nx, ny=p.ny, nz=p.nz, res=p.res, max_range=p.max_range, obs_min_h=p.obs_min_h,
                          obs_max_h=p.obs_max_h, hard_num=p.hard_num, hard_den=p.hard_den, slope_n=p.slope_n,
                          slope_min_px=p.slope_min_px, neg_max_px=p.neg_max_px, neg_thresh=p.neg_thresh)


def to_dev(points):
    return torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()


def compare_voxels(gm, om):
    hits, passes, minz = gm.extract_voxels()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hits.cpu().numpy().view(np.uint32), om.hits)
    np.testing.assert_array_equal(passes.cpu().numpy().view(np.uint32), om.passes)
    np.testing.assert_array_equal(minz.cpu().numpy(), om.minz)


def compare_lut(gm, om, params):
    table, data = oracle.lut(params, om.hits, om.passes, om.minz)
    lut, n_occ, d = gm.export_lut()
    torch.cuda.synchronize()
    assert int(n_occ.item()) == len(data["hits"])
    np.testing.assert_array_equal(lut.cpu().numpy(), table)
    np.testing.assert_array_equal(d["hits"].cpu().numpy().view(np.uint32), data["hits"])
    np.testing.assert_array_equal(d["passes"].cpu().numpy().view(np.uint32), data["passes"])
    np.testing.assert_array_equal(d["minz"].cpu().numpy(), data["minz"])
    return table, data


def test_lut_after_scans_and_shifts(gv):
    # the 256 x 256 x 64 map after shifting scans: the ring offset is not
    # zero, so the export walks logical order over toroidal storage
    cfg, scans = synth.sequence_scans("sequence", n_scans=3)
    params = oracle.OracleParams(nx=cfg.map.nx, ny=cfg.map.ny, nz=cfg.map.nz, res=cfg.map.res,
                                 neg_max_px=int(math.ceil(2.0 / cfg.map.res)))
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    for s in scans:
        om.shift_for_pose(s.vehicle_xyz)
        om.ingest(s.points, s.T_ws)
        gm.update(s.vehicle_xyz, to_dev(s.points), s.T_ws)
    assert any(int(v) % n for v, n in zip(gm.origin, gm.shape))
    table, data = compare_lut(gm, om, params)
    assert len(data["hits"]) > 1000 and (table < -1).any()
    gm.close()


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 5, 7), (37, 29, 13), (64, 33, 32)])
def test_lut_ragged_windows(gv, dims):
    # windows whose voxel counts end mid-block, single-voxel and empty maps
    nx, ny, nz = dims
    rng = np.random.default_rng(sum(dims))
    params = oracle.OracleParams(nx=nx, ny=ny, nz=nz, res=0.2)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    o = (-(nx // 2) + 3, -(ny // 2) - 1, -(nz // 2) + 1)
    om.shift_to(o)
    gm.shift(o)
    compare_lut(gm, om, params)   # empty: every entry -1
    pts = rng.normal(scale=[nx * 0.06, ny * 0.06, nz * 0.04], size=(3000, 3)).astype(np.float32)
    T = np.array([[1.0, 0, 0, 0.05], [0, 1.0, 0, -0.07], [0, 0, 1.0, 0.11]])
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    compare_lut(gm, om, params)
    gm.close()


def test_lut_several_scan_passes(gv):
    # 8.4 M voxels: 8,192 block counts, two passes of the count scan
    rng = np.random.default_rng(5)
    params = oracle.OracleParams(nx=512, ny=512, nz=32, res=0.1)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    o = (-256, -256, -16)
    om.shift_to(o)
    gm.shift(o)
    for k in range(2):
        pts = rng.normal(scale=[8.0, 8.0, 0.5], size=(20000, 3)).astype(np.float32)
        T = np.array([[1.0, 0, 0, 0.3 * k], [0, 1.0, 0, -0.2 * k], [0, 0, 1.0, 0.8]])
        om.ingest(pts, T)
        gm.ingest(to_dev(pts), T)
    table, data = compare_lut(gm, om, params)
    assert len(data["hits"]) > 10000
    gm.close()


def test_lut_capacity_smaller_than_occupied(gv):
    rng = np.random.default_rng(3)
    params = oracle.OracleParams(nx=48, ny=40, nz=24, res=0.2)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    o = (-24, -20, -12)
    om.shift_to(o)
    gm.shift(o)
    pts = rng.normal(scale=[2.5, 2.5, 0.8], size=(6000, 3)).astype(np.float32)
    T = np.array([[1.0, 0, 0, 0.0], [0, 1.0, 0, 0.0], [0, 0, 1.0, 0.5]])
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    table, data = oracle.lut(params, om.hits, om.passes, om.minz)
    n = len(data["hits"])
    cap = n // 3
    lut, n_occ, d = gm.export_lut(capacity=cap)
    torch.cuda.synchronize()
    assert int(n_occ.item()) == n                      # the full count, beyond capacity
    np.testing.assert_array_equal(lut.cpu().numpy(), table)  # the table is whole
    np.testing.assert_array_equal(d["hits"].cpu().numpy().view(np.uint32), data["hits"][:cap])
    np.testing.assert_array_equal(d["minz"].cpu().numpy(), data["minz"][:cap])
    gm.close()


def sensor_pose(th, t):
    c, s = math.cos(th), math.sin(th)
    return np.array([[c, -s, 0.0, t[0]], [s, c, 0.0, t[1]], [0.0, 0.0, 1.0, t[2]]])


@pytest.mark.parametrize("k", [1, 2, 5])
def test_multi_sensor_ingest_equals_sequential_and_oracle(gv, k):
    # k sensors on one vehicle (different mounts, ragged point counts, one
    # empty scan when k = 5) folded into one map in one launch
    rng = np.random.default_rng(40 + k)
    params = oracle.OracleParams(nx=80, ny=72, nz=32, res=0.2)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    seq = gv.VoxelMap(gpu_config(gv, params))
    vehicle = np.array([0.3, -0.4, 0.0])
    for step in range(3):
        vehicle = vehicle + rng.uniform(-0.6, 0.6, 3) * np.array([1, 1, 0.1])
        om.shift_for_pose(vehicle)
        o = om.origin
        gm.shift(o)
        seq.shift(o)
        pts, Ts = [], []
        for j in range(k):
            n = 0 if (k == 5 and j == 3) else int(rng.integers(1, 9000))
            p = rng.normal(scale=[4.0, 4.0, 0.7], size=(n, 3)).astype(np.float32)
            p[::17] = np.nan
            T = sensor_pose(rng.uniform(0, 2 * np.pi), vehicle + np.array([0.4 * j - 0.6, 0.2 * j, 1.0 + 0.1 * j]))
            pts.append(p)
            Ts.append(T)
        for p, T in zip(pts, Ts):
            om.ingest(p, T)
            seq.ingest(to_dev(p), T)
        gm.ingest_multi([to_dev(p) for p in pts], Ts)
        compare_voxels(gm, om)
        compare_voxels(seq, om)
    st, so = gm.stats(), seq.stats()
    for key in ("points_in", "rays_valid", "hits_in_window", "pass_visits"):
        assert st[key] == so[key], key
    assert st["rays_valid"] == om.stats.rays_valid
    out = {kk: v.cpu().numpy() for kk, v in gm.extract_maps().items()}
    ref = {kk: v.cpu().numpy() for kk, v in seq.extract_maps().items()}
    for kk in ("height", "flags", "density", "slope", "roughness"):
        np.testing.assert_array_equal(out[kk], ref[kk], err_msg=kk)
    gm.close()
    seq.close()


def test_multi_sensor_stride4_and_growth(gv):
    # stride-4 points, and a second call with more scans and points than the
    # first (the map's tables grow between calls)
    rng = np.random.default_rng(8)
    params = oracle.OracleParams(nx=40, ny=40, nz=20, res=0.25)
    om = oracle.OracleMap(params, (-20, -20, -10))
    gm = gv.VoxelMap(gpu_config(gv, params))
    gm.shift((-20, -20, -10))
    for k, n in ((2, 500), (11, 7000)):
        pts, Ts = [], []
        for j in range(k):
            p = rng.normal(scale=3.0, size=(n + j, 3)).astype(np.float32)
            Ts.append(sensor_pose(0.3 * j, (0.1 * j, -0.05 * j, 0.8)))
            pts.append(np.concatenate([p, np.ones((len(p), 1), np.float32)], axis=1))
            om.ingest(p, Ts[-1])
        gm.ingest_multi([to_dev(p) for p in pts], Ts)
        compare_voxels(gm, om)
    gm.close()


def test_multi_sensor_rejects_bad_arguments(gv):
    params = oracle.OracleParams(nx=16, ny=16, nz=8, res=0.2)
    gm = gv.VoxelMap(gpu_config(gv, params))
    p = to_dev(np.zeros((10, 3), np.float32))
    bad = sensor_pose(0.0, (0, 0, 0))
    bad[0, 0] = np.nan
    with pytest.raises(gv.GvomError):
        gm.ingest_multi([p, p], [sensor_pose(0.0, (0, 0, 0)), bad])
    with pytest.raises(ValueError):
        gm.ingest_multi([p, to_dev(np.zeros((10, 4), np.float32))], [bad, bad])
    assert gm.stats()["points_in"] == 0
    gm.close()
