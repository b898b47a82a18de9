"""GPU parity: the CUDA map update (through the C ABI) against the CPU oracle
on the same seeded inputs.

Bar (the method's stated tolerances): hits, passes, lowest-return heights,
the height map, and all flags bit-exact; counters equal; density within
1e-6 relative (it is computed by the same FP64 division on both sides, so
it is expected exact); slope within 1e-3 rad and roughness within 1e-4 m^2
(the device fits the plane in FP32, the oracle in FP64), with the same
pixels defined on both sides.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SLOPE_TOL = 1e-3
ROUGH_TOL = 1e-4
DENSITY_RTOL = 1e-6


@pytest.fixture(scope="module")
def gv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_13176_gb300 import build
    build.build()
    import paper_2109_13176_gb300 as m
    return m


def params_for(ms, **kw):
    d = dict(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    d.update(kw)
    return oracle.OracleParams(**d)


def gpu_config(gv, p: oracle.OracleParams):
    return gv.make_config(nx=p.nx, ny=p.ny, nz=p.nz, res=p.res, max_range=p.max_range, obs_min_h=p.obs_min_h,
                          obs_max_h=p.obs_max_h, hard_num=p.hard_num, hard_den=p.hard_den, slope_n=p.slope_n,
                          slope_min_px=p.slope_min_px, neg_max_px=p.neg_max_px, neg_thresh=p.neg_thresh)


def to_dev(points):
    return torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()


def compare_voxels(gm, om):
    hits, passes, minz = gm.extract_voxels()
    torch.cuda.synchronize()
    h = hits.cpu().numpy().view(np.uint32)
    p = passes.cpu().numpy().view(np.uint32)
    z = minz.cpu().numpy()
    assert tuple(gm.origin) == tuple(int(v) for v in om.origin)
    np.testing.assert_array_equal(h, om.hits)
    np.testing.assert_array_equal(p, om.passes)
    np.testing.assert_array_equal(z, om.minz)  # values: -0.0 == +0.0


def compare_products(gm, om):
    out = {k: v.cpu().numpy() for k, v in gm.extract_maps().items()}
    ref = om.extract()
    np.testing.assert_array_equal(out["height"], ref["height"])
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    np.testing.assert_allclose(out["density"], ref["density"], rtol=DENSITY_RTOL, atol=0)
    for k, tol in (("slope", SLOPE_TOL), ("roughness", ROUGH_TOL)):
        a, b = out[k], ref[k]
        np.testing.assert_array_equal(np.isnan(a), np.isnan(b), err_msg=k)
        m = ~np.isnan(b)
        if m.any():
            assert np.max(np.abs(a[m] - b[m])) <= tol, k
    return out, ref


def compare_stats(gm, om):
    st = gm.stats()
    assert st["rays_valid"] == om.stats.rays_valid
    assert st["hits_in_window"] == om.stats.hits_in_window
    assert st["pass_visits"] == om.stats.pass_visits
    assert st["points_in"] == om.stats.points_in


def new_map(gv, params, fused=False):
    """A device map for the oracle's parameters; fused: one kernel lists and
    walks each scan's segments (tuning fused_ingest)."""
    gm = gv.VoxelMap(gpu_config(gv, params))
    if fused:
        gm.set_fused_ingest(True)
    return gm


def run_sequence(gv, params, scans, stride=3, check_each=True, products_each=False, fused_too=False):
    """Feeds the scans to the oracle and to a device map (and, with fused_too,
    to a second device map on the fused ingest, checked the same way)."""
    om = oracle.OracleMap(params)
    gms = [new_map(gv, params)] + ([new_map(gv, params, fused=True)] if fused_too else [])
    for s in scans:
        assert tuple(gms[0].origin_for_pose(s.vehicle_xyz)) == tuple(int(v) for v in oracle.origin_for_pose(params, s.vehicle_xyz))
        om.shift_for_pose(s.vehicle_xyz)
        om.ingest(s.points, s.T_ws)
        pts = s.points
        if stride == 4:
            pts = np.concatenate([pts, np.ones((len(pts), 1), np.float32)], axis=1)
        for gm in gms:
            gm.update(s.vehicle_xyz, to_dev(pts), s.T_ws)
            if check_each:
                compare_voxels(gm, om)
            if products_each:
                compare_products(gm, om)
    for gm in gms[1:]:
        compare_stats(gm, om)
    return gms[0], om


def gen_workers():
    import os
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def test_single_scan(gv):
    s = synth.single_scan()
    params = params_for(synth.WORKLOADS["single_scan"]["map"])
    gm, om = run_sequence(gv, params, [s], fused_too=True)
    compare_stats(gm, om)
    out, ref = compare_products(gm, om)
    assert np.count_nonzero(out["flags"] & 2) > 0 and np.count_nonzero(out["flags"] & 8) > 0


def test_single_scan_stride4(gv):
    s = synth.single_scan()
    params = params_for(synth.WORKLOADS["single_scan"]["map"])
    gm, om = run_sequence(gv, params, [s], stride=4, fused_too=True)
    compare_products(gm, om)


def test_sequence_all_scans(gv):
    # the sequence workload as the benchmark times it: all 20 scans into the
    # 256 x 256 x 64 map, shifting every scan; state and every product after
    # each scan
    cfg, scans = synth.sequence_scans("sequence", workers=gen_workers())
    assert len(scans) == 20
    params = params_for(cfg.map)
    gm, om = run_sequence(gv, params, scans, products_each=True, fused_too=True)
    compare_stats(gm, om)


def test_high_speed_scans_full_size(gv):
    # the 512 x 512 x 64 map at 0.1 m: all 40 consecutive scans the benchmark
    # times (12 voxels apart), state and every product after each
    cfg, scans = synth.sequence_scans("high_speed", n_scans=40, stride=1, seed=synth.SEEDS["high_speed"],
                                      workers=gen_workers())
    assert len(scans) == 40
    params = params_for(cfg.map)
    gm, om = run_sequence(gv, params, scans, products_each=True, fused_too=True)
    compare_stats(gm, om)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n", [0, 1, 31, 33, 255, 257, 1000, 4099])
def test_ragged_point_counts(gv, n, fused):
    rng = np.random.default_rng(1000 + n)
    params = oracle.OracleParams(nx=40, ny=36, nz=20, res=0.2)
    pts = rng.normal(scale=3.0, size=(n, 3)).astype(np.float32)
    if n > 4:
        pts[::5] *= 0.0            # zero-range points
        pts[1::7, 0] = np.nan      # non-finite
        pts[2::11] *= 40.0         # beyond max range, some
    th = 0.7
    T = np.array([[math.cos(th), -math.sin(th), 0.01, 0.3], [math.sin(th), math.cos(th), -0.02, -0.1],
                  [-0.01, 0.02, 1.0, 1.5]])
    om = oracle.OracleMap(params)
    gm = new_map(gv, params, fused)
    o = oracle.origin_for_pose(params, (0.1, -0.2, 0.0))
    om.shift_to(o)
    gm.shift(o)
    om.ingest(pts, T)
    gm.ingest(to_dev(pts.reshape(-1, 3)), T)
    compare_voxels(gm, om)
    compare_stats(gm, om)
    compare_products(gm, om)


@pytest.mark.parametrize("fused", [False, True])
def test_sensor_outside_window_and_far_points(gv, fused):
    rng = np.random.default_rng(77)
    params = oracle.OracleParams(nx=24, ny=20, nz=10, res=0.25)
    pts = rng.uniform(-30, 30, size=(3000, 3)).astype(np.float32)
    T = np.array([[1.0, 0, 0, -9.0], [0, 1.0, 0, 2.0], [0, 0, 1.0, 0.4]])
    om = oracle.OracleMap(params, (0, 0, 0))
    gm = new_map(gv, params, fused)
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    compare_voxels(gm, om)
    compare_stats(gm, om)


@pytest.mark.parametrize("fused", [False, True])
def test_shift_sequences_match(gv, fused):
    # random shifts (including ones past the window) of an accumulated map
    rng = np.random.default_rng(5)
    params = oracle.OracleParams(nx=30, ny=26, nz=14, res=0.2)
    om = oracle.OracleMap(params)
    gm = new_map(gv, params, fused)
    o = np.array([-15, -13, -7])
    om.shift_to(o)
    gm.shift(o)
    T = np.array([[1.0, 0, 0, 0.05], [0, 1.0, 0, 0.03], [0, 0, 1.0, 0.2]])
    for step in range(12):
        pts = rng.normal(scale=2.5, size=(2000, 3)).astype(np.float32)
        T[:, 3] = (o[:3] + np.array([15, 13, 7])) * params.res + rng.uniform(0, 0.2, 3)
        om.ingest(pts, T)
        gm.ingest(to_dev(pts), T)
        d = rng.integers(-4, 5, 3)
        if step == 5:
            d = np.array([31, 0, 0])   # past the window: everything clears
        if step == 8:
            d = np.array([0, 0, -14])
        o = o + d
        om.shift_to(o)
        gm.shift(o)
        compare_voxels(gm, om)


def test_accumulated_products_after_many_scans(gv):
    # a longer sequence on a small map: products after each of several scans
    cfg, scans = synth.sequence_scans("sequence", n_scans=3, stride=5)
    params = params_for(cfg.map, nx=96, ny=96, nz=32)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    for s in scans:
        om.shift_for_pose(s.vehicle_xyz)
        om.ingest(s.points, s.T_ws)
        gm.update(s.vehicle_xyz, to_dev(s.points), s.T_ws)
        compare_voxels(gm, om)
        compare_products(gm, om)


def test_extract_from_random_state(gv):
    # 2D products from an arbitrary voxel state (dense random columns), so
    # every branch of the column, plane and cone code runs
    rng = np.random.default_rng(9)
    params = oracle.OracleParams(nx=70, ny=45, nz=24, res=0.2, neg_max_px=6)
    om = oracle.OracleMap(params)
    gm = gv.VoxelMap(gpu_config(gv, params))
    # build the state through scans of a rough synthetic cloud so that the
    # device state is produced by the device path
    for k in range(6):
        pts = np.concatenate([rng.normal(scale=[4, 4, 0.6], size=(3000, 3)),
                              rng.uniform(-6, 6, size=(500, 3))]).astype(np.float32)
        T = np.array([[1.0, 0, 0, rng.uniform(-1, 1)], [0, 1.0, 0, rng.uniform(-1, 1)], [0, 0, 1.0, 1.0]])
        om.ingest(pts, T)
        gm.ingest(to_dev(pts), T)
    o = (-35, -22, -12)
    om.shift_to(o)
    gm.shift(o)
    for k in range(4):
        pts = np.concatenate([rng.normal(scale=[5, 5, 0.5], size=(4000, 3)),
                              rng.uniform(-7, 7, size=(800, 3))]).astype(np.float32)
        T = np.array([[1.0, 0, 0, rng.uniform(-1, 1)], [0, 1.0, 0, rng.uniform(-1, 1)], [0, 0, 1.0, 1.2]])
        om.ingest(pts, T)
        gm.ingest(to_dev(pts), T)
    compare_voxels(gm, om)
    out, ref = compare_products(gm, om)
    assert np.isfinite(ref["slope"]).sum() > 100


def test_points_at_the_range_limit(gv):
    # points on, just inside and just outside max_range, in many directions:
    # the device decides the range filter like the oracle's FP64 test
    rng = np.random.default_rng(31)
    params = oracle.OracleParams(nx=40, ny=40, nz=24, res=0.25, max_range=3.0)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    base = (d * 3.0).astype(np.float32)
    pts = np.concatenate([base, np.nextafter(base, np.float32(0)), np.nextafter(base, np.float32(10)),
                          np.float32([[3, 0, 0], [0, -3, 0], [0, 0, 3], [3.0000002, 0, 0], [2.9999998, 0, 0]])])
    T = np.array([[1.0, 0, 0, 0.1], [0, 1.0, 0, -0.05], [0, 0, 1.0, 0.3]])
    om = oracle.OracleMap(params, (-20, -20, -12))
    gm = gv.VoxelMap(gpu_config(gv, params))
    gm.shift((-20, -20, -12))
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    compare_voxels(gm, om)
    compare_stats(gm, om)
    assert 0 < om.stats.rays_valid < len(pts)


def holes_and_blocks(rng, nx, ny, res, n):
    """Ground points over the whole window with round holes (undefined
    pixels) and raised blocks, so that the cone search meets ground of
    several heights at several distances."""
    ex, ey = nx * res, ny * res
    x = rng.uniform(-ex / 2, ex / 2, n)
    y = rng.uniform(-ey / 2, ey / 2, n)
    z = 0.25 * np.sin(x / 3.0) + 0.2 * np.cos(y / 4.0) + rng.normal(0, 0.02, n)
    keep = np.ones(n, bool)
    for _ in range(max(4, int(ex * ey / 45))):
        cx, cy, r = rng.uniform(-ex / 2, ex / 2), rng.uniform(-ey / 2, ey / 2), rng.uniform(0.3, 2.6)
        keep &= (x - cx) ** 2 + (y - cy) ** 2 > r * r
    for _ in range(max(3, int(ex * ey / 70))):
        cx, cy = rng.uniform(-ex / 2, ex / 2), rng.uniform(-ey / 2, ey / 2)
        m = (np.abs(x - cx) < rng.uniform(0.5, 2)) & (np.abs(y - cy) < rng.uniform(0.5, 2))
        z[m] += rng.uniform(0.2, 0.6)
    return np.stack([x[keep], y[keep], z[keep]], 1).astype(np.float32)


@pytest.mark.parametrize("nx,ny,halo", [(430, 410, 20), (200, 180, 13), (160, 150, 30)])
def test_pixel_tiles_for_large_search_distances(gv, nx, ny, halo):
    # search distances above 12 px: two-warp-wide tiles when the map has
    # enough of them (430 x 410, 20 px: 24-px tiles, ragged on both axes),
    # else 16-px tiles (a small map at 13 px; 30 px)
    rng = np.random.default_rng(halo)
    params = oracle.OracleParams(nx=nx, ny=ny, nz=16, res=0.1, neg_max_px=halo)
    o = (-(nx // 2), -(ny // 2), -8)
    om = oracle.OracleMap(params, o)
    gm = gv.VoxelMap(gpu_config(gv, params))
    gm.shift(o)
    pts = holes_and_blocks(rng, nx, ny, 0.1, int(1.1 * nx * ny))
    pts[:, 2] -= 20.0                     # sensor frame: the sensor 20 m above the ground
    T = np.array([[1.0, 0, 0, 0.0], [0, 1.0, 0, 0.0], [0, 0, 1.0, 20.0]])
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    compare_voxels(gm, om)
    out, ref = compare_products(gm, om)
    assert (ref["flags"] & 8).any() and np.isfinite(ref["slope"]).sum() > nx * ny // 5


# Hand-built height grids for the value of one cone (Sec. III-D, Fig. 4
# caption): a ring with several defined heights (the cone's value is the
# ring's lowest), a cone that stops at its first ring with ground, a corner
# cell shared by two cones, and a ring reaching past the grid edge. The
# expected Delta H at the test pixel is worked out by hand (the same grids
# pin the oracle on CPU in test_oracle_products.py); here the device flags
# must equal the oracle's on every pixel and show that Delta H.
def _pins(dh):
    """Delta H is exactly dh: flagged just below it, not at it (strict)."""
    return [(float(np.nextafter(np.float32(dh), np.float32(-np.inf))), True), (float(dh), False)]


CONE_CASES = [
    # (cells (x, y, height), test pixel, [(threshold, negative expected)])
    ([(9, 4, 0.5), (9, 5, 0.125), (9, 6, 0.375), (9, 7, 0.75), (9, 8, 0.625), (4, 6, 2.0)], (6, 6), _pins(1.875)),
    ([(9, 8, 0.5), (9, 7, 0.125), (9, 6, 0.375), (9, 5, 0.75), (9, 4, 0.625), (4, 6, 2.0)], (6, 6), _pins(1.875)),
    ([(9, 4, 0.5), (9, 5, 0.125), (9, 6, 0.375), (9, 7, 0.75), (9, 8, 0.625), (4, 6, -1.0)], (6, 6), _pins(1.125)),
    ([(7, 6, 1.0), (8, 6, 0.0), (5, 6, 0.75)], (6, 6), _pins(0.25)),
    # corner (8, 8) in both the +x and the +y cone: two values of 0.0
    ([(8, 8, 0.0), (9, 6, 1.0), (6, 9, 0.5)], (6, 6), [(-0.125, True), (0.0, False), (0.3, False)]),
    ([(9, 0, 0.75), (4, 1, 0.0)], (6, 1), _pins(0.75)),
    # (12, 1) lies beyond the search distance: one value only
    ([(12, 1, 0.75), (4, 1, 0.0)], (6, 1), [(-0.125, False), (0.3, False)]),
]


def _voxels_for_heights(cells, nx, ny, nz):
    """One occupied voxel (iz = 0) per defined pixel, its lowest return the
    pixel's height; every other voxel empty."""
    hits = np.zeros((nx, ny, nz), np.uint32)
    passes = np.zeros((nx, ny, nz), np.uint32)
    minz = np.full((nx, ny, nz), np.inf, np.float32)
    for x, y, h in cells:
        hits[x, y, 0] = 1
        minz[x, y, 0] = h
    return hits, passes, minz


@pytest.mark.parametrize("case", range(len(CONE_CASES)))
def test_cone_values_on_hand_built_grids(gv, case):
    cells, px, checks = CONE_CASES[case]
    nx = ny = 13
    nz = 4
    hits, passes, minz = _voxels_for_heights(cells, nx, ny, nz)
    dev = [torch.from_numpy(a.reshape(-1).view(np.int32) if a.dtype == np.uint32 else a.reshape(-1)).cuda()
           for a in (hits, passes, minz)]
    for th, expect in checks:
        p = oracle.OracleParams(nx=nx, ny=ny, nz=nz, res=0.2, neg_max_px=5, neg_thresh=th)
        ref = oracle.extract(p, hits, passes, minz)
        assert bool(ref["flags"][px] & 8) == expect, (case, th)
        h = torch.empty((nx, ny), device="cuda")
        flags = torch.full((nx, ny), 255, dtype=torch.uint8, device="cuda")
        gv.gvom_extract_maps_noalloc(gpu_config(gv, p), dev[0], dev[1], dev[2], height=h, flags=flags)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(h.cpu().numpy(), ref["height"])
        np.testing.assert_array_equal(flags.cpu().numpy(), ref["flags"])


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("case", range(6))
def test_exact_ties_on_voxel_corners_edges_and_faces(gv, case, fused):
    # res 0.25 m and coordinates on a 1/1024 m lattice make every quantised
    # endpoint exact; the sensor on a voxel corner and endpoints on the
    # quarter-voxel lattice make many crossings coincide (rays through voxel
    # corners and along faces, diagonals through edges). Windows put the
    # sensor inside, on the window's boundary, and outside, so rays enter
    # and leave the window on such ties too. Passes and hits bit-exact.
    rng = np.random.default_rng(700 + case)
    dims = [(24, 20, 12), (16, 16, 16), (32, 8, 8), (12, 30, 10), (20, 20, 6), (9, 11, 13)][case]
    params = oracle.OracleParams(nx=dims[0], ny=dims[1], nz=dims[2], res=0.25)
    n = 6000
    q = rng.integers(-40, 41, size=(n, 3)) * 64           # quarter voxels, in 1/256 voxel units
    q[: n // 4] = rng.integers(-10, 11, size=(n // 4, 3)) * 256   # voxel corners
    q[n // 4: n // 2, rng.integers(0, 3)] = 0             # rays in a coordinate plane
    k = rng.integers(1, 9, size=(n // 8, 1)) * 256
    q[n // 2: n // 2 + n // 8] = k * np.array([[1, 1, 1]]) * rng.choice([-1, 1], size=(n // 8, 3))  # body diagonals
    pts = (q.astype(np.float64) / 256.0 * params.res).astype(np.float32)   # sensor frame, metres (exact)
    sensor = np.array([0.5, -0.75, 0.25])                                   # a voxel corner (multiples of res)
    T = np.array([[1.0, 0, 0, sensor[0]], [0, 1.0, 0, sensor[1]], [0, 0, 1.0, sensor[2]]])
    sv = np.floor(sensor / params.res).astype(np.int64)
    origins = [sv - np.array(dims) // 2, sv - np.array([0, 0, 0]), sv + np.array([3, -dims[1] - 2, 1]),
               sv - np.array(dims) + 1, sv + np.array([-5, 2, -dims[2]]), sv + np.array([dims[0], 0, 0])]
    o = origins[case]
    om = oracle.OracleMap(params, tuple(int(v) for v in o))
    gm = new_map(gv, params, fused)
    gm.shift(tuple(int(v) for v in o))
    om.ingest(pts, T)
    gm.ingest(to_dev(pts), T)
    compare_voxels(gm, om)
    compare_stats(gm, om)
    assert om.stats.pass_visits > 0 or case == 5
