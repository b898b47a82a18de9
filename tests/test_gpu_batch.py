"""Batched form: many maps updated (and extracted) in one step through
gvom_batch_step must equal the same maps updated one by one through
gvom_update + gvom_extract_maps, bit for bit, with and without CUDA graph
replay, over several steps with uneven scan sizes, shifts and a jump past a
window; and it must match the CPU oracle."""
import ctypes
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


SPECS = [  # (nx, ny, nz, res): mixed sizes, z extents with and without 4 | nz
    (40, 36, 20, 0.2), (64, 64, 32, 0.25), (30, 50, 18, 0.2), (48, 40, 64, 0.1), (33, 31, 17, 0.3), (64, 48, 24, 0.2),
]


def make_maps(gv, graph_unused=None):
    return [gv.VoxelMap(nx=a, ny=b, nz=c, res=r, neg_max_px=int(math.ceil(1.0 / r))) for a, b, c, r in SPECS]


def random_scan(rng, n, centre):
    pts = np.concatenate([rng.normal(scale=[4, 4, 0.7], size=(n, 3)),
                          rng.uniform(-6, 6, size=(n // 5, 3))]).astype(np.float32)[:n]
    if n > 10:
        pts[::9] = 0.0
    th = rng.uniform(0, 2 * np.pi)
    T = np.array([[math.cos(th), -math.sin(th), 0.0, centre[0]], [math.sin(th), math.cos(th), 0.0, centre[1]],
                  [0.0, 0.0, 1.0, centre[2] + 1.2]])
    return pts, T


def snapshot(gm):
    h, p, z = (t.cpu().numpy() for t in gm.extract_voxels())
    return h.view(np.uint32), p.view(np.uint32), z


def maps_equal(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_one_by_one(gv, graph):
    rng = np.random.default_rng(7 if graph else 8)
    batched = make_maps(gv)
    plain = make_maps(gv)
    batch = gv.MapBatch(max_maps=len(SPECS), max_points=60000, graph=graph)
    centres = [np.zeros(3) for _ in SPECS]
    sizes = [[3000, 0, 1, 20000, 517, 9000], [12000, 4000, 2500, 1, 0, 7777], [256, 255, 257, 5000, 3000, 1000],
             [100, 200, 300, 400, 500, 600]]
    for step, ns in enumerate(sizes):
        scans, Ts, vs = [], [], []
        for m, n in enumerate(ns):
            centres[m] = centres[m] + rng.uniform(-0.7, 0.7, 3) * np.array([1, 1, 0.3])
            if step == 2 and m == 1:
                centres[m] = centres[m] + np.array([40.0, 0, 0])  # past the window: cleared whole
            pts, T = random_scan(rng, n, centres[m])
            scans.append(torch.from_numpy(pts).cuda())
            Ts.append(T)
            vs.append(centres[m].copy())
        outs_b = [m.alloc_maps() for m in batched]
        if step == 3:
            for o in outs_b:
                o["height"] = None  # the map's own height scratch serves the pixel pass
        batch.step(batched, vs, scans, Ts, outs=outs_b)
        for m, gm in enumerate(plain):
            gm.update(vs[m], scans[m], Ts[m])
        outs_p = [gm.extract_maps() for gm in plain]
        torch.cuda.synchronize()
        for m in range(len(SPECS)):
            assert batched[m].origin == plain[m].origin
            maps_equal(snapshot(batched[m]), snapshot(plain[m]))
            for k in ("density", "flags", "slope", "roughness") + (("height",) if step != 3 else ()):
                np.testing.assert_array_equal(outs_b[m][k].cpu().numpy(), outs_p[m][k].cpu().numpy(), err_msg=k)
            sb, sp = batched[m].stats(), plain[m].stats()
            assert sb == sp
    batch.close()


def test_batch_without_extraction_then_single_extract(gv):
    rng = np.random.default_rng(3)
    batched = make_maps(gv)
    plain = make_maps(gv)
    batch = gv.MapBatch(max_maps=8, max_points=50000)
    for step in range(3):
        scans, Ts, vs = [], [], []
        for m in range(len(SPECS)):
            pts, T = random_scan(rng, int(rng.integers(0, 8000)), np.array([0.3 * step, 0.1, 0.0]))
            scans.append(torch.from_numpy(pts).cuda())
            Ts.append(T)
            vs.append(np.array([0.3 * step, 0.1, 0.0]))
        batch.step(batched, vs, scans, Ts, outs=None)
        for m, gm in enumerate(plain):
            gm.update(vs[m], scans[m], Ts[m])
    torch.cuda.synchronize()
    for m in range(len(SPECS)):
        maps_equal(snapshot(batched[m]), snapshot(plain[m]))
        a = {k: v.cpu().numpy() for k, v in batched[m].extract_maps().items()}
        b = {k: v.cpu().numpy() for k, v in plain[m].extract_maps().items()}
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])
    batch.close()


def test_batch_matches_oracle_on_sequence_scans(gv):
    # three maps of the 256 x 256 x 64 kind, scans from the sequence workload
    cfg, scans = synth.sequence_scans("sequence", n_scans=3, stride=4)
    ms = cfg.map
    params = oracle.OracleParams(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    maps = [gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=params.neg_max_px) for _ in range(3)]
    oms = [oracle.OracleMap(params) for _ in range(3)]
    batch = gv.MapBatch(max_maps=3, max_points=3 * 131072)
    # map m sees scan (m + k) % 3 at step k
    for k in range(2):
        pick = [scans[(m + k) % 3] for m in range(3)]
        outs = [m.alloc_maps() for m in maps]
        batch.step(maps, [s.vehicle_xyz for s in pick], [torch.from_numpy(s.points).cuda() for s in pick],
                   [s.T_ws for s in pick], outs=outs)
        for om, s in zip(oms, pick):
            om.shift_for_pose(s.vehicle_xyz)
            om.ingest(s.points, s.T_ws)
    torch.cuda.synchronize()
    for gm, om, o in zip(maps, oms, outs):
        h, p, z = snapshot(gm)
        np.testing.assert_array_equal(h, om.hits)
        np.testing.assert_array_equal(p, om.passes)
        np.testing.assert_array_equal(z, om.minz)
        ref = om.extract()
        np.testing.assert_array_equal(o["height"].cpu().numpy(), ref["height"])
        np.testing.assert_array_equal(o["flags"].cpu().numpy(), ref["flags"])
        got_s = o["slope"].cpu().numpy()
        assert np.array_equal(np.isnan(got_s), np.isnan(ref["slope"]))
        ok = ~np.isnan(ref["slope"])
        assert np.max(np.abs(got_s[ok] - ref["slope"][ok])) <= 1e-3
    batch.close()


def test_batch_rejects_bad_steps_without_touching_maps(gv):
    maps = make_maps(gv)[:2]
    batch = gv.MapBatch(max_maps=2, max_points=100)
    pts = torch.zeros((60, 3), device="cuda")
    T = np.eye(3, 4)
    o0 = [m.origin for m in maps]
    with pytest.raises(gv.GvomError):  # the same map twice
        batch.step([maps[0], maps[0]], [np.zeros(3)] * 2, [pts, pts], [T, T])
    with pytest.raises(gv.GvomError):  # more points than the context holds
        batch.step(maps, [np.ones(3) * 5] * 2, [pts, pts], [T, T])
    bad = T.copy()
    bad[0, 0] = 2.0
    with pytest.raises(gv.GvomError):  # not a rotation
        batch.step(maps, [np.ones(3) * 5] * 2, [pts[:10], pts[:10]], [T, bad])
    assert [m.origin for m in maps] == o0
    batch.close()
