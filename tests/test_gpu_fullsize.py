"""Parity at the full sizes of the batched and served workloads, in the launch
configuration the benchmark times (one graph-replayed batch step; the
serving loop with continuous batching). Every map is compared bit-exactly
with the plain path on the same inputs, and sampled maps with the CPU oracle
(counts and lowest returns bit-exact, products within the stated
tolerances)."""
import math
import os

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


def workers():
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def kw_of(ms):
    return dict(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))


def params_of(ms):
    return oracle.OracleParams(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))


def same_voxels(a, b):
    for x, y in zip(a.extract_voxels(), b.extract_voxels()):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def against_oracle(gm, om, products):
    hits, passes, minz = gm.extract_voxels()
    np.testing.assert_array_equal(hits.cpu().numpy().view(np.uint32), om.hits)
    np.testing.assert_array_equal(passes.cpu().numpy().view(np.uint32), om.passes)
    np.testing.assert_array_equal(minz.cpu().numpy(), om.minz)
    out = {k: v.cpu().numpy() for k, v in products.items()}
    ref = om.extract()
    np.testing.assert_array_equal(out["height"], ref["height"])
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    np.testing.assert_allclose(out["density"], ref["density"], rtol=1e-6, atol=0)
    for k, tol in (("slope", SLOPE_TOL), ("roughness", ROUGH_TOL)):
        np.testing.assert_array_equal(np.isnan(out[k]), np.isnan(ref[k]), err_msg=k)
        m = ~np.isnan(ref[k])
        if m.any():
            assert np.max(np.abs(out[k][m] - ref[k][m])) <= tol, k


def test_batched_workload_full_size(gv):
    # 64 maps of 256 x 256 x 64, scans of 8,192-262,144 points: the two
    # generated steps the benchmark cycles, each one graph-replayed batch step
    cfg4, steps = synth.batched_scans(n_maps=64, n_steps=2, workers=workers())
    ms = cfg4.map
    nm = len(steps[0])
    maps_b = [gv.VoxelMap(**kw_of(ms)) for _ in range(nm)]
    maps_p = [gv.VoxelMap(**kw_of(ms)) for _ in range(nm)]
    devs = [[torch.from_numpy(s.points).cuda() for s in st] for st in steps]
    batch = gv.MapBatch(nm, max(sum(int(p.shape[0]) for p in d) for d in devs), graph=True)
    outs = [m.alloc_maps() for m in maps_b]
    sizes = [len(s.points) for s in steps[0]]
    sampled = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))})
    oms = {i: oracle.OracleMap(params_of(ms)) for i in sampled}
    for scans, dev in zip(steps, devs):
        batch.step(maps_b, [s.vehicle_xyz for s in scans], dev, [s.T_ws for s in scans], outs=outs)
        for m, p, s in zip(maps_p, dev, scans):
            m.update(s.vehicle_xyz, p, s.T_ws)
        torch.cuda.synchronize()
        for i, (a, b) in enumerate(zip(maps_b, maps_p)):
            same_voxels(a, b)
            ref = b.extract_maps()
            for k in ref:
                np.testing.assert_array_equal(outs[i][k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=f"map {i} {k}")
        for i, om in oms.items():
            om.shift_for_pose(scans[i].vehicle_xyz)
            om.ingest(scans[i].points, scans[i].T_ws)
            against_oracle(maps_b[i], om, outs[i])
    batch.close()
    for m in maps_b + maps_p:
        m.close()


def served_pools(robots, arrivals):
    """scans[robot][k]: the arrival's cast (pinned, shared between the
    arrivals of one span) with the arrival's own pose."""
    casts = {i: [torch.from_numpy(c.points).pin_memory() for c in r["casts"]] for i, r in enumerate(robots)}
    pools = {i: {} for i in range(len(robots))}
    for t, rid, k, c, T, veh in arrivals:
        pools[rid][k] = dict(points=casts[rid][c], T_ws=T, vehicle_xyz=veh, cast=c)
    return pools


def test_served_workload_full_size(gv):
    # 32 robots with the workload's mixed sensors and maps on their own
    # trajectories, every request admitted at once (saturation), continuous
    # batching over two slots, maps created by per-scan admission
    from paper_2109_13176_gb300.serve import Server
    robots, arrivals = synth.served_stream(n_robots=32, duration_s=0.6, casts=2, workers=workers())
    specs = {i: r["map"] for i, r in enumerate(robots)}
    pools = served_pools(robots, arrivals)
    arr = [(t, rid, k) for t, rid, k, *_ in arrivals]
    max_pts = sum(max(int(s["points"].shape[0]) for s in pools[i].values()) for i in pools)
    srv = Server(specs, slots=2, max_batch_maps=len(robots), max_batch_points=max_pts, reserve_bytes=1 << 30)
    last = {}

    def on_done(req):
        last[req.robot] = {k: v.clone() for k, v in srv.host_outs[req.robot].items()}

    stats = srv.run(arr, pools, realtime=False, on_done=on_done).summary()
    assert stats["requests"] == len(arr) and stats["batches"] >= 1 and stats["waited_scans"] == 0
    order = {}
    for _, rid, k in arr:
        order.setdefault(rid, []).append(k)
    # every robot: the same map and last products as its scans applied alone
    for rid, ks in order.items():
        solo = gv.VoxelMap(**kw_of(specs[rid]))
        for k in ks:
            sc = pools[rid][k]
            solo.update(sc["vehicle_xyz"], sc["points"].cuda(), sc["T_ws"])
        ref = solo.extract_maps()
        same_voxels(srv.maps[rid], solo)
        for key in ref:
            np.testing.assert_array_equal(last[rid][key].numpy(), ref[key].cpu().numpy(), err_msg=f"{rid} {key}")
        solo.close()
    # a sampled robot (the smallest map) against the oracle over its requests
    rid = min(order, key=lambda r: specs[r].nx * specs[r].ny * specs[r].nz)
    om = oracle.OracleMap(params_of(specs[rid]))
    for k in order[rid]:
        sc = pools[rid][k]
        om.shift_for_pose(sc["vehicle_xyz"])
        om.ingest(robots[rid]["casts"][sc["cast"]].points, sc["T_ws"])
    against_oracle(srv.maps[rid], om, {k: v for k, v in last[rid].items()})
    srv.close()
