"""Served form: scans of many robots arriving over time, batched
continuously over two stream slots with overlapping work. Every robot's map
and every scan's 2D products must be the same as when that robot's scans are
applied alone, in order, through the plain path."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import MapSpec  # noqa: E402


@pytest.fixture(scope="module")
def gv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_13176_gb300 import build
    build.build()
    import paper_2109_13176_gb300 as m
    return m


SPECS = [MapSpec(48, 40, 24, 0.2), MapSpec(64, 64, 32, 0.25), MapSpec(40, 44, 20, 0.2), MapSpec(64, 48, 64, 0.1),
         MapSpec(32, 32, 16, 0.3), MapSpec(56, 56, 32, 0.2)]


def make_pool(rng, k):
    pool = []
    centre = np.zeros(3)
    for j in range(k):
        n = int(rng.integers(0, 6000)) if j != 1 else 0
        centre = centre + rng.uniform(-0.5, 0.5, 3) * np.array([1, 1, 0.2])
        pts = rng.normal(scale=[4, 4, 0.6], size=(n, 3)).astype(np.float32)
        th = rng.uniform(0, 2 * np.pi)
        T = np.array([[math.cos(th), -math.sin(th), 0, centre[0]], [math.sin(th), math.cos(th), 0, centre[1]],
                      [0, 0, 1.0, centre[2] + 1.0]])
        pool.append(dict(points=torch.from_numpy(pts).pin_memory(), T_ws=T, vehicle_xyz=centre.copy()))
    return pool


@pytest.mark.parametrize("realtime", [True, False])
def test_served_results_equal_solo(gv, realtime):
    from paper_2109_13176_gb300.serve import Server
    rng = np.random.default_rng(11)
    specs = {r: SPECS[r] for r in range(len(SPECS))}
    pools = {r: make_pool(rng, 5) for r in specs}
    # arrivals: every robot's 5 scans, Poisson-jittered over 0.6 s, interleaved
    arrivals = []
    for r in specs:
        t = float(rng.uniform(0, 0.05))
        for k in range(5):
            arrivals.append((t, r, k))
            t += float(rng.exponential(0.1))
    arrivals.sort()
    srv = Server(specs, slots=2, max_batch_maps=8, max_batch_points=20000, reserve_bytes=0)
    last = {}

    def on_done(req):
        last[req.robot] = {k: v.clone() for k, v in srv.host_outs[req.robot].items()}

    stats = srv.run(arrivals, pools, realtime=realtime, on_done=on_done)
    s = stats.summary()
    assert s["requests"] == len(arrivals) and s["batches"] >= 1
    assert s["p99_ms"] is not None and s["p99_ms"] >= s["p50_ms"] > 0
    # solo: each robot alone, its scans in arrival order, plain path
    for r, spec in specs.items():
        solo = gv.VoxelMap(nx=spec.nx, ny=spec.ny, nz=spec.nz, res=spec.res, neg_max_px=int(math.ceil(2.0 / spec.res)))
        for t, rr, k in arrivals:
            if rr != r:
                continue
            sc = pools[r][k]
            solo.update(sc["vehicle_xyz"], sc["points"].cuda(), sc["T_ws"])
        ref = {k: v.cpu() for k, v in solo.extract_maps().items()}
        a = [t.cpu().numpy() for t in srv.maps[r].extract_voxels()]
        b = [t.cpu().numpy() for t in solo.extract_voxels()]
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
        for k in ref:
            np.testing.assert_array_equal(last[r][k].numpy(), ref[k].numpy(), err_msg=k)
        solo.close()
    srv.close()


def test_admission_by_memory_waits_and_retries(gv):
    # a budget that holds one map at a time: robot 1's scans wait for memory
    # until robot 0 has been idle for 50 ms and gives its map back; then
    # robot 1 is admitted and its scans run in order. Each robot's results
    # equal its scans applied alone.
    from paper_2109_13176_gb300.serve import Server, map_bytes
    rng = np.random.default_rng(3)
    specs = {0: SPECS[0], 1: SPECS[1]}
    pools = {r: make_pool(rng, 4) for r in specs}
    arrivals = [(0.00, 0, 0), (0.01, 1, 0), (0.02, 0, 1), (0.03, 1, 1), (0.04, 0, 2), (0.05, 1, 2),
                (0.06, 0, 3), (0.07, 1, 3)]
    budget = max(map_bytes(sp) for sp in specs.values()) + 1000
    srv = Server(specs, slots=1, max_batch_maps=2, max_batch_points=20000, budget_bytes=budget, idle_release_s=0.05)
    last = {}

    def on_done(req):
        last[req.robot] = {k: v.clone() for k, v in srv.host_outs[req.robot].items()}

    st = srv.run(arrivals, pools, realtime=True, on_done=on_done).summary()
    assert st["requests"] == len(arrivals) and st["unserved_scans"] == 0
    assert st["refused_robots"] == [1] and st["waited_scans"] == 4 and st["released_maps"] >= 1
    for r, spec in specs.items():
        solo = gv.VoxelMap(nx=spec.nx, ny=spec.ny, nz=spec.nz, res=spec.res, neg_max_px=int(math.ceil(2.0 / spec.res)))
        for k in range(4):
            sc = pools[r][k]
            solo.update(sc["vehicle_xyz"], sc["points"].cuda(), sc["T_ws"])
        ref = {k: v.cpu() for k, v in solo.extract_maps().items()}
        for k in ref:
            np.testing.assert_array_equal(last[r][k].numpy(), ref[k].numpy(), err_msg=k)
        solo.close()
    assert 1 in srv.maps
    srv.close()


def test_oversized_scan_is_rejected_and_the_rest_served(gv):
    from paper_2109_13176_gb300.serve import Server
    rng = np.random.default_rng(4)
    specs = {0: SPECS[0]}
    pools = {0: make_pool(rng, 3)}
    big = torch.zeros((30000, 3), dtype=torch.float32).pin_memory()
    pools[0].append(dict(points=big, T_ws=pools[0][0]["T_ws"], vehicle_xyz=pools[0][0]["vehicle_xyz"]))
    srv = Server(specs, slots=1, max_batch_maps=1, max_batch_points=20000, reserve_bytes=0)
    st = srv.run([(0.0, 0, 0), (0.0, 0, 3), (0.0, 0, 1), (0.0, 0, 2)], pools, realtime=False).summary()
    assert st["rejected_scans"] == 1 and st["requests"] == 3
    srv.close()
