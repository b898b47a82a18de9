"""The asynchronous scan pipeline (upload, map and products stages on three
streams joined by events) gives, scan by scan, the same products as the
plain path (gvom_update then gvom_extract_maps) on the same inputs, with
several scans in flight."""
import math

import numpy as np
import pytest

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


def run_both(gv, kw, scans, max_points, om=None):
    """Pipeline against the plain path, scan by scan; with an oracle map om,
    each scan's products are also compared with the oracle's."""
    plain = gv.VoxelMap(**kw)
    piped = gv.VoxelMap(**kw)
    pipe = gv.Pipeline(piped, max_points)
    tickets, outs = [], []
    for s in scans:
        o = pipe.alloc_host_outs()
        host_pts = torch.from_numpy(np.ascontiguousarray(s["points"], dtype=np.float32)).pin_memory()
        tickets.append(pipe.submit(s["vehicle_xyz"], host_pts, s["T_ws"], o))
        outs.append((o, host_pts))
    pipe.wait(tickets[-1])
    for t in tickets:
        assert pipe.query(t)
    for s, (o, _) in zip(scans, outs):
        plain.update(s["vehicle_xyz"], torch.from_numpy(np.ascontiguousarray(s["points"], np.float32)).cuda(),
                     s["T_ws"])
        ref = plain.extract_maps()
        torch.cuda.synchronize()
        for k in ref:
            np.testing.assert_array_equal(o[k].numpy(), ref[k].cpu().numpy(), err_msg=k)
        if om is not None:
            om.shift_for_pose(s["vehicle_xyz"])
            om.ingest(s["points"], s["T_ws"])
            oracle_products_match({k: v.numpy() for k, v in o.items()}, om.extract())
    for x, y in zip(plain.extract_voxels(), piped.extract_voxels()):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    pipe.close()
    plain.close()
    piped.close()


def oracle_products_match(out, ref):
    """The tolerances of the parity tests: height, flags bit-exact, density
    1e-6 relative, slope 1e-3 rad, roughness 1e-4 m^2, same defined pixels."""
    np.testing.assert_array_equal(out["height"], ref["height"])
    np.testing.assert_array_equal(out["flags"], ref["flags"])
    np.testing.assert_allclose(out["density"], ref["density"], rtol=1e-6, atol=0)
    for k, tol in (("slope", 1e-3), ("roughness", 1e-4)):
        np.testing.assert_array_equal(np.isnan(out[k]), np.isnan(ref[k]), err_msg=k)
        m = ~np.isnan(ref[k])
        if m.any():
            assert np.max(np.abs(out[k][m] - ref[k][m])) <= tol, k


def test_pipeline_full_size_sequence(gv):
    # five scans of the sequence workload in flight through the pipeline:
    # each scan's host products equal the plain path's and the oracle's
    import oracle
    cfg, scans = synth.sequence_scans("sequence", n_scans=5)
    ms = cfg.map
    kw = dict(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    seq = [dict(points=s.points, T_ws=s.T_ws, vehicle_xyz=s.vehicle_xyz) for s in scans]
    om = oracle.OracleMap(oracle.OracleParams(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res,
                                              neg_max_px=int(math.ceil(2.0 / ms.res))))
    run_both(gv, kw, seq, max(len(s.points) for s in scans), om=om)


@pytest.mark.parametrize("K", [0, 2])
def test_pipeline_many_scans_in_flight(gv, K):
    rng = np.random.default_rng(50 + K)
    kw = dict(nx=96, ny=80, nz=32, res=0.2, neg_max_px=10, scan_buffer=K)
    seq, centre = [], np.zeros(3)
    for j in range(10):
        centre = centre + rng.uniform(-0.6, 0.6, 3) * np.array([1, 1, 0.1])
        n = 0 if j == 3 else int(rng.integers(100, 9000))
        pts = rng.normal(scale=[4, 4, 0.6], size=(n, 3)).astype(np.float32)
        if j % 2:
            pts = np.concatenate([pts, np.ones((n, 1), np.float32)], axis=1)
        th = rng.uniform(0, 2 * np.pi)
        T = np.array([[math.cos(th), -math.sin(th), 0, centre[0]], [math.sin(th), math.cos(th), 0, centre[1]],
                      [0, 0, 1.0, centre[2] + 1.0]])
        seq.append(dict(points=pts, T_ws=T, vehicle_xyz=centre.copy()))
    run_both(gv, kw, seq, 9000)


def test_pipeline_tickets_and_slots(gv):
    m = gv.VoxelMap(nx=32, ny=32, nz=16, res=0.2)
    pipe = gv.Pipeline(m, 100)
    pts = torch.zeros((10, 3), dtype=torch.float32).pin_memory()
    T = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 1.0]])
    t1 = pipe.submit((0, 0, 0), pts, T)
    pipe.wait(t1)
    prods = gv.gvom_pipeline_products(pipe.handle, t1)
    assert all(v for v in prods.values())
    ts = [pipe.submit((0, 0, 0), pts, T) for _ in range(3)]
    pipe.wait(ts[-1])
    assert pipe.query(t1)                       # finished long ago
    with pytest.raises(gv.GvomError):
        gv.gvom_pipeline_products(pipe.handle, t1)   # its slot has been reused
    with pytest.raises(gv.GvomError):
        pipe.wait(ts[-1] + 1)                   # not submitted
    with pytest.raises(gv.GvomError):
        pipe.submit((0, 0, 0), torch.zeros((101, 3), dtype=torch.float32), T)  # beyond max_points
    pipe.close()
    m.close()


def test_packed_products_equal_separate(gv):
    # the products written into one packed buffer (one readback copy) equal
    # the separately allocated ones
    cfg, scans = synth.sequence_scans("sequence", n_scans=1)
    ms = cfg.map
    m = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    s = scans[0]
    m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    ref = m.extract_maps()
    buf, views = m.alloc_maps_packed()
    m.extract_maps(views)
    host = torch.empty(buf.numel(), dtype=torch.uint8, pin_memory=True)
    host.copy_(buf)
    _, hviews = m.alloc_maps_packed(device=torch.device("cpu"))
    for k, v in ref.items():
        np.testing.assert_array_equal(views[k].cpu().numpy(), v.cpu().numpy(), err_msg=k)
    # the host copy holds the same bytes at the same offsets
    off = 0
    for k in ("height", "density", "slope", "roughness", "flags"):
        n = ref[k].numel() * ref[k].element_size()
        np.testing.assert_array_equal(host[off:off + n].numpy(), views[k].contiguous().view(torch.uint8).reshape(-1).cpu().numpy())
        off += (n + 255) // 256 * 256
    m.close()


def test_update_extract_equals_separate_calls(gv):
    cfg, scans = synth.sequence_scans("sequence", n_scans=2)
    ms = cfg.map
    kw = dict(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    a, b = gv.VoxelMap(**kw), gv.VoxelMap(**kw)
    _, views = a.alloc_maps_packed()
    for s in scans:
        p = torch.from_numpy(s.points).cuda()
        a.update_extract(s.vehicle_xyz, p, s.T_ws, views)
        b.update(s.vehicle_xyz, p, s.T_ws)
    ref = b.extract_maps()
    for k in ref:
        np.testing.assert_array_equal(views[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=k)
    a.close()
    b.close()
