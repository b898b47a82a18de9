"""Launch shapes never change results: every extraction shape the tuner may
pick (pixel tile edge, column-pass chunk shape) and walk shape gives the
same products and voxels, bit for bit, as the defaults (which the parity
tests compare with the oracle)."""
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


def products(m):
    return {k: v.cpu().numpy() for k, v in m.extract_maps().items()}


def same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("workload", ["single_scan", "sequence"])
def test_extraction_shapes_give_identical_products(gv, workload):
    from paper_2109_13176_gb300 import tune
    if workload == "single_scan":
        scans, ms = [synth.single_scan()], synth.WORKLOADS["single_scan"]["map"]
    else:
        cfg, scans = synth.sequence_scans("sequence", n_scans=2, stride=5)
        ms = cfg.map
    m = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, neg_max_px=int(math.ceil(2.0 / ms.res)))
    for s in scans:
        m.update(s.vehicle_xyz, torch.from_numpy(s.points).cuda(), s.T_ws)
    ref = products(m)
    tried = 0
    for px_tile, col_shape in tune.extract_candidates(m) + [(5, 0), (64, 1)]:
        try:
            m.set_extract_tuning(px_tile, col_shape)
        except gv.GvomError:
            continue  # does not fit shared memory for this map
        same(products(m), ref)
        tried += 1
    assert tried >= 8
    m.close()


def test_walk_shapes_give_identical_voxels(gv):
    cfg, scans = synth.sequence_scans("sequence", n_scans=1)
    ms = cfg.map
    s = scans[0]
    pts = torch.from_numpy(s.points).cuda()
    ref = None
    for seg_len, block in ((1, 128), (7, 256), (16, 256), (64, 128), (4096, 256)):
        m = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
        m.set_tuning(seg_len, block, 0)
        m.update(s.vehicle_xyz, pts, s.T_ws)
        vox = [t.cpu().numpy() for t in m.extract_voxels()]
        st = m.stats()
        if ref is None:
            ref = (vox, st)
        else:
            for x, y in zip(vox, ref[0]):
                np.testing.assert_array_equal(x, y)
            assert st == ref[1]
        m.close()


def voxels_and_stats(m):
    return [t.cpu().numpy() for t in m.extract_voxels()], m.stats()


def same_state(a, b):
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)
    assert a[1] == b[1]


@pytest.mark.parametrize("workload", ["sequence", "high_speed"])
def test_fused_ingest_gives_identical_voxels(gv, workload):
    # the fused ingest (one kernel lists and walks) against the two-kernel
    # path, scan by scan along a shifting sequence, under several segment
    # lengths and block shapes; the status word stays clear
    cfg, scans = synth.sequence_scans(workload, n_scans=4, stride=2)
    ms = cfg.map
    pts = [torch.from_numpy(s.points).cuda() for s in scans]
    for seg_len, block in ((16, 256), (1, 128), (8, 256), (48, 128)):
        ref = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
        fu = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
        ref.set_tuning(seg_len, block, 0, fused_ingest=False)
        fu.set_tuning(seg_len, block, 0, fused_ingest=True)
        for s, p in zip(scans, pts):
            ref.update(s.vehicle_xyz, p, s.T_ws)
            fu.update(s.vehicle_xyz, p, s.T_ws)
            same_state(voxels_and_stats(fu), voxels_and_stats(ref))
        ref.close()
        fu.close()


def test_fused_and_two_kernel_ingests_alternate(gv):
    # list entries one path leaves behind never reach the other: switching
    # the tuning between scans keeps the state equal to a map that never
    # switches; also small and empty scans, and blocks per SM capped
    cfg, scans = synth.sequence_scans("sequence", n_scans=6, stride=1)
    ms = cfg.map
    ref = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    alt = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    for k, s in enumerate(scans):
        alt.set_tuning(16, 256, 1 + (k % 2), fused_ingest=k % 3 != 1)
        for n in (len(s.points), 0, 31, 33):
            p = torch.from_numpy(s.points[:n]).cuda()
            ref.update(s.vehicle_xyz, p, s.T_ws)
            alt.update(s.vehicle_xyz, p, s.T_ws)
        same_state(voxels_and_stats(alt), voxels_and_stats(ref))
    ref.close()
    alt.close()


def test_fused_flag_on_a_scan_buffer_map(gv):
    # maps with a scan buffer take the two kernels whatever the flag says
    cfg, scans = synth.sequence_scans("sequence", n_scans=3, stride=2)
    ms = cfg.map
    ref = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, scan_buffer=2)
    fu = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res, scan_buffer=2)
    fu.set_fused_ingest(True)
    for s in scans:
        p = torch.from_numpy(s.points).cuda()
        ref.update(s.vehicle_xyz, p, s.T_ws)
        fu.update(s.vehicle_xyz, p, s.T_ws)
    same_state(voxels_and_stats(fu), voxels_and_stats(ref))
    ref.close()
    fu.close()


def test_fused_flag_while_capturing_a_graph(gv):
    # a capturing stream takes the two kernels (a replayed fused launch would
    # repeat its list tag): two replays equal two plain ingests
    cfg, scans = synth.sequence_scans("sequence", n_scans=1)
    ms = cfg.map
    s = scans[0]
    p = torch.from_numpy(s.points).cuda()
    ref = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    cap = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    cap.set_fused_ingest(True)
    o = ref.origin_for_pose(s.vehicle_xyz)
    ref.shift(o)
    cap.shift(o)
    cap.reserve(len(s.points))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            cap.ingest(p, s.T_ws, stream=side)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        ref.ingest(p, s.T_ws)
    torch.cuda.synchronize()
    a, b = voxels_and_stats(cap), voxels_and_stats(ref)
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)
    ref.close()
    cap.close()


def test_fused_ingest_on_a_side_stream(gv):
    # the first ingest grows the map's scratch (its list is cleared on the
    # caller's stream, before the fused kernel reads the tags): a map fed on a
    # side stream equals a two-kernel map fed on the default stream
    cfg, scans = synth.sequence_scans("sequence", n_scans=3, stride=2)
    ms = cfg.map
    ref = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    fu = gv.VoxelMap(nx=ms.nx, ny=ms.ny, nz=ms.nz, res=ms.res)
    fu.set_fused_ingest(True)
    side = torch.cuda.Stream()
    for s in scans:
        p = torch.from_numpy(s.points).cuda()
        torch.cuda.synchronize()
        ref.update(s.vehicle_xyz, p, s.T_ws)
        with torch.cuda.stream(side):
            fu.update(s.vehicle_xyz, p, s.T_ws, stream=side)
        side.synchronize()
    torch.cuda.synchronize()
    same_state(voxels_and_stats(fu), voxels_and_stats(ref))
    ref.close()
    fu.close()
