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
