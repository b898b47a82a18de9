"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/gvom.h declares, and
rejects invalid arguments before touching the device."""
import ctypes

import pytest

import paper_2109_13176_gb300 as gv
from paper_2109_13176_gb300 import build as gvbuild


@pytest.fixture(scope="module")
def lib():
    gvbuild.build()
    return gv.load_library()


def test_exports_every_declared_symbol(lib):
    names = gv.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # and the binding exposes the same names
    for name in names:
        assert callable(getattr(gv, name, None)), name


def test_status_strings(lib):
    assert gv.status_string(0) == "ok"
    assert "invalid" in gv.status_string(gv.GVOM_ERR_INVALID_ARG)
    assert gv.status_string(12345) == "unknown status"


def test_config_default(lib):
    c = gv.gvom_config_default()
    assert (c.nx, c.ny, c.nz) == (128, 128, 32)
    assert c.res == pytest.approx(0.2) and c.max_range == 100.0
    assert (c.hard_num, c.hard_den, c.slope_n, c.slope_min_px, c.neg_max_px) == (1, 2, 5, 3, 10)


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("nz", 5000), ("res", 0.0), ("res", -0.1), ("max_range", 0.0), ("hard_den", 0),
    ("hard_num", 3), ("slope_n", 4), ("slope_n", 17), ("slope_min_px", 2), ("neg_max_px", 0),
    ("scan_buffer", -1), ("scan_buffer", 65), ("obs_max_h", 0.1), ("hard_den", 70000),
    ("neg_max_px", 65), ("slope_min_px", 26), ("res", float("inf")), ("neg_thresh", float("nan")),
    ("obs_min_h", -0.1),
])
def test_create_rejects_invalid_config_before_device_work(lib, field, value):
    c = gv.gvom_config_default()
    setattr(c, field, value)
    h = ctypes.c_void_p(1234)
    rc = lib.gvom_create(ctypes.byref(c), ctypes.byref(h))
    assert rc == gv.GVOM_ERR_INVALID_ARG
    assert h.value is None


def test_create_rejects_oversized_map(lib):
    c = gv.gvom_config_default()
    c.nx, c.ny, c.nz = 4096, 4096, 128
    h = ctypes.c_void_p()
    assert lib.gvom_create(ctypes.byref(c), ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG


def test_null_arguments_rejected(lib):
    T = (ctypes.c_double * 12)()
    o = (ctypes.c_int64 * 3)()
    assert lib.gvom_create(None, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_ingest_scan(None, None, 0, 3, T, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_shift(None, o, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_extract_maps(None, None, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_get_stats(None, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_origin_for_pose(None, None, o) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_config_default(None) == gv.GVOM_ERR_INVALID_ARG
    ptrs = (ctypes.c_void_p * 1)()
    ns = (ctypes.c_int64 * 1)(0)
    assert lib.gvom_ingest_multi(None, 1, ptrs, ns, 3, T, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_export_lut(None, None, None, None, None, 0, None, None) == gv.GVOM_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.gvom_pipeline_create(None, 10, ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG and h.value is None
    t = ctypes.c_int64()
    assert lib.gvom_pipeline_submit(None, T, None, 0, 3, T, None, ctypes.byref(t)) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_pipeline_query(None, 1) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_pipeline_wait(None, 1) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_pipeline_products(None, 1, None) == gv.GVOM_ERR_INVALID_ARG
    lib.gvom_pipeline_destroy(None)  # no-op
    assert lib.gvom_update_extract(None, T, None, 0, 3, T, None, None) == gv.GVOM_ERR_INVALID_ARG
    lib.gvom_destroy(None)  # no-op


def test_config_limit_on_range_over_resolution(lib):
    c = gv.gvom_config_default()
    c.res, c.max_range = 0.01, 100.0  # 10,000 voxels of range: beyond the 8192 limit
    h = ctypes.c_void_p()
    assert lib.gvom_create(ctypes.byref(c), ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG


def test_batch_and_noalloc_reject_invalid_arguments(lib):
    h = ctypes.c_void_p(1234)
    assert lib.gvom_batch_create(0, 10, 0, ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG and h.value is None
    h = ctypes.c_void_p(1234)
    assert lib.gvom_batch_create(4097, 10, 0, ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG and h.value is None
    assert lib.gvom_batch_create(1, 0, 0, ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_batch_create(1, 10, 2, ctypes.byref(h)) == gv.GVOM_ERR_INVALID_ARG  # unknown flag
    assert lib.gvom_batch_create(1, 10, 0, None) == gv.GVOM_ERR_INVALID_ARG
    assert lib.gvom_batch_set_tuning(None, None) == gv.GVOM_ERR_INVALID_ARG
    T = (ctypes.c_double * 12)()
    v = (ctypes.c_double * 3)()
    ns = (ctypes.c_int64 * 1)(0)
    ptrs = (ctypes.c_void_p * 1)()
    assert lib.gvom_batch_step(None, ptrs, 1, v, ptrs, ns, 3, T, None, None) == gv.GVOM_ERR_INVALID_ARG
    lib.gvom_batch_destroy(None)  # no-op
    # the no-alloc extraction validates the configuration and its map-size
    # limit (512 x 512 pixels) before any launch
    out = gv.gvom_maps_out()
    fake = ctypes.c_void_p(256)
    assert lib.gvom_extract_maps_noalloc(None, fake, fake, fake, ctypes.byref(out), None) == gv.GVOM_ERR_INVALID_ARG
    c = gv.gvom_config_default()
    assert lib.gvom_extract_maps_noalloc(ctypes.byref(c), None, fake, fake, ctypes.byref(out), None) == \
        gv.GVOM_ERR_INVALID_ARG
    c.nx, c.ny = 1024, 512
    assert lib.gvom_extract_maps_noalloc(ctypes.byref(c), fake, fake, fake, ctypes.byref(out), None) == \
        gv.GVOM_ERR_INVALID_ARG


def test_noalloc_rejects_misaligned_grids_before_any_launch(lib):
    # nz % 4 == 0: the grids are read with 16-byte loads, so a grid that
    # starts 4 bytes into an allocation (a torch slice, say) is refused with
    # an error instead of faulting on the device; other nz need 4 bytes.
    # These fake device addresses are never dereferenced: the checks come
    # before any CUDA call (this test runs without a GPU).
    c = gv.gvom_config_default()      # nz = 32
    out = gv.gvom_maps_out()
    ok, off4, off2 = ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 4), ctypes.c_void_p(4096 + 2)
    for grids in ((off4, ok, ok), (ok, off4, ok), (ok, ok, off4)):
        assert lib.gvom_extract_maps_noalloc(ctypes.byref(c), *grids, ctypes.byref(out), None) == \
            gv.GVOM_ERR_INVALID_ARG
    c.nz = 30
    for grids in ((off2, ok, ok), (ok, off2, ok), (ok, ok, off2)):
        assert lib.gvom_extract_maps_noalloc(ctypes.byref(c), *grids, ctypes.byref(out), None) == \
            gv.GVOM_ERR_INVALID_ARG
    # misaligned float outputs
    c.nz = 32
    for k in ("height_dev", "density_dev", "slope_dev", "roughness_dev"):
        o = gv.gvom_maps_out()
        setattr(o, k, 4096 + 2)
        assert lib.gvom_extract_maps_noalloc(ctypes.byref(c), ok, ok, ok, ctypes.byref(o), None) == \
            gv.GVOM_ERR_INVALID_ARG


def test_no_cpu_fallback_without_a_gpu(lib, monkeypatch):
    # the product path fails loudly: no device, no map; no library, no calls
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    c = gv.gvom_config_default()
    h = ctypes.c_void_p()
    assert lib.gvom_create(ctypes.byref(c), ctypes.byref(h)) == gv.GVOM_ERR_CUDA and h.value is None
    with pytest.raises(RuntimeError):
        gv.VoxelMap(nx=16, ny=16, nz=8, res=0.2)
    monkeypatch.setattr(gv, "_lib", None)
    monkeypatch.setattr(gv, "LIB_PATH", "/nonexistent/libgvom.so")
    with pytest.raises(RuntimeError):
        gv.load_library()
