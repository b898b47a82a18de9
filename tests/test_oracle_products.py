"""Pins the oracle's 2D products (Sec. III-D): height, positive obstacles and
density, slope and roughness, negative obstacles; plus the qualitative
outcomes the paper reports (a box is a hard obstacle, vegetation is soft, a
ditch is a negative obstacle, a tilted plane gives its slope)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- height and positive obstacles -----------------------------------------
def _columns_map(nz=12):
    params = oracle.OracleParams(nx=1, ny=8, nz=nz, res=0.2)
    hits = np.zeros((1, 8, nz), np.uint32)
    passes = np.zeros((1, 8, nz), np.uint32)
    minz = np.full((1, 8, nz), np.inf, np.float32)
    return params, hits, passes, minz


def test_columns_hand_built():
    params, hits, passes, minz = _columns_map()

    def put(col, z, h, p, mz):
        hits[0, col, z], passes[0, col, z], minz[0, col, z] = h, p, mz

    # col 0: ground at 0.10, a dense voxel 0.85 above (in band), one 2.4 above (out)
    put(0, 2, 4, 0, 0.10)
    put(0, 5, 3, 1, 0.95)
    put(0, 9, 1, 10, 2.5)
    # col 1: sparse voxel above ground -> soft (1 / 6 < 1 / 2)
    put(1, 3, 2, 0, 0.5)
    put(1, 6, 1, 5, 1.0)
    # col 2: density exactly at the threshold 1/2 -> hard
    put(2, 0, 1, 0, -1.0)
    put(2, 4, 2, 2, -0.5)
    # col 3: band edges: exactly obs_min_h and exactly obs_max_h above ground are in
    put(3, 0, 1, 0, 0.0)
    put(3, 3, 1, 3, np.float32(0.3))
    put(3, 10, 1, 5, 2.0)
    # col 4: just above the band -> nothing
    put(4, 0, 1, 0, 0.0)
    put(4, 10, 5, 0, np.nextafter(np.float32(2.0), np.float32(3.0)))
    # col 5: empty; col 6: passes only (no returns) -> undefined
    passes[0, 6, :] = 7
    # col 7: ground only, with the lowest return in a higher voxel than another's
    put(7, 1, 1, 0, 0.31)
    put(7, 2, 1, 0, 0.25)  # not physically consistent, but height is the min of minz
    out = oracle.columns(params, hits, passes, minz)
    h, d, f = out["height"][0], out["density"][0], out["flags"][0]
    np.testing.assert_array_equal(h[:5], np.float32([0.10, 0.5, -1.0, 0.0, 0.0]))
    assert np.isnan(h[5]) and np.isnan(h[6])
    assert h[7] == np.float32(0.25)
    np.testing.assert_array_equal(f, np.uint8([3, 5, 3, 5, 0, 0, 0, 0]))
    assert d[0] == np.float32(3 / 4)
    assert d[1] == np.float32(1 / 6)
    assert d[2] == np.float32(2 / 4)
    assert d[3] == np.float32(2 / 10)
    assert d[4] == 0 and d[5] == 0 and d[7] == 0


def test_hard_threshold_integer_compare():
    params, hits, passes, minz = _columns_map()
    params.hard_num, params.hard_den = 2, 3
    hits[0, 0, 0], minz[0, 0, 0] = 1, 0.0
    # densities 2/3 (hard, equal), 1999/3000 (soft, just below)
    hits[0, 1, 0], minz[0, 1, 0] = 1, 0.0
    hits[0, 0, 5], passes[0, 0, 5], minz[0, 0, 5] = 2, 1, 1.0
    hits[0, 1, 5], passes[0, 1, 5], minz[0, 1, 5] = 1999, 1001, 1.0
    f = oracle.columns(params, hits, passes, minz)["flags"][0]
    assert f[0] == 3 and f[1] == 5


# --- slope and roughness ---------------------------------------------------
def test_tilted_plane_gives_its_slope_exactly():
    # dyadic heights: an exact plane in float32, so the fit is exact
    for gx, gy, res in ((1 / 64, 0.0, 0.25), (1 / 64, 1 / 64, 0.25), (-3 / 128, 1 / 32, 0.5)):
        params = oracle.OracleParams(nx=12, ny=10, nz=4, res=res)
        ix, iy = np.meshgrid(np.arange(12), np.arange(10), indexing="ij")
        height = (gx * ix + gy * iy + 0.5).astype(np.float32)
        s, r = oracle.slope_roughness(params, height)
        expect = np.float32(np.arctan(np.hypot(gx, gy) / res))
        assert np.all(s == expect)
        assert np.all(np.abs(r) < 1e-12)


def test_flat_plane_zero_slope_and_roughness():
    params = oracle.OracleParams(nx=9, ny=9, nz=4, res=0.2)
    height = np.full((9, 9), 1.25, np.float32)
    height[4, 4] = np.nan
    s, r = oracle.slope_roughness(params, height)
    assert np.isnan(s[4, 4]) and np.isnan(r[4, 4])
    m = ~np.isnan(height)
    assert np.all(s[m] == 0) and np.all(r[m] == 0)


def test_checkerboard_roughness_closed_form():
    # +-e checkerboard on a flat plane, full 5x5 window: the plane is flat at
    # the window mean and the mean squared error is e^2 (1 - 1/625)
    e = 0.125
    params = oracle.OracleParams(nx=11, ny=11, nz=4, res=0.2)
    ix, iy = np.meshgrid(np.arange(11), np.arange(11), indexing="ij")
    height = (2.0 + e * (-1.0) ** (ix + iy)).astype(np.float32)
    s, r = oracle.slope_roughness(params, height)
    inner = (slice(2, 9), slice(2, 9))
    np.testing.assert_allclose(r[inner], e * e * (1 - 1 / 625), rtol=1e-6)
    np.testing.assert_allclose(s[inner], 0.0, atol=1e-7)


def test_slope_roughness_match_library_least_squares():
    # random heights with holes: every pixel checked against numpy's lstsq
    params = oracle.OracleParams(nx=14, ny=13, nz=4, res=0.2, slope_n=5, slope_min_px=3)
    rng = np.random.default_rng(17)
    height = rng.normal(scale=0.4, size=(14, 13)).astype(np.float32)
    height[rng.random((14, 13)) < 0.35] = np.nan
    s, r = oracle.slope_roughness(params, height)
    rr = params.slope_n // 2
    checked = 0
    for x in range(14):
        for y in range(13):
            rows, z = [], []
            if np.isnan(height[x, y]):
                assert np.isnan(s[x, y])
                continue
            for i in range(-rr, rr + 1):
                for j in range(-rr, rr + 1):
                    if 0 <= x + i < 14 and 0 <= y + j < 13 and not np.isnan(height[x + i, y + j]):
                        rows.append((i, j, 1.0))
                        z.append(float(height[x + i, y + j]) - float(height[x, y]))
            A = np.array(rows, float)
            if len(rows) < params.slope_min_px or np.linalg.matrix_rank(A) < 3:
                assert np.isnan(s[x, y])
                continue
            coef, *_ = np.linalg.lstsq(A, np.array(z), rcond=None)
            res = np.array(z) - A @ coef
            assert abs(s[x, y] - np.arctan(np.hypot(coef[0], coef[1]) / params.res)) < 1e-6
            assert abs(r[x, y] - np.mean(res ** 2)) < 1e-6 * max(1.0, np.mean(res ** 2))
            checked += 1
    assert checked > 50


# --- negative obstacles ----------------------------------------------------
def _load_fig4():
    cells, meta = [], {}
    with open(os.path.join(GOLDEN, "fig4_cone_search.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0].replace(".", "").replace("-", "").isdigit() and len(parts) == 3:
                cells.append((int(parts[0]), int(parts[1]), float(parts[2])))
            else:
                meta[parts[0]] = [float(v) for v in parts[1:]]
    return cells, meta


def _grid_from(cells, nx, ny):
    h = np.full((nx, ny), np.nan, np.float32)
    for x, y, v in cells:
        h[x, y] = v
    return h


def test_fig4_scenario():
    cells, meta = _load_fig4()
    nx, ny = (int(v) for v in meta["grid"])
    cx, cy = (int(v) for v in meta["centre"])
    params = oracle.OracleParams(nx=nx, ny=ny, nz=4, res=0.2, neg_max_px=int(meta["neg_max_px"][0]),
                                 neg_thresh=meta["neg_thresh"][0])
    f = oracle.negative(params, _grid_from(cells, nx, ny))
    assert bool(f[cx, cy] & 8) == bool(meta["expect_negative"][0])
    # three cones hold values: with only the two low cells left, Delta H = 0.1
    f2 = oracle.negative(params, _grid_from(cells[:2], nx, ny))
    assert not f2[cx, cy] & 8
    params.neg_thresh = 0.05
    assert oracle.negative(params, _grid_from(cells[:2], nx, ny))[cx, cy] & 8
    # a single value is never enough, whatever the threshold
    params.neg_thresh = -1.0
    assert not oracle.negative(params, _grid_from(cells[:1], nx, ny))[cx, cy] & 8
    # the blue cone found nothing: a cell beyond the edge cannot count, and a
    # cell on the -y side within reach does (min of 4 values, Delta H = 1.0)
    params.neg_thresh = 0.95
    assert oracle.negative(params, _grid_from(cells, nx, ny))[cx, cy] & 8
    params.neg_thresh = 1.05
    g = _grid_from(cells + [(7, 0, -0.2)], nx, ny)
    assert oracle.negative(params, g)[cx, cy] & 8


def test_cliff_is_negative_and_hole_in_flat_ground_is_not():
    params = oracle.OracleParams(nx=30, ny=20, nz=4, res=0.2, neg_max_px=10, neg_thresh=0.3)
    h = np.full((30, 20), np.nan, np.float32)
    h[:10] = 0.0
    h[14:] = -1.0
    f = oracle.negative(params, h)
    assert np.all(f[10:14] & 8)
    assert not np.any(f[:10] & 8) and not np.any(f[14:] & 8)
    flat = np.zeros((30, 20), np.float32)
    flat[12:16, 8:12] = np.nan
    assert not np.any(oracle.negative(params, flat) & 8)


def test_negative_threshold_is_strict_and_distance_bounded():
    params = oracle.OracleParams(nx=20, ny=9, nz=4, res=0.2, neg_max_px=3, neg_thresh=0.5)
    h = np.full((20, 9), np.nan, np.float32)
    h[:8] = 0.0
    h[12:] = 0.5
    f = oracle.negative(params, h)
    assert not np.any(f & 8)  # Delta H equals the threshold
    h[12:] = np.nextafter(np.float32(0.5), np.float32(1.0))
    f = oracle.negative(params, h)
    # x = 9, 10 reach both sides within 3 pixels; x = 8 and 11 reach only
    # their own side (all cones find the same height there)
    assert np.all(f[9:11] & 8) and not np.any(f[8] & 8) and not np.any(f[11] & 8)
    # a wider gap: the middle pixels reach neither side within 3 pixels
    h2 = np.full((20, 9), np.nan, np.float32)
    h2[:4] = 0.0
    h2[16:] = 2.0
    f2 = oracle.negative(params, h2)
    assert not np.any(f2 & 8)


# --- the value of one cone (Sec. III-D, Fig. 4 caption) --------------------
# Reading: a cone's assumed height is the lowest height on the first ring
# (Chebyshev distance d) where it holds a defined in-grid pixel; corner cells
# (|j| = d) belong to both cones that meet there; in-grid cells of a ring that
# also reaches past the grid edge still count. The grids below are built by
# hand so that each alternative reading flags the test pixel differently;
# every expected value is worked out in the comments. Heights are multiples
# of 1/8, so every Delta H is exact in float32 and float64.

def _thresh_pins(params, grid, px, dh):
    """Delta H at pixel px is exactly dh: flagged just below, not at dh
    (strict threshold)."""
    params.neg_thresh = float(np.nextafter(np.float32(dh), np.float32(-np.inf)))
    assert oracle.negative(params, grid)[px] & 8, "flag expected just below Delta H"
    params.neg_thresh = float(dh)
    assert not oracle.negative(params, grid)[px] & 8, "no flag expected at Delta H"


def test_cone_value_is_ring_minimum_not_first_last_axis_max_or_mean():
    # P = (6, 6) undefined in a 13 x 13 grid, search distance 5.
    # +x cone, ring 3 = cells (9, 3..9); five non-corner cells defined:
    #   (9,4) 0.5  (9,5) 0.125  (9,6) 0.375 (on the axis)  (9,7) 0.75  (9,8) 0.625
    # -x cone, ring 2: the single cell (4, 6) = 2.0 (its value under any reading).
    # No other cone reaches a defined cell. Delta H = 2.0 - v(+x):
    #   ring minimum 0.125 -> 1.875 (the reading)
    #   first cell in ring order 0.5 -> 1.5, last 0.625 -> 1.375,
    #   axis cell 0.375 -> 1.625, ring maximum 0.75 -> 1.25, mean 0.475 -> 1.525.
    params = oracle.OracleParams(nx=13, ny=13, nz=4, res=0.2, neg_max_px=5)
    g = _grid_from([(9, 4, 0.5), (9, 5, 0.125), (9, 6, 0.375), (9, 7, 0.75), (9, 8, 0.625), (4, 6, 2.0)], 13, 13)
    _thresh_pins(params, g, (6, 6), 1.875)
    # the same ring in reverse order: first and last swap, the minimum stays
    g2 = _grid_from([(9, 8, 0.5), (9, 7, 0.125), (9, 6, 0.375), (9, 5, 0.75), (9, 4, 0.625), (4, 6, 2.0)], 13, 13)
    _thresh_pins(params, g2, (6, 6), 1.875)
    # an upper reference: Delta H = v(+x) - (-1.0) = 1.125 with the ring
    # minimum (the ring maximum would give 1.75)
    g3 = _grid_from([(9, 4, 0.5), (9, 5, 0.125), (9, 6, 0.375), (9, 7, 0.75), (9, 8, 0.625), (4, 6, -1.0)], 13, 13)
    _thresh_pins(params, g3, (6, 6), 1.125)


def test_cone_stops_at_first_ring_with_ground_not_at_a_nearer_cell_further_out():
    # P = (6, 6); +x ring 1 holds (7, 6) = 1.0 only; ring 2 holds a lower cell
    # (8, 6) = 0.0 that the cone never reaches. -x ring 1: (5, 6) = 0.75.
    # Values {1.0, 0.75}: Delta H = 0.25. A cone that took the lowest height
    # within the search distance would give {0.0, 0.75}: Delta H = 0.75.
    params = oracle.OracleParams(nx=13, ny=13, nz=4, res=0.2, neg_max_px=5)
    g = _grid_from([(7, 6, 1.0), (8, 6, 0.0), (5, 6, 0.75)], 13, 13)
    _thresh_pins(params, g, (6, 6), 0.25)


def test_corner_cell_belongs_to_both_cones():
    # P = (6, 6). The corner (8, 8) = 0.0 lies on ring 2 of both the +x cone
    # (cells (8, 4..8)) and the +y cone (cells (4..8, 8)). Further out:
    # (9, 6) = 1.0 on +x ring 3 and (6, 9) = 0.5 on +y ring 3. -x and -y
    # find nothing. Threshold 0.3:
    #   corner in both cones: +x = 0.0, +y = 0.0 -> Delta H 0 -> not negative
    #   corner only in +x:    +x = 0.0, +y = 0.5 -> 0.5 -> negative
    #   corner only in +y:    +y = 0.0, +x = 1.0 -> 1.0 -> negative
    #   corner in neither:    +x = 1.0, +y = 0.5 -> 0.5 -> negative
    params = oracle.OracleParams(nx=13, ny=13, nz=4, res=0.2, neg_max_px=5, neg_thresh=0.3)
    g = _grid_from([(8, 8, 0.0), (9, 6, 1.0), (6, 9, 0.5)], 13, 13)
    assert not oracle.negative(params, g)[6, 6] & 8
    # two values are there (0.0 twice): any threshold below 0 flags the pixel,
    # which one value alone never does
    params.neg_thresh = -0.125
    assert oracle.negative(params, g)[6, 6] & 8
    assert not oracle.negative(params, _grid_from([(9, 6, 1.0)], 13, 13))[6, 6] & 8
    # the other three corners of ring 2, each with the +x/-x/+y/-y cones they join
    for (cx, cy) in ((4, 8), (4, 4), (8, 4)):
        params.neg_thresh = -0.125
        assert oracle.negative(params, _grid_from([(cx, cy, 0.0)], 13, 13))[6, 6] & 8


def test_cone_ring_partly_outside_the_grid_keeps_searching():
    # P = (6, 1) near the y = 0 edge of a 13 x 13 grid.
    # +x cone: ring 2 = (8, -1..3) reaches past the edge at (8, -1) and has no
    # defined in-grid cell; ring 3 = (9, -2..4) holds (9, 0) = 0.75.
    # -x cone, ring 2: (4, 1) = 0.0. -y cone: ring 1 = (5..7, 0) empty, ring 2
    # would be y = -1, off the grid: the cone stops without a value. +y finds
    # nothing. Values {0.75, 0.0}: Delta H = 0.75. A cone that gave up at
    # the first ring reaching past the edge would leave one value: no flag.
    params = oracle.OracleParams(nx=13, ny=13, nz=4, res=0.2, neg_max_px=5)
    g = _grid_from([(9, 0, 0.75), (4, 1, 0.0)], 13, 13)
    _thresh_pins(params, g, (6, 1), 0.75)
    # a defined cell beyond the search distance does not count: (12, 1) is
    # on +x ring 6 > 5
    g2 = _grid_from([(12, 1, 0.75), (4, 1, 0.0)], 13, 13)
    params.neg_thresh = -0.125
    assert not oracle.negative(params, g2)[6, 1] & 8


# --- qualitative scene outcomes (the single-scan test scene) ---------------
@pytest.fixture(scope="module")
def single_scan_maps():
    import synth
    s = synth.single_scan()
    params = oracle.OracleParams()
    m = oracle.OracleMap(params)
    m.shift_for_pose(s.vehicle_xyz)
    m.ingest(s.points, s.T_ws)
    return m, m.extract()


def _px(m, x, y):
    return int(np.floor(x / m.params.res)) - m.origin[0], int(np.floor(y / m.params.res)) - m.origin[1]


def test_scene_box_is_hard_obstacle(single_scan_maps):
    m, out = single_scan_maps
    for bx, by in ((5.0, 3.0), (-4.0, -5.0)):
        ix, iy = _px(m, bx, by)
        win = out["flags"][ix - 4:ix + 5, iy - 4:iy + 5]
        assert np.count_nonzero(win & 2) >= 4
        assert np.count_nonzero(win & 4) <= np.count_nonzero(win & 2)


def test_scene_vegetation_is_soft(single_scan_maps):
    m, out = single_scan_maps
    x0, y0 = _px(m, -6.0, 2.0)
    x1, y1 = _px(m, -3.0, 5.0)
    win = out["flags"][x0 + 1:x1 - 1, y0 + 1:y1 - 1]
    assert np.count_nonzero(win & 4) > 0.5 * win.size
    assert np.count_nonzero(win & 2) < 0.1 * win.size


def test_scene_ditch_is_negative(single_scan_maps):
    # the ditch (x in [7, 9]) hides its floor and the ground just past its far
    # lip; the hidden pixels there see assumed heights that differ by more
    # than the threshold (Fig. 3, hole type)
    m, out = single_scan_maps
    x0, y0 = _px(m, 7.0, -3.0)
    x1, y1 = _px(m, 10.6, 3.0)
    win = out["flags"][x0:x1, y0:y1]
    n_ditch = np.count_nonzero(win & 8)
    assert n_ditch > 0.25 * win.size
    # the mirrored band of open ground behind the vehicle has far fewer
    x0, y0 = _px(m, -10.6, -3.0)
    x1, y1 = _px(m, -7.0, 3.0)
    assert 5 * np.count_nonzero(out["flags"][x0:x1, y0:y1] & 8) < n_ditch
    # open ground in front of the vehicle is neither obstacle nor negative
    gx, gy = _px(m, 2.5, -2.0)
    assert not np.any(out["flags"][gx - 2:gx + 3, gy - 2:gy + 3])


def test_scene_ground_slope_is_five_degrees(single_scan_maps):
    m, out = single_scan_maps
    x0, y0 = _px(m, 1.0, -3.0)
    x1, y1 = _px(m, 4.0, 0.0)
    s = out["slope"][x0:x1, y0:y1]
    assert abs(np.degrees(np.nanmedian(s)) - 5.0) < 1.0
