"""Pins the oracle's per-scan update (Sec. III-A, III-C, III-D combination)
against brute force in exact rational arithmetic and against invariants.

Inputs are chosen so that the quantised endpoints are exact without any
rounding (resolution 0.25 m, coordinates on a 1/1024 m grid, poses that are
the identity or an exact 90 degree yaw), which lets the brute force derive
every expected count from the definitions alone.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.test_oracle_traversal import meets

RES = 0.25
Q = 1024  # 1/1024 m grid: w / res * 256 = 1024 w


def small_params(**kw):
    p = dict(nx=7, ny=6, nz=5, res=RES, max_range=100.0)
    p.update(kw)
    return oracle.OracleParams(**p)


def exact_world(p, T):
    """w = R p + t for an exact R (entries 0, +-1) on Fractions."""
    R = [[Fraction(T[i][j]) for j in range(3)] for i in range(3)]
    t = [Fraction(T[i][3]) for i in range(3)]
    pf = [Fraction(float(v)) for v in p]
    return [sum(R[i][j] * pf[j] for j in range(3)) + t[i] for i in range(3)]


def brute_update(params, origin, pts, T):
    """Expected hits, passes, minz, from the definitions (Sec. III-A)."""
    nx, ny, nz = params.nx, params.ny, params.nz
    hits = np.zeros((nx, ny, nz), np.uint32)
    passes = np.zeros((nx, ny, nz), np.uint32)
    minz = np.full((nx, ny, nz), np.inf, np.float32)
    A = [int(Fraction(T[i][3]) * Q) - 256 * int(origin[i]) for i in range(3)]
    valid = 0
    for p in pts:
        if not np.all(np.isfinite(p)):
            continue
        r2 = sum(Fraction(float(v)) ** 2 for v in p)
        if not (0 < r2 <= Fraction(params.max_range) ** 2):
            continue
        valid += 1
        w = exact_world(p, T)
        B = [w[i] * Q - 256 * int(origin[i]) for i in range(3)]
        assert all(b.denominator == 1 for b in B)
        B = [int(b) for b in B]
        ce = tuple(b // 256 for b in B)
        if all(0 <= ce[i] < (nx, ny, nz)[i] for i in range(3)):
            hits[ce] += 1
            minz[ce] = min(minz[ce], np.float32(float(w[2])))
        for ix in range(nx):
            for iy in range(ny):
                for iz in range(nz):
                    c = (ix, iy, iz)
                    if c != ce and meets(A, B, c):
                        passes[c] += 1
    return hits, passes, minz, valid


def grid_points(rng, n, lo, hi):
    return (rng.integers(int(lo * Q), int(hi * Q), size=(n, 3)) / Q).astype(np.float32)


IDENTITY = np.array([[1, 0, 0, 0.0], [0, 1, 0, 0.0], [0, 0, 1, 0.0]])
YAW90 = np.array([[0, -1, 0, 0.0], [1, 0, 0, 0.0], [0, 0, 1, 0.0]])


@pytest.mark.parametrize("rot", ["identity", "yaw90"])
@pytest.mark.parametrize("sensor", [(0.8125, 0.7509765625, 0.5), (-0.5, 0.75, 0.25), (1.0, 0.5, 0.75)])
def test_update_matches_exact_brute_force(rot, sensor):
    params = small_params()
    rng = np.random.default_rng(hash((rot, sensor)) % 2**32)
    T = (IDENTITY if rot == "identity" else YAW90).copy()
    T[:, 3] = sensor
    pts = grid_points(rng, 40, -1.5, 1.5)
    # endpoints on cell faces, edges and corners (multiples of res) too
    pts[:8] = (rng.integers(-6, 6, size=(8, 3)) * RES).astype(np.float32)
    origin = np.array([0, 0, 0], np.int64)
    m = oracle.OracleMap(params, origin)
    st = m.ingest(pts, T)
    hits, passes, minz, valid = brute_update(params, origin, pts, T)
    assert st.rays_valid == valid
    np.testing.assert_array_equal(m.hits, hits)
    np.testing.assert_array_equal(m.passes, passes)
    np.testing.assert_array_equal(m.minz, minz)
    assert int(m.hits.sum()) == st.hits_in_window
    assert int(m.passes.sum()) == st.pass_visits


def test_origin_offsets_window():
    # a non-zero (and negative) origin moves the window in whole voxels
    params = small_params()
    rng = np.random.default_rng(5)
    T = IDENTITY.copy()
    T[:, 3] = (-2.0, 3.5, -0.25)
    pts = grid_points(rng, 30, -1.5, 1.5)
    origin = np.array([-11, 12, -3], np.int64)
    m = oracle.OracleMap(params, origin)
    m.ingest(pts, T)
    hits, passes, minz, _ = brute_update(params, origin, pts, T)
    np.testing.assert_array_equal(m.hits, hits)
    np.testing.assert_array_equal(m.passes, passes)
    np.testing.assert_array_equal(m.minz, minz)


def test_filter_drops_invalid_points():
    # non-finite, zero-range and over-range points are dropped; the squared
    # range of these points is exact in FP64, so the rational count is exact
    params = small_params(max_range=1.0)
    T = IDENTITY.copy()
    T[:, 3] = (0.8125, 0.8125, 0.625)
    pts = np.array([[0.125, 0.25, 0.375], [np.nan, 0, 0], [np.inf, 0, 0], [0, 0, -np.inf], [0, 0, 0],
                    [1.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.5, 0.5, 0.75], [0.0, 0.0, 1.0000001],
                    [0.0, -1.0, 0.0], [2.0, 0, 0]], np.float32)
    m = oracle.OracleMap(params)
    st = m.ingest(pts, T)
    assert st.points_in == len(pts)
    assert st.rays_valid == 4  # rows 0, 5, 6 and 9
    hits, passes, minz, valid = brute_update(params, np.zeros(3, np.int64), pts, T)
    assert valid == st.rays_valid
    np.testing.assert_array_equal(m.hits, hits)
    np.testing.assert_array_equal(m.passes, passes)


def test_stride4_points_equal_stride3():
    params = small_params()
    rng = np.random.default_rng(9)
    T = YAW90.copy()
    T[:, 3] = (0.75, 0.75, 0.5)
    pts = grid_points(rng, 50, -1.5, 1.5)
    p4 = np.concatenate([pts, rng.normal(size=(50, 1)).astype(np.float32)], axis=1)
    a = oracle.OracleMap(params)
    b = oracle.OracleMap(params)
    a.ingest(pts, T)
    b.ingest(p4, T)
    np.testing.assert_array_equal(a.hits, b.hits)
    np.testing.assert_array_equal(a.passes, b.passes)


def test_sum_of_hits_equals_in_window_points_large():
    # Sec. III-A: every in-window return adds exactly one hit
    params = oracle.OracleParams(nx=32, ny=32, nz=16, res=0.2)
    rng = np.random.default_rng(3)
    th = 0.3
    T = np.array([[np.cos(th), -np.sin(th), 0, 0.13], [np.sin(th), np.cos(th), 0, -0.21], [0, 0, 1, 1.5]])
    pts = rng.normal(scale=4.0, size=(4000, 3)).astype(np.float32)
    m = oracle.OracleMap(params, (-16, -16, -8))
    st = m.ingest(pts, T)
    assert int(m.hits.sum()) == st.hits_in_window
    assert st.rays_valid == 4000
    # per-ray pass identity: increments = sum over rays of |S in window| - [end in window]
    assert int(m.passes.sum()) == st.pass_visits


def test_combination_equals_sum_and_min():
    # Sec. III-D: combining maps adds hits and misses and takes the min height
    params = oracle.OracleParams(nx=24, ny=20, nz=12, res=0.2)
    rng = np.random.default_rng(4)
    T1 = np.array([[1, 0, 0, 0.05], [0, 1, 0, 0.1], [0, 0, 1, 1.2]])
    T2 = np.array([[0.8, -0.6, 0, -0.3], [0.6, 0.8, 0, 0.2], [0, 0, 1, 1.0]])
    A = rng.normal(scale=2.0, size=(800, 3)).astype(np.float32)
    B = rng.normal(scale=2.0, size=(900, 3)).astype(np.float32)
    o = (-12, -10, -6)
    both = oracle.OracleMap(params, o)
    both.ingest(A, T1)
    both.ingest(B, T2)
    ma = oracle.OracleMap(params, o)
    ma.ingest(A, T1)
    mb = oracle.OracleMap(params, o)
    mb.ingest(B, T2)
    np.testing.assert_array_equal(both.hits, ma.hits + mb.hits)
    np.testing.assert_array_equal(both.passes, ma.passes + mb.passes)
    np.testing.assert_array_equal(both.minz, np.minimum(ma.minz, mb.minz))


def _filled(params, origin, seed):
    rng = np.random.default_rng(seed)
    m = oracle.OracleMap(params, origin)
    m.hits[...] = rng.integers(0, 5, m.hits.shape)
    m.passes[...] = rng.integers(0, 50, m.passes.shape)
    m.minz[...] = np.where(m.hits > 0, rng.normal(size=m.hits.shape), np.inf).astype(np.float32)
    return m


def test_shift_identities():
    params = oracle.OracleParams(nx=9, ny=8, nz=6, res=0.2)
    base = _filled(params, (3, -4, 2), 1)
    # zero shift is the identity
    m = base.copy()
    m.shift_to((3, -4, 2))
    np.testing.assert_array_equal(m.hits, base.hits)
    np.testing.assert_array_equal(m.minz, base.minz)
    # shift(a) then shift(b) equals shift(a + b) on cells inside all windows
    for a, b in (((2, 0, 0), (1, -3, 1)), ((-4, 2, -1), (3, 3, 2)), ((0, 0, 5), (0, -1, -5))):
        m1 = base.copy()
        m1.shift_to(base.origin + np.array(a))
        m1.shift_to(base.origin + np.array(a) + np.array(b))
        m2 = base.copy()
        m2.shift_to(base.origin + np.array(a) + np.array(b))
        lo = np.maximum.reduce([np.zeros(3, int), np.array(a), np.array(a) + np.array(b)]) - (np.array(a) + np.array(b))
        hi = np.minimum.reduce([np.array([9, 8, 6]), np.array([9, 8, 6]) + np.array(a),
                                np.array([9, 8, 6]) + np.array(a) + np.array(b)]) - (np.array(a) + np.array(b))
        sl = tuple(slice(max(l, 0), max(h, 0)) for l, h in zip(lo, hi))
        np.testing.assert_array_equal(m1.hits[sl], m2.hits[sl])
        np.testing.assert_array_equal(m1.passes[sl], m2.passes[sl])
        np.testing.assert_array_equal(m1.minz[sl], m2.minz[sl])
    # a cell that stays keeps its value at the offset index
    m = base.copy()
    m.shift_to(base.origin + np.array([2, -1, 1]))
    np.testing.assert_array_equal(m.hits[:7, 1:, :5], base.hits[2:, :7, 1:])
    # entering cells are empty
    assert (m.hits[7:] == 0).all() and (m.passes[:, :1] == 0).all() and np.isinf(m.minz[:, :, 5:]).all()
    # a shift by at least the window clears everything
    m = base.copy()
    m.shift_to(base.origin + np.array([9, 0, 0]))
    assert m.hits.sum() == 0 and m.passes.sum() == 0 and np.isinf(m.minz).all()


def test_shift_then_ingest_equals_ingest_then_shift_on_overlap():
    # the world-fixed traversal does not depend on the window: with exact
    # endpoints, counts of cells inside both windows agree either way
    params = small_params(nx=10, ny=9, nz=6)
    rng = np.random.default_rng(21)
    T = YAW90.copy()
    T[:, 3] = (1.25, 1.0, 0.5)
    pts = grid_points(rng, 60, -2.0, 2.0)
    o1 = np.array([0, 0, 0])
    o2 = np.array([2, -1, 1])
    a = oracle.OracleMap(params, o1)
    a.ingest(pts, T)
    a.shift_to(o2)
    b = oracle.OracleMap(params, o1)
    b.shift_to(o2)
    b.ingest(pts, T)
    sl = (slice(0, 8), slice(1, 9), slice(0, 5))
    np.testing.assert_array_equal(a.hits[sl], b.hits[sl])
    np.testing.assert_array_equal(a.passes[sl], b.passes[sl])
    np.testing.assert_array_equal(a.minz[sl], b.minz[sl])


def test_origin_for_pose_exact_values():
    params = oracle.OracleParams(nx=128, ny=128, nz=32, res=0.2)
    assert list(oracle.origin_for_pose(params, (0.0, 0.0, 0.0))) == [-64, -64, -16]
    assert list(oracle.origin_for_pose(params, (1.0, -1.0, 0.39))) == [5 - 64, -5 - 64, 1 - 16]
    assert list(oracle.origin_for_pose(params, (-0.01, 0.19, -0.2))) == [-1 - 64, 0 - 64, -1 - 16]
    p2 = oracle.OracleParams(nx=7, ny=6, nz=5, res=0.25)
    assert list(oracle.origin_for_pose(p2, (2.6, 0.24, -1.0))) == [10 - 3, 0 - 3, -4 - 2]


def test_sensor_outside_window_counts_only_inside_cells():
    params = small_params()
    rng = np.random.default_rng(8)
    T = IDENTITY.copy()
    T[:, 3] = (-1.0, 0.75, 0.5)  # 4 voxels left of the window
    pts = grid_points(rng, 30, 0.0, 2.5)
    origin = np.zeros(3, np.int64)
    m = oracle.OracleMap(params, origin)
    m.ingest(pts, T)
    hits, passes, minz, _ = brute_update(params, origin, pts, T)
    np.testing.assert_array_equal(m.passes, passes)
    np.testing.assert_array_equal(m.hits, hits)


def test_lut_encoding_hand_built_and_round_trip():
    # Sec. III-A: occupied voxels index the data array in linear order;
    # other voxels hold -1 - misses
    params = oracle.OracleParams(nx=2, ny=2, nz=3, res=0.2)
    hits = np.zeros((2, 2, 3), np.uint32)
    passes = np.zeros((2, 2, 3), np.uint32)
    minz = np.full((2, 2, 3), np.inf, np.float32)
    hits[0, 0, 2], passes[0, 0, 2], minz[0, 0, 2] = 2, 5, 0.5
    hits[1, 0, 0], passes[1, 0, 0], minz[1, 0, 0] = 1, 0, -0.25
    passes[0, 1, 1] = 7
    passes[1, 1, 2] = 4294967295  # the largest miss count stays exact
    table, data = oracle.lut(params, hits, passes, minz)
    expect = np.array([[[-1, -1, 0], [-1, -8, -1]], [[1, -1, -1], [-1, -1, -1 - 4294967295]]], np.int64)
    np.testing.assert_array_equal(table, expect)
    np.testing.assert_array_equal(data["hits"], [2, 1])
    np.testing.assert_array_equal(data["passes"], [5, 0])
    np.testing.assert_array_equal(data["minz"], np.float32([0.5, -0.25]))


def test_lut_round_trip_random_state():
    rng = np.random.default_rng(12)
    params = oracle.OracleParams(nx=9, ny=7, nz=5, res=0.2)
    m = _filled(params, (0, 0, 0), 3)
    table, data = oracle.lut(params, m.hits, m.passes, m.minz)
    occ = table >= 0
    assert np.array_equal(occ, m.hits > 0)
    idx = table[occ]
    assert np.array_equal(idx, np.arange(len(idx)))  # rising with the linear index
    np.testing.assert_array_equal(data["hits"][idx], m.hits[occ])
    np.testing.assert_array_equal(data["passes"][idx], m.passes[occ])
    np.testing.assert_array_equal(data["minz"][idx], m.minz[occ])
    np.testing.assert_array_equal(-1 - table[~occ], m.passes[~occ].astype(np.int64))
