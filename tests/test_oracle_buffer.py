"""Pins of the oracle's map buffer (Sec. III-A / III-B: per-scan maps held in
a buffer of the last K scans and combined by summing counts and taking the
lowest return), against identities that fix it independently of its code:
an unbounded buffer equals plain accumulation (counts add, shifts are
linear), a one-scan buffer equals a fresh map of the last scan, a sliding
buffer subtracts the evicted scans exactly, and a voxel that leaves the
window and comes back is empty."""
import math

import numpy as np

import oracle


def scan(rng, n, centre):
    pts = rng.normal(scale=[3.0, 3.0, 0.6], size=(n, 3)).astype(np.float32)
    th = rng.uniform(0, 2 * np.pi)
    T = np.array([[math.cos(th), -math.sin(th), 0.0, centre[0]], [math.sin(th), math.cos(th), 0.0, centre[1]],
                  [0.0, 0.0, 1.0, centre[2]]])
    return pts, T


PARAMS = oracle.OracleParams(nx=36, ny=32, nz=16, res=0.25)


def test_unbounded_buffer_equals_accumulation_across_shifts():
    rng = np.random.default_rng(1)
    acc = oracle.OracleMap(PARAMS, (-18, -16, -8))
    buf = oracle.BufferedOracleMap(PARAMS, K=10, origin=(-18, -16, -8))
    o = np.array([-18, -16, -8])
    for step in range(6):
        pts, T = scan(rng, 1500, (o + np.array([18, 16, 8])) * PARAMS.res)
        acc.ingest(pts, T)
        buf.ingest(pts, T)
        o = o + rng.integers(-3, 4, 3)
        acc.shift_to(o)
        buf.shift_to(o)
    np.testing.assert_array_equal(buf.hits, acc.hits)
    np.testing.assert_array_equal(buf.passes, acc.passes)
    np.testing.assert_array_equal(buf.minz, acc.minz)
    assert buf.stats.rays_valid == acc.stats.rays_valid
    a, b = buf.extract(), acc.extract()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_one_scan_buffer_is_a_fresh_map_of_the_last_scan():
    rng = np.random.default_rng(2)
    buf = oracle.BufferedOracleMap(PARAMS, K=1, origin=(-18, -16, -8))
    for step in range(3):
        pts, T = scan(rng, 1200, (0.2 * step, 0.0, 2.0))
        buf.ingest(pts, T)
    fresh = oracle.OracleMap(PARAMS, (-18, -16, -8))
    fresh.ingest(pts, T)
    np.testing.assert_array_equal(buf.hits, fresh.hits)
    np.testing.assert_array_equal(buf.passes, fresh.passes)
    np.testing.assert_array_equal(buf.minz, fresh.minz)


def test_sliding_buffer_subtracts_evicted_scans_exactly():
    rng = np.random.default_rng(3)
    o = (-18, -16, -8)
    scans = [scan(rng, 1000 + 300 * j, (0.3 * j, -0.2 * j, 2.0)) for j in range(5)]
    buf = oracle.BufferedOracleMap(PARAMS, K=2, origin=o)
    everything, evicted = oracle.OracleMap(PARAMS, o), oracle.OracleMap(PARAMS, o)
    for j, (pts, T) in enumerate(scans):
        buf.ingest(pts, T)
        everything.ingest(pts, T)
        if j < 3:
            evicted.ingest(pts, T)
    np.testing.assert_array_equal(buf.hits, everything.hits - evicted.hits)
    np.testing.assert_array_equal(buf.passes, everything.passes - evicted.passes)
    # the lowest return of the last two scans: the minimum of their own maps
    last = [oracle.OracleMap(PARAMS, o) for _ in range(2)]
    for m, (pts, T) in zip(last, scans[3:]):
        m.ingest(pts, T)
    np.testing.assert_array_equal(buf.minz, np.minimum(last[0].minz, last[1].minz))


def test_voxels_that_leave_and_return_are_empty():
    rng = np.random.default_rng(4)
    o = np.array([-18, -16, -8])
    buf = oracle.BufferedOracleMap(PARAMS, K=4, origin=o)
    pts, T = scan(rng, 2000, (0.0, 0.0, 2.0))
    buf.ingest(pts, T)
    assert buf.hits.sum() > 0
    buf.shift_to(o + np.array([40, 0, 0]))   # past the window: everything leaves
    buf.shift_to(o)
    assert buf.hits.sum() == 0 and buf.passes.sum() == 0 and np.isinf(buf.minz).all()
    pts2, T2 = scan(rng, 900, (0.5, 0.1, 2.0))
    buf.ingest(pts2, T2)
    fresh = oracle.OracleMap(PARAMS, o)
    fresh.ingest(pts2, T2)
    np.testing.assert_array_equal(buf.hits, fresh.hits)
    np.testing.assert_array_equal(buf.passes, fresh.passes)
