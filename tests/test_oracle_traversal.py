"""Pins the oracle's ray traversal to an exact brute force (Sec. III-A misses,
Sec. III-C ray tracing).

The brute force tests every cell of a small grid directly against the
definition: the closed segment A + t (B - A), t in [0, 1], meets the
half-open cell [256 c, 256 (c + 1))^3 iff the per-axis t-intervals, with
their open and closed ends, intersect. It uses exact rationals and shares
nothing with the oracle's event walk.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _axis_interval(a, d, c):
    """t-interval (lo, lo_closed, hi, hi_closed) where 256c <= a + t d < 256(c+1)."""
    lo_b, hi_b = 256 * c, 256 * (c + 1)
    if d == 0:
        if lo_b <= a < hi_b:
            return (Fraction(0), True, Fraction(1), True)
        return None
    if d > 0:
        return (Fraction(lo_b - a, d), True, Fraction(hi_b - a, d), False)
    # d < 0: a + t d >= lo_b  <=>  t <= (a - lo_b)/|d|; a + t d < hi_b <=> t > (a - hi_b)/|d|
    return (Fraction(a - hi_b, -d), False, Fraction(a - lo_b, -d), True)


def meets(A, B, cell):
    lo, lo_c, hi, hi_c = Fraction(0), True, Fraction(1), True
    for a, b, c in zip(A, B, cell):
        iv = _axis_interval(a, b - a, c)
        if iv is None:
            return False
        l, lc, h, hc = iv
        if l > lo or (l == lo and not lc):
            lo, lo_c = l, lc
        if h < hi or (h == hi and not hc):
            hi, hi_c = h, hc
    return lo < hi or (lo == hi and lo_c and hi_c)


def brute_cells(A, B, lo=-2, hi=8):
    out = set()
    for c in itertools.product(range(lo, hi), repeat=3):
        if meets(A, B, c):
            out.add(c)
    return out


def check_walk(A, B):
    cells = [tuple(int(v) for v in c) for c in oracle.traverse_cells(A, B)]
    # order: first is the start cell, last the endpoint cell, no repeats, and
    # each move changes every axis by at most one voxel in the ray's direction
    assert cells[0] == tuple(a // 256 for a in A)
    assert cells[-1] == tuple(b // 256 for b in B)
    assert len(set(cells)) == len(cells)
    for u, v in zip(cells, cells[1:]):
        for ax in range(3):
            step = v[ax] - u[ax]
            assert step in (0, int(np.sign(B[ax] - A[ax])))
    span = [min(min(a, b) // 256 for a, b in zip(A, B)) - 1, max(max(a, b) // 256 for a, b in zip(A, B)) + 2]
    assert set(cells) == brute_cells(A, B, span[0], span[1])
    return cells


def test_random_segments_match_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(300):
        A = [int(v) for v in rng.integers(-256, 256 * 5, 3)]
        B = [int(v) for v in rng.integers(-256, 256 * 5, 3)]
        check_walk(A, B)


def test_boundary_aligned_segments_match_brute_force():
    # endpoints on faces, edges and corners of cells (multiples of 128 / 256)
    rng = np.random.default_rng(12)
    for _ in range(300):
        A = [int(v) * 128 for v in rng.integers(-2, 10, 3)]
        B = [int(v) * 128 for v in rng.integers(-2, 10, 3)]
        check_walk(A, B)


def test_all_26_direction_sign_patterns():
    centre = [640, 640, 640]
    for s in itertools.product((-1, 0, 1), repeat=3):
        if s == (0, 0, 0):
            continue
        for mag in ([300, 517, 771], [256, 512, 768], [512, 512, 512]):
            B = [c + si * m for c, si, m in zip(centre, s, mag)]
            check_walk(centre, B)
            check_walk([c + 1 for c in centre], B)


def test_zero_length_is_one_cell():
    for A in ([0, 0, 0], [255, 256, -1], [-256, 511, 1000]):
        cells = check_walk(A, A)
        assert len(cells) == 1


def test_axis_aligned_counts():
    # along one axis the walk meets |floor(b/256) - floor(a/256)| + 1 cells
    for a, b in ((10, 900), (900, 10), (256, 1024), (1024, 256), (-300, 300)):
        for ax in range(3):
            A = [100, 100, 100]
            B = [100, 100, 100]
            A[ax], B[ax] = a, b
            cells = check_walk(A, B)
            assert len(cells) == abs(b // 256 - a // 256) + 1


def test_exact_diagonal_through_corner_takes_no_side_cells():
    # both axes cross together at t = 1/4 and 3/4 (upward: at t; downward: just after t)
    assert [tuple(c) for c in oracle.traverse_cells([128, 128, 5], [640, 640, 5])] == \
        [(0, 0, 0), (1, 1, 0), (2, 2, 0)]
    assert [tuple(c) for c in oracle.traverse_cells([640, 640, 5], [128, 128, 5])] == \
        [(2, 2, 0), (1, 1, 0), (0, 0, 0)]
    # mixed: x up and y down cross at the same t; the upward step comes first
    assert [tuple(c) for c in oracle.traverse_cells([128, 640, 5], [640, 128, 5])] == \
        [(0, 2, 0), (1, 2, 0), (1, 1, 0), (2, 1, 0), (2, 0, 0)]


@pytest.mark.parametrize("seed", [0, 1])
def test_long_segments_match_brute_force_sampled(seed):
    # longer rays (tens of cells): compare the walk to the brute force on a
    # box around the segment
    rng = np.random.default_rng(100 + seed)
    for _ in range(5):
        A = [int(v) for v in rng.integers(0, 256 * 3, 3)]
        B = [int(v) for v in rng.integers(256 * 10, 256 * 16, 3)]
        B[int(rng.integers(0, 3))] = int(rng.integers(0, 256 * 3))
        cells = [tuple(int(v) for v in c) for c in oracle.traverse_cells(A, B)]
        lo = min(min(a, b) // 256 for a, b in zip(A, B)) - 1
        hi = max(max(a, b) // 256 for a, b in zip(A, B)) + 2
        assert set(cells) == brute_cells(A, B, lo, hi)
