"""Pins of the oracle's column reduction + transpose (paper Sec. 5.1) against
numpy's sort, exact arithmetic on integers, and the layout definition."""
import numpy as np
import pytest

import oracle


def _q4(x, dmax):
    """Q4 code by the reading: NaN / <= 0 -> 0, >= dmax -> 16 dmax, else round(16 x) half to even."""
    x = np.asarray(x, np.float32)
    with np.errstate(invalid="ignore"):
        q = np.rint(np.float32(16) * x)
        q = np.where(np.isnan(x) | (x <= 0), 0, np.where(x >= dmax, 16 * dmax, q))
    return q.astype(np.int64)


def _nasty_image(rng, H, W, dmax):
    D = rng.uniform(-2, dmax + 3, size=(H, W)).astype(np.float32)
    D[rng.random((H, W)) < 0.05] = np.nan
    D[rng.random((H, W)) < 0.05] = 0.0
    halves = rng.random((H, W)) < 0.1                  # exact 1/32 multiples: rounding ties
    D[halves] = (rng.integers(0, 32 * dmax, size=int(halves.sum())) / 32.0).astype(np.float32)
    D[rng.random((H, W)) < 0.02] = np.inf
    return D


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 7, 8, 11, 16])
def test_median_matches_sorted_middle(s):
    rng = np.random.default_rng(s)
    H, W, dmax = 23, 5 * s + (s - 1), 64           # ragged: W mod s pixels are dropped
    D = _nasty_image(rng, H, W, dmax)
    q = oracle.reduce(D, s, dmax, mode=0)
    C = W // s
    assert q.shape == (C, H)
    codes = _q4(D, dmax)
    for c in range(C):
        for r in range(H):
            vals = np.sort(codes[r, c * s:(c + 1) * s])
            assert q[c, H - 1 - r] == vals[(s - 1) // 2]


def test_q4_code_is_within_half_step_and_ties_to_even():
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 64, size=4000).astype(np.float32)
    x[:200] = ((2 * np.arange(200) + 1) / 32.0).astype(np.float32)      # 16 x = i + 1/2 exactly
    D = x.reshape(1, -1)
    q = oracle.reduce(D, 1, 64, mode=0)[:, 0]
    assert np.all(np.abs(q / 16.0 - x) <= 1.0 / 32)
    ties = q[:200]
    assert np.all(ties % 2 == 0)                      # halves go to the even code


@pytest.mark.parametrize("s", [2, 3, 5, 6])
def test_mean_mode_rounds_half_up(s):
    rng = np.random.default_rng(11 + s)
    H, W, dmax = 17, 4 * s, 128
    D = _nasty_image(rng, H, W, dmax)
    q = oracle.reduce(D, s, dmax, mode=1)
    codes = _q4(D, dmax)
    for c in range(W // s):
        for r in range(H):
            tot = int(codes[r, c * s:(c + 1) * s].sum())
            m = q[c, H - 1 - r]
            assert m - 0.5 <= tot / s < m + 0.5             # nearest integer to the exact mean, halves up


def test_layout_bottom_up_column_major():
    H, W, s = 9, 12, 3
    D = np.zeros((H, W), np.float32)
    for r in range(H):
        for x in range(W):
            D[r, x] = r + 10 * (x // s)                  # row index + 10 * column
    q = oracle.reduce(D, s, 64, mode=0)
    for c in range(W // s):
        for v in range(H):
            assert q[c, v] == 16 * ((H - 1 - v) + 10 * c)


# ---- whole-pixel grid (the integer disparities of Sec. 3.4's LUT_cost variant)

def test_pixel_grid_rounds_to_the_nearest_whole_pixel_halves_up():
    # px value -> expected code, from the definition: the Q4 code first (16 x
    # rounded, halves to even), then the nearest whole pixel of that code,
    # halves up, times 16.  The two roundings compose: 3.49 px is Q4 56 = 3.5 px
    # and so 4 px; 0.47 px is Q4 8 = 0.5 px and so 1 px; 2.46875 px is Q4 40.
    cases = [(0.0, 0), (2.0, 32), (2.4375, 32), (2.46875, 48), (2.5, 48), (2.5625, 48), (3.49, 64),
             (3.46, 48), (63.5, 1024), (64.0, 1024), (70.0, 1024), (-1.0, 0), (float("nan"), 0),
             (0.5, 16), (0.47, 16), (0.4, 0)]
    x = np.array([c[0] for c in cases], np.float32).reshape(1, -1)
    q = oracle.reduce(x, 1, 64, mode=0, pixel_grid=1)[:, 0]
    assert list(q) == [c[1] for c in cases]


@pytest.mark.parametrize("s,mode", [(1, 0), (1, 1), (3, 0), (5, 0), (4, 0)])
def test_pixel_grid_is_the_identity_on_whole_pixel_inputs(s, mode):
    # integer disparities stay on the whole-pixel grid through clamping and the
    # median (and through any reduction when s = 1)
    rng = np.random.default_rng(40 + s)
    D = rng.integers(-3, 70, size=(13, 6 * s)).astype(np.float32)
    a = oracle.reduce(D, s, 64, mode=mode, pixel_grid=0)
    b = oracle.reduce(D, s, 64, mode=mode, pixel_grid=1)
    assert np.array_equal(a, b)
    assert np.all(b % 16 == 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_pixel_grid_is_within_half_a_pixel_of_the_q4_reduction(mode):
    rng = np.random.default_rng(50 + mode)
    D = _nasty_image(rng, 19, 25, 96)
    a = oracle.reduce(D, 5, 96, mode=mode, pixel_grid=0).astype(np.int64)
    b = oracle.reduce(D, 5, 96, mode=mode, pixel_grid=1).astype(np.int64)
    assert np.all(b % 16 == 0)
    assert np.all((a - 8 < b) & (b <= a + 8))          # a - 1/2 px < b <= a + 1/2 px (halves up)
    assert np.all((0 <= b) & (b <= 16 * 96))
