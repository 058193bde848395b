"""Pins of the oracle's v-disparity ground estimate (the paper assumes the
ground slope and horizon known per image, Sec. 3; this step supplies them from
the frame): exact recovery of planted ground lines, bounded error under the
benchmark's noise, equality of the whole frame with the camera-parameter
result when the estimate is exact, and the fallback when no ground is seen."""
import numpy as np
import pytest

import oracle
import scenes

# (baseline, camera height) pairs whose slope alpha = b / h is a multiple of 1/256
EXACT = [(0.3, 1.2, 64), (0.5, 1.0, 128), (0.3, 1.6, 48)]


def _cam(b, h, horizon, W=320, H=120, dmax=64):
    return scenes.Camera(W, H, stixel_width=5, dmax=dmax, focal_px=700.0, baseline_m=b, camera_height_m=h,
                         pitch_rad=0.0, horizon_row=horizon)


@pytest.mark.parametrize("b,h,k", EXACT)
@pytest.mark.parametrize("horizon", [30, 40, 71])
def test_planted_ground_line_is_recovered_exactly(b, h, k, horizon):
    cam = _cam(b, h, horizon)
    if cam.alpha * (cam.height - 1 - horizon) > cam.dmax:
        pytest.skip("ground leaves the disparity range")
    for obstacles in [(0, 0), (2, 4)]:
        sc = scenes.make_scene(cam, 900 + horizon, n_obstacles=obstacles, integer_disp=True, noise_sigma=0,
                               p_outlier=0, p_invalid=0)
        q = oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax)
        kk, hh, votes = oracle.ground_estimate(q, cam.dmax)
        assert (kk, hh) == (k, horizon), obstacles
        assert votes > 0


@pytest.mark.parametrize("k0,h0,copies", [(40, 30, 1), (40, 30, 2), (100, 10, 1), (7, 5, 3), (256, 60, 2)])
def test_votes_of_a_planted_line_are_the_triangle_peak_per_row(k0, h0, copies):
    """Codes exactly on the line (k0, h0) in `copies` identical columns: each
    row whose code lies in [16, 16 dmax] gives that line the smoothing
    triangle's peak weight 17 once per column, and every other line gets less
    on some row, so the estimate is that line with 17 * copies * rows votes
    (a closed form of the histogram, the triangle's weights and the row range)."""
    H, dmax = 100, 64
    r = np.arange(H)
    code = np.where(r > h0, (k0 * (r - h0) + 8) >> 4, 0)
    rows = int(((code >= 16) & (code <= 16 * dmax)).sum())
    q = np.tile(code[::-1].astype(np.int16), (copies, 1))       # bottom-up: v = H - 1 - r
    assert oracle.ground_estimate(q, dmax) == (k0, h0, 17 * copies * rows)


@pytest.mark.parametrize("seed", range(4))
def test_noisy_ground_line_is_close(seed):
    cam = scenes.CONFIG2                                   # alpha = 0.25 (k = 64), horizon 180
    sc = scenes.make_scene(cam, 5000 + seed, n_obstacles=(8, 20))
    q = oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax)
    kk, hh, _ = oracle.ground_estimate(q, cam.dmax)
    assert abs(kk - 64) <= 2 and abs(hh - cam.horizon_row) <= 3, (kk, hh)


def test_frame_with_an_exact_estimate_equals_the_camera_frame():
    cam = _cam(0.3, 1.2, 40)
    sc = scenes.make_scene(cam, 4500, n_obstacles=(3, 6), integer_disp=True, noise_sigma=0, p_outlier=0,
                           p_invalid=0)
    a = oracle.frame(oracle.make_params(cam), sc.disparity, cap=64)
    wrong = dict(horizon_row=10, baseline_m=0.2)           # camera parameters the estimate must override
    b = oracle.frame(oracle.make_params(cam, ground_estimate=1, **wrong), sc.disparity, cap=64)
    c = oracle.frame(oracle.make_params(cam, **wrong), sc.disparity, cap=64)
    assert np.array_equal(a.cost, b.cost) and np.array_equal(a.counts, b.counts)
    assert not np.array_equal(a.cost, c.cost)
    for col in range(len(a.counts)):
        assert np.array_equal(a.stixels[col, :a.counts[col]], b.stixels[col, :b.counts[col]])


def test_no_ground_seen_keeps_the_camera_line():
    cam = scenes.CONFIG1
    D = np.zeros((cam.height, cam.width), np.float32)       # all sky / invalid: no vote anywhere
    q = oracle.reduce(D, cam.stixel_width, cam.dmax)
    assert oracle.ground_estimate(q, cam.dmax)[2] == 0
    a = oracle.frame(oracle.make_params(cam), D, cap=64)
    b = oracle.frame(oracle.make_params(cam, ground_estimate=1), D, cap=64)
    assert np.array_equal(a.cost, b.cost)
