"""The frame's ground line from its v-disparity (the step before the path):
the estimate (slope, horizon, votes) and whole frames computed with it must
equal the oracle's exactly; the camera's line is kept when nothing votes; the
paths that do not support the estimate refuse it (batched and served frames:
test_gpu_batch_variants.py)."""
import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import assert_frame_equal, cuda  # noqa: E402

WRONG = dict(horizon_row=10, baseline_m=0.2)       # camera parameters the estimate overrides


def _scenes():
    out = [(scenes.CONFIG1, scenes.make_scene(scenes.CONFIG1, 6000, n_obstacles=(3, 6))),
           (scenes.CONFIG1, scenes.make_scene(scenes.CONFIG1, 6001, n_obstacles=(3, 6), integer_disp=True,
                                              noise_sigma=0, p_outlier=0, p_invalid=0)),
           (scenes.CONFIG2, scenes.make_scene(scenes.CONFIG2, 6002, n_obstacles=(8, 20))),
           (scenes.Camera(83, 97, stixel_width=5, dmax=48, horizon_row=30, baseline_m=0.4, camera_height_m=1.0),
            None)]
    cam = out[-1][0]
    out[-1] = (cam, scenes.make_scene(cam, 6003, n_obstacles=(1, 3), span_cols=(1, 6)))
    return out


@pytest.mark.parametrize("i", range(4))
def test_estimate_equals_oracle(i):
    cam, sc = _scenes()[i]
    h = S.Stixels(S.default_params(cam, ground_estimate=1))
    q = h.reduce(cuda(sc.disparity))
    ncols = cam.width // cam.stixel_width
    got = h.estimate_ground(q, cam.height, ncols)
    ref = oracle.ground_estimate(oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax), cam.dmax)
    assert got == ref
    h.close()


def test_estimate_equals_oracle_2048x880():
    cam = scenes.CONFIG3[-1]
    sc = scenes.make_scene(cam, 6010, n_obstacles=(8, 20))
    h = S.Stixels(S.default_params(cam, ground_estimate=1))
    q = h.reduce(cuda(sc.disparity))
    got = h.estimate_ground(q, cam.height, cam.width // cam.stixel_width)
    ref = oracle.ground_estimate(oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax), cam.dmax)
    assert got == ref
    h.close()


@pytest.mark.parametrize("W, H, dmax, horizon, seed", [
    (1000, 2048, 128, 700, 6020),     # the tallest column: 16 vote CTAs per slope
    (1000, 1800, 255, 600, 6024),     # the largest disparity range the fixed-point budget allows at this
                                      # height: 4081 codes per histogram row (the 65.7 KB shared-memory opt-in)
    (40, 1, 16, 0, 6021),             # one row: no line has a row above its horizon
    (40, 3, 16, 1, 6022),             # a partial group of four histogram rows
    (45, 6, 4, 2, 6023)])
def test_estimate_equals_oracle_at_the_limits(W, H, dmax, horizon, seed):
    cam = scenes.Camera(W, H, stixel_width=5, dmax=dmax, horizon_row=horizon, baseline_m=0.4, camera_height_m=1.0)
    sc = scenes.make_scene(cam, seed, n_obstacles=(2, 4), span_cols=(1, 6))
    h = S.Stixels(S.default_params(cam, ground_estimate=1))
    q = h.reduce(cuda(sc.disparity))
    got = h.estimate_ground(q, cam.height, cam.width // cam.stixel_width)
    ref = oracle.ground_estimate(oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax), cam.dmax)
    assert got == ref
    h.close()


@pytest.mark.parametrize("k0,h0,copies", [(40, 30, 1), (40, 30, 2), (100, 10, 1), (7, 5, 3), (256, 60, 2)])
def test_votes_of_a_planted_line_are_the_triangle_peak_per_row(k0, h0, copies):
    """Codes exactly on the line (k0, h0) in identical columns, fed to the
    estimate directly: that line with 17 votes per column and row whose code
    lies in [16, 16 dmax] (the closed form the oracle is pinned to)."""
    H, dmax = 100, 64
    r = np.arange(H)
    code = np.where(r > h0, (k0 * (r - h0) + 8) >> 4, 0)
    rows = int(((code >= 16) & (code <= 16 * dmax)).sum())
    q = np.tile(code[::-1].astype(np.int16), (copies, 1))
    cam = scenes.Camera(5 * copies, H, stixel_width=5, dmax=dmax, horizon_row=30, baseline_m=0.4,
                        camera_height_m=1.0)
    h = S.Stixels(S.default_params(cam, ground_estimate=1))
    got = h.estimate_ground(torch.from_numpy(q).cuda(), H, copies)
    assert got == (k0, h0, 17 * copies * rows) == oracle.ground_estimate(q, dmax)
    h.close()


@pytest.mark.parametrize("i", range(4))
def test_frames_with_the_estimate_equal_oracle(i):
    cam, sc = _scenes()[i]
    lp = S.default_params(cam, ground_estimate=1, **WRONG)
    op = oracle.make_params(cam, ground_estimate=1, **WRONG)
    h = S.Stixels(lp)
    out = h.compute(cuda(sc.disparity))
    torch.cuda.synchronize()
    res = S.Stixels.to_host(out)
    err = h.get_error()
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == (S.ERR_CAPACITY if (fr.counts > lp.max_stixels_per_col).any() else 0)
    assert_frame_equal(res, fr, cam.height, lp.max_stixels_per_col, op)
    # and through host buffers
    st, counts, cost, rc = h.compute_host(sc.disparity)
    assert np.array_equal(counts, res[1]) and np.array_equal(cost, res[2])
    h.close()


def test_no_ground_keeps_the_camera_line():
    cam = scenes.CONFIG1
    D = np.zeros((cam.height, cam.width), np.float32)
    a, b = S.Stixels(S.default_params(cam)), S.Stixels(S.default_params(cam, ground_estimate=1))
    q = b.reduce(cuda(D))
    assert b.estimate_ground(q, cam.height, cam.width // cam.stixel_width)[2] == 0
    ra, rb = S.Stixels.to_host(a.compute(cuda(D))), S.Stixels.to_host(b.compute(cuda(D)))
    torch.cuda.synchronize()
    assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[3], rb[3])


def test_unsupported_paths_refuse_the_estimate():
    cam = scenes.CONFIG1
    with pytest.raises(S.StixelsError):
        S.Stixels(S.default_params(cam, ground_estimate=1, sigma_gain=0.5))
    h = S.Stixels(S.default_params(cam, ground_estimate=1))
    h.reserve(cam.height, cam.width)
    out = h.alloc_output(cam.height, cam.width)
    with pytest.raises(S.StixelsError):
        h.compute_noalloc(cuda(np.zeros((cam.height, cam.width), np.float32)), out)
    plain = S.Stixels(S.default_params(cam))
    q = plain.reduce(cuda(np.zeros((cam.height, cam.width), np.float32)))
    with pytest.raises(S.StixelsError):
        plain.estimate_ground(q, cam.height, cam.width // cam.stixel_width)
