"""The seeded input generator (inputs only: it does none of the method's
arithmetic) makes the frames its recipe states: the flat-ground line below the
horizon and sky above it, obstacles standing on the ground and painted far to
near, then the stated noise, outlier and invalid-pixel rates, clamped to
[0, dmax]; the same seed gives the same bytes."""
import numpy as np
import pytest

import scenes


def test_same_seed_same_bytes_and_different_seeds_differ():
    cam = scenes.CONFIG1
    a = scenes.make_scene(cam, 11).disparity
    b = scenes.make_scene(cam, 11).disparity
    c = scenes.make_scene(cam, 12).disparity
    assert a.dtype == np.float32 and a.shape == (cam.height, cam.width)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("cam", [scenes.CONFIG1, scenes.CONFIG2])
def test_noise_free_frame_is_ground_sky_and_obstacles(cam):
    sc = scenes.make_scene(cam, 21, n_obstacles=(3, 6), integer_disp=True, noise_sigma=0, p_outlier=0,
                           p_invalid=0)
    D, lab = sc.disparity, sc.labels
    r = np.arange(cam.height)[:, None].repeat(cam.width, axis=1)
    ground = np.clip(cam.alpha * (r - cam.horizon_row), 0, cam.dmax)
    assert np.allclose(D[lab == 1], ground[lab == 1], atol=1e-4)     # ground: the flat-ground line
    assert np.all(r[lab == 1] > cam.horizon_row)
    assert np.all(D[lab == 2] == 0) and np.all(r[lab == 2] <= cam.horizon_row)   # sky above the horizon
    assert np.array_equal(D[lab == 0], sc.obj_disp[lab == 0])        # obstacles: their own disparity
    for d, c0, span, top, bottom in sc.obstacles:
        assert d == int(d) and 0 <= top <= bottom < cam.height
        assert 0 <= c0 and c0 + span <= cam.ncols
        # it stands on the ground: its base row is where the ground has its disparity
        assert bottom == min(cam.height - 1, int(round(cam.horizon_row + d / cam.alpha)))
    # far to near: where two obstacles overlap, the nearer (larger disparity) is seen
    for d, c0, span, top, bottom in sc.obstacles:
        seen = sc.obj_disp[top:bottom + 1, c0 * cam.stixel_width:(c0 + span) * cam.stixel_width]
        assert np.all(seen >= d)


def test_noise_rates_and_clamp():
    cam = scenes.CONFIG2
    sc = scenes.make_scene(cam, 31, n_obstacles=(8, 20))
    clean = scenes.make_scene(cam, 31, n_obstacles=(8, 20), noise_sigma=0, p_outlier=0, p_invalid=0)
    D = sc.disparity
    assert D.min() >= 0 and D.max() <= cam.dmax
    zeros_where_clean_positive = np.mean((D == 0) & (clean.disparity > 3))
    assert 0.015 < zeros_where_clean_positive / np.mean(clean.disparity > 3) < 0.025     # 2 % invalid
    far = np.abs(D - clean.disparity) > 6                          # beyond 6 sigma: outliers (and invalid)
    assert 0.04 < far.mean() < 0.09                                # 5 % uniform outliers, 2 % invalid
    resid = (D - clean.disparity)[~far & (clean.disparity > 6) & (clean.disparity < cam.dmax - 6)]
    assert abs(resid.std() - 1.0) < 0.05 and abs(resid.mean()) < 0.02          # sigma = 1 px
