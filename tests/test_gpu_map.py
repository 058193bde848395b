"""The global MAP (ordering prior exact, object states carry their disparity):
GPU frames must equal the oracle's element by element; without the ordering
prior it must agree with the paper's DP; the scratch-free entry point refuses
it (batched and served frames: test_gpu_batch_variants.py)."""
import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import assert_frame_equal, both_params, cuda, run_frame  # noqa: E402


@pytest.mark.parametrize("seed", [7000, 7001, 7002])
def test_global_map_config1(seed):
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, seed, n_obstacles=(3, 6))
    lp, op = both_params(cam, global_map=1, cost_order=2.5)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == 0
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("H", [1, 2, 31, 33, 97])
def test_global_map_ragged_heights(H):
    cam = scenes.Camera(83, H, stixel_width=5, dmax=48, horizon_row=max(0, H // 3), baseline_m=0.4,
                        camera_height_m=1.0)
    sc = scenes.make_scene(cam, 700 + H, n_obstacles=(1, 4), span_cols=(1, 6))
    lp, op = both_params(cam, global_map=1, cost_order=3.0, eps_order=-0.5)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert_frame_equal(out, fr, H, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("variant", [
    dict(pixel_grid=1, reduce_mode=1),
    dict(sigma_gain=1.0, sigma_mid=30.0, sigma_width=8.0),
    dict(prior_trans=((1.5, 1.0, 4.0), (1.5, 6.0, 9.0), (0.5, 0.5, 7.0)), prior_first=(0.3, 0.3, 0.3)),
])
def test_global_map_model_variants(variant):
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 7100, n_obstacles=(3, 6))
    lp, op = both_params(cam, global_map=1, **variant)
    out, _ = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


def test_global_map_paper_size_sampled_columns():
    """1024x440 s=5 dmax 128 on the GPU; the oracle (O(H^2 dmax) per column) checks
    a spread of columns one by one, from its own reduction of the frame."""
    cam = scenes.CONFIG2
    sc = scenes.make_scene(cam, 7200, n_obstacles=(8, 20))
    lp, op = both_params(cam, global_map=1)
    (st, counts, cost, cost_fixed), _ = run_frame(lp, sc.disparity)
    q = oracle.reduce(sc.disparity, cam.stixel_width, cam.dmax)
    H, cap = cam.height, lp.max_stixels_per_col
    for c in [0, 17, 63, 101, 150, 203]:
        col = oracle.column(op, q[c], cap=cap)
        assert counts[c] == len(col.stixels) or counts[c] > cap
        assert cost_fixed[c] == np.int64(col.cost * S.UNITS_PER_COST)
        n = min(int(counts[c]), cap)
        assert np.array_equal(st[c, :n]["row_top"], H - 1 - col.stixels[:n]["v_top"])
        assert np.array_equal(st[c, :n]["row_bottom"], H - 1 - col.stixels[:n]["v_bottom"])
        assert np.array_equal(st[c, :n]["cls"], col.stixels[:n]["cls"])


def test_without_ordering_global_map_costs_equal_the_paper_dp():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 7300, n_obstacles=(3, 6))
    a, _ = run_frame(S.default_params(cam, cost_order=0.0), sc.disparity)
    b, _ = run_frame(S.default_params(cam, cost_order=0.0, global_map=1), sc.disparity)
    assert np.array_equal(a[3], b[3])
    c, _ = run_frame(S.default_params(cam, cost_order=2.5), sc.disparity)
    d, _ = run_frame(S.default_params(cam, cost_order=2.5, global_map=1), sc.disparity)
    assert np.all(d[3] <= c[3])


def test_the_scratch_free_entry_point_refuses_global_map():
    cam = scenes.CONFIG1
    h = S.Stixels(S.default_params(cam, global_map=1))
    h.reserve(cam.height, cam.width)
    out = h.alloc_output(cam.height, cam.width)
    with pytest.raises(S.StixelsError):
        h.compute_noalloc(cuda(np.zeros((cam.height, cam.width), np.float32)), out)


def test_global_map_tall_columns_with_the_largest_dmax():
    """A column's global-MAP state (its current block's bins and rows of the
    ordering table, the state values of every row) lives in one CTA's shared
    memory; tall columns at dmax 255 fit and match the oracle."""
    cam = scenes.Camera(10, 1800, stixel_width=5, dmax=255, horizon_row=600, baseline_m=0.4, camera_height_m=1.0)
    sc = scenes.make_scene(cam, 7400, n_obstacles=(1, 2), span_cols=(1, 2))
    lp, op = both_params(cam, global_map=1)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)
