"""Batched mode: many frames of different sizes, stixel widths, dmax and
camera parameters through one graph-captured launch sequence (persistent DP
over a longest-first column work list).  Each frame's results must equal the
per-frame path's exactly, for every DP launch shape the autotuner can pick."""
import os

import numpy as np
import pytest

import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mixed_frames():
    cams = [
        scenes.Camera(640, 240, stixel_width=5, dmax=64, horizon_row=80),
        scenes.Camera(640, 240, stixel_width=7, dmax=128, horizon_row=80),
        scenes.CONFIG2,
        scenes.Camera(1024, 440, stixel_width=7, dmax=128, horizon_row=180),
        scenes.Camera(333, 97, stixel_width=4, dmax=48, horizon_row=30, baseline_m=0.4, camera_height_m=1.0),
        scenes.CONFIG1,
        scenes.Camera(640, 240, stixel_width=5, dmax=64, horizon_row=80),
        scenes.Camera(640, 240, stixel_width=7, dmax=64, horizon_row=80),
    ]
    out = []
    for i, cam in enumerate(cams):
        kw = {}
        if i == 4:   # a camera with non-standard transitions: the general DP instantiation
            kw = dict(prior_trans=((1.5, 1.0, 4.0), (1.5, 6.0, 9.0), (0.5, 0.5, 7.0)))
        if i == 6:   # the whole-pixel grid (LUT_cost variant), mean reduction
            kw = dict(pixel_grid=1, reduce_mode=1)
        if i == 7:   # disparity-dependent sigma
            kw = dict(sigma_gain=1.2, sigma_mid=30.0, sigma_width=8.0)
        h = S.Stixels(S.default_params(cam, **kw))
        sc = scenes.make_scene(cam, 4400 + i, n_obstacles=(3, 10))
        out.append((h, cam, sc.disparity))
    return out


def _reference(h, disp):
    out = h.compute(torch.from_numpy(disp).cuda())
    torch.cuda.synchronize()
    return S.Stixels.to_host(out)


def _assert_same(got, ref, cap):
    st, cnt, cost, fix = got
    r_st, r_cnt, r_cost, r_fix = ref
    assert np.array_equal(cnt, r_cnt)
    assert np.array_equal(fix, r_fix) and np.array_equal(cost, r_cost)
    for c in range(len(cnt)):
        n = min(int(cnt[c]), cap)
        assert np.array_equal(st[c, :n], r_st[c, :n])


def test_batch_equals_per_frame_for_every_launch_shape():
    frames = _mixed_frames()
    refs = [_reference(h, d) for h, _, d in frames]
    b = S.Batch([(h, cam.height, cam.width) for h, cam, _ in frames])
    for i, (_, _, d) in enumerate(frames):
        b.set_input(i, torch.from_numpy(d).cuda())
    for shape in [(8, 2), (16, 1), (8, 1), (8, 3)]:
        b.set_config(*shape)
        assert b.config == shape
        b.launch()
        torch.cuda.synchronize()
        for i, (h, cam, _) in enumerate(frames):
            _assert_same(b.output(i), refs[i], h.params.max_stixels_per_col)
    for h, _, _ in frames:
        assert h.get_error() == 0
    b.close()


def test_batch_with_a_maximum_height_frame():
    """A 2048-row frame (the most shared memory a column takes) batched with
    small frames: every launch shape still equals the per-frame path."""
    cams = [scenes.Camera(20, 2048, stixel_width=5, dmax=128, horizon_row=680, camera_height_m=1.2),
            scenes.CONFIG1,
            scenes.Camera(640, 240, stixel_width=7, dmax=64, horizon_row=80)]
    frames = []
    for i, cam in enumerate(cams):
        h = S.Stixels(S.default_params(cam))
        frames.append((h, cam, scenes.make_scene(cam, 4600 + i, n_obstacles=(1, 4), span_cols=(1, 4)).disparity))
    refs = [_reference(h, d) for h, _, d in frames]
    b = S.Batch([(h, cam.height, cam.width) for h, cam, _ in frames])
    for i, (_, _, d) in enumerate(frames):
        b.set_input(i, d)
    for shape in [(8, 2), (16, 1), (8, 1), (8, 3)]:
        b.set_config(*shape)
        b.launch()
        torch.cuda.synchronize()
        for i, (h, cam, _) in enumerate(frames):
            _assert_same(b.output(i), refs[i], h.params.max_stixels_per_col)
    for h, _, _ in frames:
        assert h.get_error() == 0
    b.close()


def test_batch_relaunch_with_new_inputs_and_host_sources():
    frames = _mixed_frames()[:3]
    b = S.Batch([(h, cam.height, cam.width) for h, cam, _ in frames])
    for rnd in range(2):
        disps = [scenes.make_scene(cam, 4500 + 10 * rnd + i).disparity for i, (_, cam, _) in enumerate(frames)]
        for i, d in enumerate(disps):
            b.set_input(i, d)                      # host numpy source
        b.launch()
        torch.cuda.synchronize()
        for i, (h, cam, _) in enumerate(frames):
            _assert_same(b.output(i), _reference(h, disps[i]), h.params.max_stixels_per_col)
    b.close()


def test_autotuner_picks_a_shape_and_caches_it(tmp_path):
    frames = _mixed_frames()[:4]
    b = S.Batch([(h, cam.height, cam.width) for h, cam, _ in frames])
    for i, (_, _, d) in enumerate(frames):
        b.set_input(i, d)
    cache = str(tmp_path / "tune.tsv")
    chosen = b.tune(cache)
    assert chosen in [(8, 2), (16, 1), (8, 1), (8, 3)]
    assert os.path.exists(cache) and open(cache).read().count("\n") == 1
    b2 = S.Batch([(h, cam.height, cam.width) for h, cam, _ in frames])
    assert b2.tune(cache) == chosen                # served from the cache, no new line
    assert open(cache).read().count("\n") == 1
    b.close()
    b2.close()


def test_batch_rejects_bad_frames():
    h = S.Stixels(S.default_params())
    with pytest.raises(S.StixelsError):
        S.Batch([(h, 0, 100)])
    with pytest.raises(S.StixelsError):
        S.Batch([(h, S.MAX_HEIGHT + 1, 100)])
    h.close()
