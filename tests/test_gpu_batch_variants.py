"""The ground line estimated per frame (v-disparity) and the global MAP in the
batched and served modes: mixed with plain frames in one graph launch / one
server, each frame must equal the oracle and the per-frame path exactly."""
import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import assert_frame_equal, cuda  # noqa: E402

WRONG = dict(horizon_row=10, baseline_m=0.2)       # camera parameters the estimate overrides
SMALL = scenes.Camera(333, 97, stixel_width=4, dmax=48, horizon_row=30, baseline_m=0.4, camera_height_m=1.0)


def _frames():
    """(camera, library / oracle parameter overrides, disparity) of a mixed set."""
    specs = [
        (scenes.CONFIG1, dict(ground_estimate=1, **WRONG), 8100),
        (scenes.CONFIG1, dict(global_map=1, cost_order=2.5), 8101),
        (scenes.CONFIG1, dict(ground_estimate=1, global_map=1, cost_order=2.5, **WRONG), 8102),
        (scenes.CONFIG1, {}, 8103),
        (SMALL, dict(ground_estimate=1, **WRONG), 8104),
        (SMALL, dict(global_map=1, cost_order=3.0, eps_order=-0.5), 8105),
        (scenes.Camera(640, 240, stixel_width=5, dmax=64, horizon_row=80), {}, 8106),
    ]
    out = []
    for cam, kw, seed in specs:
        sc = scenes.make_scene(cam, seed, n_obstacles=(3, 8))
        out.append((cam, kw, sc.disparity))
    return out


def _lib_params(cam, kw):
    return S.default_params(cam, **kw)


def _oracle_params(cam, kw):
    return oracle.make_params(cam, **kw)


def _per_frame(h, disp):
    out = h.compute(cuda(disp))
    torch.cuda.synchronize()
    return S.Stixels.to_host(out)


def _same(got, ref, cap):
    st, cnt, cost, fix = got
    r_st, r_cnt, r_cost, r_fix = ref
    assert np.array_equal(cnt, r_cnt)
    assert np.array_equal(fix, r_fix) and np.array_equal(cost, r_cost)
    for c in range(len(cnt)):
        n = min(int(cnt[c]), cap)
        assert np.array_equal(st[c, :n], r_st[c, :n])


def test_batched_estimate_and_global_map_equal_oracle_and_per_frame():
    frames = _frames()
    hs = [S.Stixels(_lib_params(cam, kw)) for cam, kw, _ in frames]
    refs = [_per_frame(h, d) for h, (_, _, d) in zip(hs, frames)]
    b = S.Batch([(h, cam.height, cam.width) for h, (cam, _, _) in zip(hs, frames)])
    for i, (_, _, d) in enumerate(frames):
        b.set_input(i, cuda(d))
    for _ in range(2):                      # the second launch reruns the same graph
        b.launch()
        torch.cuda.synchronize()
        for i, (h, (cam, kw, d)) in enumerate(zip(hs, frames)):
            got = b.output(i)
            cap = h.params.max_stixels_per_col
            _same(got, refs[i], cap)
            fr = oracle.frame(_oracle_params(cam, kw), d, cap=cap)
            assert_frame_equal(got, fr, cam.height, cap, _oracle_params(cam, kw))
    b.close()
    for h in hs:
        h.close()


def test_served_estimate_and_global_map_equal_per_frame():
    frames = _frames()
    hs = [S.Stixels(_lib_params(cam, kw)) for cam, kw, _ in frames]
    refs = [_per_frame(h, d) for h, (_, _, d) in zip(hs, frames)]
    srv = S.Server(1 << 30, max_slots=16)
    tickets = [srv.submit(h, d) for h, (_, _, d) in zip(hs, frames)]
    for i, (t, h, (cam, kw, d)) in enumerate(zip(tickets, hs, frames)):
        out = h.alloc_host_output(cam.height, cam.width)
        assert srv.poll(t, out, timeout_us=20_000_000) == S.OK
        st, cnt, cost = out
        n, cap = cam.width // cam.stixel_width, h.params.max_stixels_per_col
        r_st, r_cnt, r_cost, _ = refs[i]
        assert np.array_equal(cnt, r_cnt) and np.array_equal(cost, r_cost)
        st = st[:n * cap].reshape(n, cap)
        for c in range(n):
            k = min(int(cnt[c]), cap)
            assert np.array_equal(st[c, :k], r_st[c, :k])
    srv.close()
    for h in hs:
        h.close()


def test_batched_global_map_mixed_heights_equal_per_frame():
    """Global-MAP frames of different heights and dmax in one launch of the
    batch kernel (its shared memory sized for the tallest, each CTA laid out
    for its own frame), beside plain frames, twice through the same graph:
    each frame equals its own per-frame call bit for bit (the per-frame MAP
    is checked against the oracle in test_gpu_map)."""
    specs = [
        (scenes.CONFIG2, dict(global_map=1), 8200),
        (SMALL, dict(global_map=1, cost_order=3.0), 8201),
        (scenes.Camera(640, 240, stixel_width=7, dmax=64, horizon_row=80), dict(global_map=1, eps_order=-0.5), 8202),
        (scenes.CONFIG2, {}, 8203),
        (scenes.CONFIG1, dict(global_map=1, ground_estimate=1, **WRONG), 8204),
    ]
    hs, frames = [], []
    for cam, kw, seed in specs:
        hs.append(S.Stixels(S.default_params(cam, **kw)))
        frames.append((cam, scenes.make_scene(cam, seed, n_obstacles=(5, 12)).disparity))
    refs = [_per_frame(h, d) for h, (_, d) in zip(hs, frames)]
    b = S.Batch([(h, cam.height, cam.width) for h, (cam, _) in zip(hs, frames)])
    for i, (_, d) in enumerate(frames):
        b.set_input(i, cuda(d))
    for _ in range(2):
        b.launch()
        torch.cuda.synchronize()
        for i, h in enumerate(hs):
            _same(b.output(i), refs[i], h.params.max_stixels_per_col)
    b.close()
    for h in hs:
        h.close()


def test_batched_global_map_ragged_heights_equal_oracle():
    """Global-MAP frames of 1, 2, 31, 33 and 64 rows (a block of 32 rows
    partly filled, one row, exactly two blocks) in one batched launch, against
    the oracle frame by frame."""
    specs = []
    for H in (1, 2, 31, 33, 64):
        cam = scenes.Camera(83, H, stixel_width=5, dmax=48, horizon_row=max(0, H // 3), baseline_m=0.4,
                            camera_height_m=1.0)
        kw = dict(global_map=1, cost_order=3.0, eps_order=-0.5)
        specs.append((cam, kw, scenes.make_scene(cam, 8300 + H, n_obstacles=(1, 4), span_cols=(1, 6)).disparity))
    hs = [S.Stixels(_lib_params(cam, kw)) for cam, kw, _ in specs]
    b = S.Batch([(h, cam.height, cam.width) for h, (cam, _, _) in zip(hs, specs)])
    for i, (_, _, d) in enumerate(specs):
        b.set_input(i, cuda(d))
    b.launch()
    torch.cuda.synchronize()
    for i, (h, (cam, kw, d)) in enumerate(zip(hs, specs)):
        cap = h.params.max_stixels_per_col
        fr = oracle.frame(_oracle_params(cam, kw), d, cap=cap)
        assert_frame_equal(b.output(i), fr, cam.height, cap, _oracle_params(cam, kw))
    b.close()
    for h in hs:
        h.close()
