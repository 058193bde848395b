"""Parity of the CUDA library with the CPU oracle, element by element, on seeded
synthetic inputs (all through the C ABI).  The library's DP decides in exact
fixed point, so the bar against the oracle's fixed-grid mode is bit-exact:
identical Q4 codes, identical prefix LUTs, identical stixel boundaries /
classes / counts, identical fixed-point column minima, and disparities equal
to the float of the exact mean.  The reported column cost is the segmentation's
cost in real arithmetic: it must equal the oracle's real-arithmetic evaluation
of the same segmentation within 1e-6 relative (FP32 per-pixel terms, a few
1e-8 relative each; their sum exact in fixed point at 2^-24, which rounds each
pixel by at most 3e-8; the total rounded to FP32 once)."""
import math

import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def both_params(cam, **kw):
    return S.default_params(cam, **kw), oracle.make_params(cam, **kw)


REAL_COST_RTOL = 1e-6


def real_params(op):
    """The same oracle parameters in plain real arithmetic (no cost grid)."""
    pu = type(op).from_buffer_copy(op)
    pu.quantize = 0
    return pu


def real_costs(op, fr):
    """Costs of the oracle's own segmentations of frame fr in real arithmetic
    (NaN where a column's list exceeds the capacity and is incomplete)."""
    return oracle.eval_frame(real_params(op), fr.q, fr.stixels, fr.counts)


def assert_real_costs(cost, expected):
    ok = ~np.isnan(expected)
    e = expected[ok]
    g = cost[ok].astype(np.float64)
    fin = np.isfinite(e)
    assert np.array_equal(np.isfinite(g), fin)
    rel = np.abs(g[fin] - e[fin]) / np.abs(e[fin])
    assert rel.size == 0 or rel.max() <= REAL_COST_RTOL, (rel.max(), int(np.argmax(rel)))


def assert_frame_equal(out, fr, H, cap, op):
    st, counts, cost, cost_fixed = out
    assert np.array_equal(counts, fr.counts), np.nonzero(counts != fr.counts)[0][:10]
    assert np.array_equal(cost_fixed, (fr.cost * S.UNITS_PER_COST).astype(np.int64))
    assert_real_costs(cost, real_costs(op, fr))
    for c in range(len(counts)):
        n = min(int(counts[c]), cap)
        g = st[c, :n]
        o = fr.stixels[c, :n]
        assert np.array_equal(g["row_top"], H - 1 - o["v_top"]), c
        assert np.array_equal(g["row_bottom"], H - 1 - o["v_bottom"]), c
        assert np.array_equal(g["cls"], o["cls"]), c
        n_px = (o["v_top"] - o["v_bottom"] + 1).astype(np.float32)
        exact = o["sum_q"].astype(np.float32) / (np.float32(16) * n_px)
        assert np.array_equal(g["disparity"], exact), c
        assert np.all(np.abs(g["disparity"] - o["disparity"]) <= 1e-3)


def run_frame(lp, disp):
    h = S.Stixels(lp)
    out = h.compute(cuda(disp))
    torch.cuda.synchronize()
    res = S.Stixels.to_host(out)
    err = h.get_error()
    h.close()
    return res, err


def nasty_image(rng, H, W, dmax):
    D = rng.uniform(-2, dmax + 3, size=(H, W)).astype(np.float32)
    D[rng.random((H, W)) < 0.05] = np.nan
    D[rng.random((H, W)) < 0.05] = 0.0
    m = rng.random((H, W)) < 0.1
    D[m] = (rng.integers(0, 32 * dmax, size=int(m.sum())) / 32.0).astype(np.float32)
    D[rng.random((H, W)) < 0.02] = np.inf
    return D


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 7, 8, 11, 16])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("grid", [0, 1])
def test_reduce_parity(s, mode, grid):
    rng = np.random.default_rng(10 * s + mode + 100 * grid)
    for H, W in [(1, 7 * s + 3), (33, 40 * s + s - 1), (120, 70 * s)]:
        D = nasty_image(rng, H, W, 64)
        lp = S.default_params(stixel_width=s, dmax=64, reduce_mode=mode, pixel_grid=grid)
        h = S.Stixels(lp)
        q = h.reduce(cuda(D))
        torch.cuda.synchronize()
        ref = oracle.reduce(D, s, 64, mode, grid)
        assert np.array_equal(q.cpu().numpy()[:W // s, :H], ref)
        h.close()


@pytest.mark.parametrize("cam", [scenes.CONFIG1, scenes.Camera(160, 37, stixel_width=4, dmax=40, horizon_row=11)])
@pytest.mark.parametrize("grid", [0, 1])
@pytest.mark.parametrize("gain", [0.0, 1.3, -0.4])
def test_lut_parity(cam, grid, gain):
    sc = scenes.make_scene(cam, 77)
    lp, op = both_params(cam, sigma_ground=0.8, sigma_sky=1.4, p_out=0.1, pixel_grid=grid, sigma_gain=gain,
                         sigma_mid=20.0, sigma_width=5.0)
    h = S.Stixels(lp)
    H, W = sc.disparity.shape
    q = h.reduce(cuda(sc.disparity))
    ncols = W // cam.stixel_width
    pd, pg, ps, po = h.build_luts(q, H, ncols)
    torch.cuda.synchronize()
    pd, pg, ps, po = (t.cpu().numpy() for t in (pd, pg, ps, po))
    qh = q.cpu().numpy()
    U = S.UNITS_PER_COST
    P = S.lut_pitch(H)
    for c in range(ncols):
        rpd, rpg, rps, rpo = oracle.prefix(op, qh[c])
        assert np.array_equal(pd[c, :H + 1], rpd)
        assert np.array_equal(pg[c, :H + 1], rpg * U)
        assert np.array_equal(ps[c, :H + 1], rps * U)
        assert np.array_equal(po[c, :, :H + 1], rpo * U)
        # padding repeats the total
        assert np.all(pd[c, H + 1:P] == pd[c, H]) and np.all(po[c, :, H + 1:P] == po[c, :, H:H + 1])
    h.close()


@pytest.mark.parametrize("seed", [1000, 1001, 1002, 1003])
def test_pipeline_config1(seed):
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, seed, n_obstacles=(3, 6))
    lp, op = both_params(cam)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == 0
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


def test_pipeline_config2():
    cam = scenes.CONFIG2
    sc = scenes.config_frames(2)[0]
    lp, op = both_params(cam)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == 0
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("i", range(len(scenes.CONFIG3)))
def test_pipeline_config3_sweep(i):
    cam = scenes.CONFIG3[i]
    sc = scenes.make_scene(cam, 3000 + i, n_obstacles=(8, 20))
    lp, op = both_params(cam)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == 0
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("H", [1, 2, 3, 31, 32, 33, 63, 64, 65, 97])
def test_pipeline_ragged_heights(H):
    cam = scenes.Camera(83, H, stixel_width=5, dmax=48, horizon_row=max(0, H // 3), baseline_m=0.4,
                        camera_height_m=1.0)
    sc = scenes.make_scene(cam, 500 + H, n_obstacles=(1, 4), span_cols=(1, 6))
    lp, op = both_params(cam)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert_frame_equal(out, fr, H, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("s", [3, 5, 7])
@pytest.mark.parametrize("mode", [0, 1])
def test_compute_equals_the_staged_pipeline(s, mode):
    """On hostile pixels (NaN, inf, negatives, beyond dmax, on and off the
    1/16 grid) stixels_compute must equal the staged reduce -> LUT -> solve
    entry points, and both the oracle."""
    rng = np.random.default_rng(40 + 10 * s + mode)
    H, ncols, dmax = 97, 61, 64
    D = nasty_image(rng, H, ncols * s, dmax)
    cam = scenes.Camera(ncols * s, H, stixel_width=s, dmax=dmax, horizon_row=30, baseline_m=0.4, camera_height_m=1.0)
    h = S.Stixels(S.default_params(cam, reduce_mode=mode))
    d = cuda(D)
    fused = S.Stixels.to_host(h.compute(d))
    q = h.reduce(d)
    staged = S.Stixels.to_host(h.solve(*h.build_luts(q, H, ncols), H, ncols))
    torch.cuda.synchronize()
    for a, b in zip(fused, staged):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    op = oracle.make_params(cam, reduce_mode=mode)
    fr = oracle.frame(op, D, cap=h.params.max_stixels_per_col)
    assert_frame_equal(fused, fr, H, h.params.max_stixels_per_col, op)
    h.close()


@pytest.mark.parametrize("ncols,H", [(153, 1), (153, 97), (200, 33), (257, 440), (304, 450), (304, 500)])
def test_pipeline_column_counts_between_one_and_two_per_sm(ncols, H):
    """Frames with more columns than SMs (up to twice as many on a 152-SM
    part) run two 8-warp CTAs per SM instead of one 16-warp CTA per column;
    every column must still equal the oracle, at ragged heights and at the
    tallest height that launch shape takes."""
    cam = scenes.Camera(ncols * 5, H, stixel_width=5, dmax=64, horizon_row=H // 3, baseline_m=0.4,
                        camera_height_m=1.2)
    sc = scenes.make_scene(cam, 900 + ncols + H, n_obstacles=(3, 12), span_cols=(1, 12))
    lp, op = both_params(cam, cost_order=2.0)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == (S.ERR_CAPACITY if (fr.counts > lp.max_stixels_per_col).any() else 0)
    assert_frame_equal(out, fr, H, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("H,dmax", [(2048, 128), (1800, 255)])
def test_pipeline_maximum_height(H, dmax):
    """The tallest column the library takes (64 row blocks), and the largest
    dmax at a height its cost budget admits, against the oracle."""
    cam = scenes.Camera(4 * 5, H, stixel_width=5, dmax=dmax, horizon_row=H // 3, baseline_m=0.3,
                        camera_height_m=1.2)
    sc = scenes.make_scene(cam, 950 + dmax, n_obstacles=(1, 3), span_cols=(1, 3))
    lp, op = both_params(cam)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert err == (S.ERR_CAPACITY if (fr.counts > lp.max_stixels_per_col).any() else 0)
    assert_frame_equal(out, fr, H, lp.max_stixels_per_col, op)


@pytest.mark.parametrize("variant", [
    dict(reduce_mode=1),
    dict(cost_order=0.0),
    dict(eps_order=-0.7, cost_order=3.5, eps_gravity=0.3, eps_diving=2.6, cost_gravity=0.7),
    dict(sigma_object=1.6, sigma_ground=0.7, sigma_sky=2.0, p_out=0.2, cost_new_stixel=1.0),
    dict(prior_trans=((1.5, 1.0, 4.0), (1.5, 6.0, 9.0), (0.5, 0.5, 7.0)), prior_first=(0.3, 0.3, 0.3)),
    dict(pitch_rad=0.035, horizon_row=52, baseline_m=0.5, camera_height_m=1.5),
    dict(pixel_grid=1),
    dict(pixel_grid=1, reduce_mode=1, sigma_object=1.5),
    dict(sigma_gain=1.5, sigma_mid=25.0, sigma_width=6.0),
    dict(sigma_gain=-0.5, sigma_mid=10.0, sigma_width=3.0, pixel_grid=1),
])
def test_pipeline_model_variants(variant):
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 1234, n_obstacles=(3, 6))
    lp, op = both_params(cam, **variant)
    out, _ = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)


def test_capacity_overflow_is_flagged():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 1000)
    lp, op = both_params(cam, max_stixels_per_col=2, cost_new_stixel=0.2)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=2)
    assert (fr.counts > 2).any()
    assert err & S.ERR_CAPACITY
    assert_frame_equal(out, fr, cam.height, 2, op)


def test_infeasible_columns_are_flagged():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 1000)
    inf = float("inf")
    lp = S.default_params(cam, prior_first=(inf, inf, inf))
    out, err = run_frame(lp, sc.disparity)
    assert err & S.ERR_INFEASIBLE
    assert np.all(out[1] == 0)


def test_empty_inputs_are_noops():
    lp = S.default_params()
    h = S.Stixels(lp)
    for H, W in [(0, 100), (10, 0), (10, 4)]:           # W < stixel width -> no columns
        d = torch.zeros((max(H, 1), max(W, 1)), dtype=torch.float32, device="cuda")[:H, :W]
        out = h.alloc_output(H, W)
        h.compute(d.contiguous() if H and W else torch.zeros((H, W), device="cuda"), out=out)
    torch.cuda.synchronize()
    assert h.get_error() == 0
    h.close()


def test_invalid_arguments_rejected():
    lp = S.default_params()
    h = S.Stixels(lp)
    d = torch.zeros((20, 50), dtype=torch.float32, device="cuda")
    out = h.alloc_output(20, 50)
    out_bad = dict(out, ncols=out["ncols"] + 1)
    with pytest.raises(S.StixelsError) as e:
        h.compute(d, out=out_bad)
    assert e.value.status == S.E_INVALID_ARG
    big = torch.zeros((S.MAX_HEIGHT + 1, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(S.StixelsError):
        h.compute(big)
    h.close()


def test_compute_host_equals_device_path_and_is_deterministic():
    cam = scenes.CONFIG2
    sc = scenes.config_frames(2)[0]
    lp, _ = both_params(cam)
    h = S.Stixels(lp)
    st_h, counts_h, cost_h, rc = h.compute_host(sc.disparity)
    assert rc == S.OK
    for _ in range(3):
        out = S.Stixels.to_host(h.compute(cuda(sc.disparity)))
        torch.cuda.synchronize()
        assert np.array_equal(out[1], counts_h)
        assert np.array_equal(out[2], cost_h)
        for c in range(len(counts_h)):
            n = min(counts_h[c], lp.max_stixels_per_col)
            assert np.array_equal(out[0][c, :n], st_h[c, :n])
    h.close()


def test_compute_host_pinned_buffers_in_place():
    """Page-locked host buffers are read and written in place by the kernels
    (no staging copies): every mix of pinned and pageable input and outputs,
    including a pinned frame that starts inside its allocation, gives the
    device path's results."""
    cam = scenes.CONFIG2
    sc = scenes.make_scene(cam, 7500, n_obstacles=(8, 20))
    lp, _ = both_params(cam)
    h = S.Stixels(lp)
    ref = S.Stixels.to_host(h.compute(cuda(sc.disparity)))
    torch.cuda.synchronize()
    H, W = sc.disparity.shape
    # a frame one float into a pinned allocation: the device reads it at that offset
    pinned_in = torch.empty(H * W + 1, dtype=torch.float32, pin_memory=True).numpy()[1:].reshape(H, W)
    pinned_in[:] = sc.disparity
    for in_pinned in (False, True):
        for out_pinned in (False, True):
            src = pinned_in if in_pinned else sc.disparity.copy()
            st, counts, cost, rc = h.compute_host(src, h.alloc_host_output(H, W, pinned=out_pinned))
            assert rc == S.OK
            assert np.array_equal(counts, ref[1]) and np.array_equal(cost, ref[2])
            for c in range(len(counts)):
                n = min(counts[c], lp.max_stixels_per_col)
                assert np.array_equal(st[c, :n], ref[0][c, :n])
    h.close()


def test_compute_host_reports_its_own_frame_status():
    """compute_host returns CAPACITY when its frame overflows a column's
    capacity (pinned and pageable buffers), and leaves the handle's error word,
    which stixels_get_error reads, as it was."""
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 7600, n_obstacles=(3, 6))
    h = S.Stixels(S.default_params(cam, max_stixels_per_col=1))
    H, W = sc.disparity.shape
    pinned_in = torch.from_numpy(sc.disparity).pin_memory().numpy()
    for src, pinned in ((sc.disparity, False), (pinned_in, True)):
        _, counts, _, rc = h.compute_host(src, h.alloc_host_output(H, W, pinned=pinned))
        assert rc == S.E_CAPACITY and counts.max() > 1
        assert h.get_error() == 0
    h.close()


@pytest.mark.parametrize("i", [1, 4])
def test_pixel_grid_pipeline_paper_sizes(i):
    """The LUT_cost variant (whole-pixel grid, Sec. 3.4) at 1024x440 s=5 and the
    2048x880 frame, against the oracle element by element."""
    cam = scenes.CONFIG3[i]
    sc = scenes.make_scene(cam, 3100 + i, n_obstacles=(8, 20))
    lp, op = both_params(cam, pixel_grid=1, reduce_mode=1)
    out, err = run_frame(lp, sc.disparity)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    # the mean keeps outliers, so a few columns may need more than the capacity:
    # the flag is raised exactly then, and the stored prefix still matches
    assert err == (S.ERR_CAPACITY if (fr.counts > lp.max_stixels_per_col).any() else 0)
    assert_frame_equal(out, fr, cam.height, lp.max_stixels_per_col, op)
