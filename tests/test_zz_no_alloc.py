"""stixels_compute_noalloc -- the pipeline without device allocation.

Some callers cannot allocate device memory while they process frames (a
real-time loop where cudaMalloc could stall or fail, code inside another
framework's memory pool or under a fixed budget, code that must not let an
allocation synchronise the device).  This entry point keeps the frame's
intermediates in a fixed array inside the library instead.  It must return
exactly what stixels_compute returns (the library's results are deterministic),
on consecutive calls that reuse the same array, and reject frames too large for
it or heights it has no tables for.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _host(out):
    return S.Stixels.to_host(out)


def test_noalloc_matches_compute_on_consecutive_calls():
    cam = scenes.CONFIG2                         # 1024 x 440, s = 5, dmax 128: fits the array
    frames = [scenes.make_scene(cam, 7100 + i, n_obstacles=(8, 20)).disparity for i in range(2)]
    h = S.Stixels(S.default_params(cam))
    h.reserve(cam.height, cam.width)             # the one allocating step, at start-up
    L = S.lib()
    stream = torch.cuda.current_stream()
    for disp in frames:                          # two calls in a row on the shared array
        d = torch.from_numpy(disp).cuda()
        ref = h.compute(d, stream=stream)
        got = h.alloc_output(cam.height, cam.width)
        o = S.Stixels._out_struct(got)
        rc = L.stixels_compute_noalloc(h.handle, d.data_ptr(), cam.height, cam.width,
                                       stream.cuda_stream, C.byref(o))
        assert rc == S.OK, L.stixels_status_string(rc)
        torch.cuda.synchronize()
        r_st, r_cnt, r_cost, r_fix = _host(ref)
        g_st, g_cnt, g_cost, g_fix = _host(got)
        assert np.array_equal(g_cnt, r_cnt)
        assert np.array_equal(g_fix, r_fix) and np.array_equal(g_cost, r_cost)
        for c in range(len(r_cnt)):
            n = min(int(r_cnt[c]), h.params.max_stixels_per_col)
            assert np.array_equal(g_st[c, :n], r_st[c, :n])
    assert h.get_error() == 0
    h.close()


def test_noalloc_rejects_frames_larger_than_the_array():
    cam = scenes.CONFIG3[-1]                     # 2048 x 880, dmax 128: intermediates ~190 MB
    h = S.Stixels(S.default_params(cam))
    h.reserve(cam.height, cam.width)
    d = torch.zeros((cam.height, cam.width), dtype=torch.float32, device="cuda")
    out = h.alloc_output(cam.height, cam.width)
    o = S.Stixels._out_struct(out)
    rc = S.lib().stixels_compute_noalloc(h.handle, d.data_ptr(), cam.height, cam.width,
                                         torch.cuda.current_stream().cuda_stream, C.byref(o))
    assert rc == S.E_INVALID_ARG
    h.close()


def test_noalloc_refuses_a_height_the_handle_has_no_tables_for():
    """Creating the row tables of a new height would allocate: without a reserve
    (or an earlier allocating call) for that height the call is refused."""
    cam = scenes.CONFIG1
    h = S.Stixels(S.default_params(cam))
    d = torch.zeros((cam.height, cam.width), dtype=torch.float32, device="cuda")
    out = h.alloc_output(cam.height, cam.width)
    o = S.Stixels._out_struct(out)
    rc = S.lib().stixels_compute_noalloc(h.handle, d.data_ptr(), cam.height, cam.width,
                                         torch.cuda.current_stream().cuda_stream, C.byref(o))
    assert rc == S.E_INVALID_ARG
    h.close()
