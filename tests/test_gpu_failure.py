"""Failure detection on the GPU without a fault: the bounded wait every DP
kernel uses between its warps gives up on a flag that nothing sets, reports
STIXELS_ERR_TIMEOUT through the error word, and leaves the context usable."""
import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import assert_frame_equal, cuda  # noqa: E402


def test_bounded_wait_gives_up_with_a_status_and_the_context_stays_usable():
    cam = scenes.CONFIG1
    h = S.Stixels(S.default_params(cam))
    assert h.selftest_wait(1000) == S.ERR_TIMEOUT
    assert h.get_error() == 0                      # read once, then cleared
    assert h.selftest_wait(1) == S.ERR_TIMEOUT
    sc = scenes.make_scene(cam, 8000, n_obstacles=(3, 6))
    out = S.Stixels.to_host(h.compute(cuda(sc.disparity)))
    torch.cuda.synchronize()
    assert h.get_error() == 0
    op = oracle.make_params(cam)
    fr = oracle.frame(op, sc.disparity, cap=h.params.max_stixels_per_col)
    assert_frame_equal(out, fr, cam.height, h.params.max_stixels_per_col, op)
    h.close()


@pytest.mark.parametrize("polls", [0, -5, (1 << 22) + 1])
def test_selftest_rejects_bad_poll_counts(polls):
    h = S.Stixels(S.default_params(scenes.CONFIG1))
    with pytest.raises(S.StixelsError):
        h.selftest_wait(polls)
    h.close()
