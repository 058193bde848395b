"""Serving: frames from several cameras admitted one by one and run with
continuous batching.  A served frame's result must equal the per-frame path's
exactly (and the oracle's, for one frame checked directly), whatever else was
in its iteration; admission must refuse what does not fit the slots or the
memory budget; poll must report frames that are not done yet."""
import threading

import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import assert_real_costs, real_costs  # noqa: E402


def _cameras():
    cams = scenes.serving_cameras()
    hs = [S.Stixels(S.default_params(c)) for c in cams]
    return cams, hs


def _per_frame(h, disp):
    out = h.compute(torch.from_numpy(disp).cuda())
    torch.cuda.synchronize()
    st, cnt, cost, fix = S.Stixels.to_host(out)
    return st, cnt, cost


def _same(got, ref):
    st, cnt, cost = got
    r_st, r_cnt, r_cost = ref
    n, cap = r_st.shape
    st = st[:n * cap].reshape(n, cap)
    assert np.array_equal(cnt[:n], r_cnt)
    assert np.array_equal(cost[:n], r_cost)
    for c in range(n):
        k = min(int(r_cnt[c]), cap)
        assert np.array_equal(st[c, :k], r_st[c, :k]), c


def _poll_done(srv, t, out, limit_s=20.0):
    rc = srv.poll(t, out, timeout_us=int(limit_s * 1e6))
    assert rc == S.OK, rc
    return out


def test_served_frames_equal_per_frame_results():
    cams, hs = _cameras()
    frames = [scenes.make_scene(cams[i % 8], 7000 + i, n_obstacles=(3, 12)).disparity for i in range(24)]
    refs = [_per_frame(hs[i % 8], d) for i, d in enumerate(frames)]
    srv = S.Server(4 << 30, max_slots=64)
    tickets = []
    for i, d in enumerate(frames):
        # alternate host and device inputs
        src = d if i % 2 == 0 else torch.from_numpy(d).cuda()
        t = srv.submit(hs[i % 8], src)
        assert t is not None
        tickets.append(t)
    for i, t in enumerate(tickets):
        cam = cams[i % 8]
        out = _poll_done(srv, t, hs[i % 8].alloc_host_output(cam.height, cam.width))
        _same(out, refs[i])
    st = srv.stats()
    assert st["submitted"] == st["admitted"] == st["completed"] == 24 and st["rejected"] == 0
    assert st["frames_in_iterations"] == 24 and 1 <= st["iterations"] <= 24
    assert st["slots_in_use"] == 0 and st["bytes_in_use"] == 0
    srv.close()


def test_served_frame_matches_oracle():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 7100)
    lp = S.default_params(cam)
    h = S.Stixels(lp)
    srv = S.Server(64 << 20, max_slots=4)
    t = srv.submit(h, sc.disparity)
    out = _poll_done(srv, t, h.alloc_host_output(cam.height, cam.width))
    op = oracle.make_params(cam)
    fr = oracle.frame(op, sc.disparity, cap=lp.max_stixels_per_col)
    st, cnt, cost = out
    n, cap = cam.ncols, lp.max_stixels_per_col
    assert np.array_equal(cnt[:n], fr.counts)
    assert_real_costs(cost[:n], real_costs(op, fr))
    st = st[:n * cap].reshape(n, cap)
    for c in range(n):
        k = min(int(cnt[c]), cap)
        assert np.array_equal(st[c, :k]["row_top"], cam.height - 1 - fr.stixels[c, :k]["v_top"])
        assert np.array_equal(st[c, :k]["row_bottom"], cam.height - 1 - fr.stixels[c, :k]["v_bottom"])
        assert np.array_equal(st[c, :k]["cls"], fr.stixels[c, :k]["cls"])
    srv.close()


def test_device_output_buffers_and_capacity_status():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 1000)
    lp = S.default_params(cam, max_stixels_per_col=2, cost_new_stixel=0.2)
    h = S.Stixels(lp)
    ref_out = h.compute(torch.from_numpy(sc.disparity).cuda())
    torch.cuda.synchronize()
    ref = S.Stixels.to_host(ref_out)
    assert h.get_error() & S.ERR_CAPACITY
    srv = S.Server(64 << 20, max_slots=4)
    t = srv.submit(h, sc.disparity)
    out = h.alloc_output(cam.height, cam.width)
    rc = srv.poll(t, out, timeout_us=20_000_000)
    assert rc == S.E_CAPACITY
    got = S.Stixels.to_host(out)
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[3], ref[3])
    for c in range(cam.ncols):
        assert np.array_equal(got[0][c, :2], ref[0][c, :2])
    srv.close()


def test_admission_by_slots_and_budget():
    cams, hs = _cameras()
    big = scenes.make_scene(cams[6], 7200).disparity                      # 2048 x 880
    # a 4 MiB arena cannot hold a 2048 x 880 frame (7.2 MB input alone)
    srv = S.Server(4 << 20, max_slots=8)
    assert srv.submit(hs[6], big) is None
    st = srv.stats()
    assert st["rejected"] == 1 and st["admitted"] == 0 and st["bytes_budget"] == 4 << 20
    srv.close()
    # two slots: the third frame waits for a poll
    small = [scenes.make_scene(cams[0], 7300 + i).disparity for i in range(3)]
    srv = S.Server(256 << 20, max_slots=2)
    t0 = srv.submit(hs[0], small[0])
    t1 = srv.submit(hs[0], small[1])
    assert t0 is not None and t1 is not None
    assert srv.submit(hs[0], small[2]) is None
    _poll_done(srv, t0, hs[0].alloc_host_output(cams[0].height, cams[0].width))
    t2 = srv.submit(hs[0], small[2])
    assert t2 is not None
    for t in (t1, t2):
        _poll_done(srv, t, hs[0].alloc_host_output(cams[0].height, cams[0].width))
    st = srv.stats()
    assert st["admitted"] == 3 and st["rejected"] == 1 and st["completed"] == 3 and st["bytes_in_use"] == 0
    srv.close()


def test_poll_statuses():
    cams, hs = _cameras()
    srv = S.Server(2 << 30, max_slots=32)
    frames = [scenes.make_scene(cams[6 + i % 2], 7400 + i).disparity for i in range(8)]
    tickets = [srv.submit(hs[6 + i % 2], d) for i, d in enumerate(frames)]
    assert all(t is not None for t in tickets)
    out = hs[7].alloc_host_output(cams[7].height, cams[7].width)
    # the last of eight 2048 x 880 frames cannot be finished microseconds after submission
    # on any current GPU, but only the set of legal answers is asserted
    rc = srv.poll(tickets[-1], out, timeout_us=0)
    assert rc in (S.E_NOT_READY, S.OK)
    if rc == S.E_NOT_READY:
        rc = srv.poll(tickets[-1], out, timeout_us=1)
        assert rc in (S.E_TIMEOUT, S.OK)
    for i, t in enumerate(tickets):
        if i == len(tickets) - 1 and rc == S.OK:
            continue
        o = hs[6 + i % 2].alloc_host_output(cams[6 + i % 2].height, cams[6 + i % 2].width)
        # a busy-wait poll loop with timeout 0 ends in OK
        for _ in range(2_000_000):
            r = srv.poll(t, o, timeout_us=0)
            if r != S.E_NOT_READY:
                break
        assert r == S.OK
    # retired and unknown tickets are invalid
    with pytest.raises(S.StixelsError):
        srv.poll(tickets[0], out, timeout_us=0)
    with pytest.raises(S.StixelsError):
        srv.poll(123456789, out, timeout_us=0)
    srv.close()


def test_one_ticket_polled_from_many_threads_is_delivered_once():
    """Threads racing to poll the same ticket: exactly one gets the frame (its
    slot is freed once), the others are refused; the arena balances."""
    import threading
    cams, hs = _cameras()
    srv = S.Server(2 << 30, max_slots=8)
    cam, h = cams[2], hs[2]
    frame = scenes.make_scene(cam, 7600).disparity
    for rep in range(5):
        t = srv.submit(h, frame)
        assert t is not None
        outs = [h.alloc_host_output(cam.height, cam.width) for _ in range(4)]
        results = [None] * 4

        def worker(i):
            try:
                results[i] = srv.poll(t, outs[i], timeout_us=2_000_000)
            except S.StixelsError:
                results[i] = "refused"

        th = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert results.count(S.OK) == 1 and results.count("refused") == 3, results
    st = srv.stats()
    assert st["slots_in_use"] == 0 and st["bytes_in_use"] == 0
    srv.close()


def test_concurrent_submitters():
    cams, hs = _cameras()
    frames = [scenes.make_scene(cams[i % 6], 7500 + i, n_obstacles=(3, 12)).disparity for i in range(36)]
    refs = [_per_frame(hs[i % 6], d) for i, d in enumerate(frames)]
    srv = S.Server(4 << 30, max_slots=128)
    results = {}
    errors = []

    def worker(k):
        try:
            for i in range(k, len(frames), 3):
                cam = cams[i % 6]
                t = srv.submit(hs[i % 6], frames[i])
                assert t is not None
                results[i] = _poll_done(srv, t, hs[i % 6].alloc_host_output(cam.height, cam.width))
        except Exception as e:            # surfaced below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(3)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for i in range(len(frames)):
        _same(results[i], refs[i])
    srv.close()
