"""The continuous-batching frame server (trk_server_*): admission by HBM budget, frames of many sessions
overlapping on the device, each session's result identical alone and in the mix, bounded waits."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _models(n):
    out = []
    for s in range(n):
        m = synth.make_model(1, session=s, V=1500 + 300 * s, width=96 + 16 * (s % 3))
        o = oracle.Oracle(m)
        frames = [synth.add_noise(o.render(synth.gt_theta(m, 0.0), synth.gt_offsets(m, 0.0)), 1,
                                  np.random.default_rng(100 * s + f)) for f in range(3)]
        out.append((m, frames))
    return out


@pytest.mark.parametrize("dispatch", [trk.SERVER_DISPATCH_BATCHED, trk.SERVER_DISPATCH_SESSION])
def test_each_result_is_the_same_alone_and_in_the_mix(dispatch):
    data = _models(5)
    alone = []
    for m, frames in data:
        with trk.Session(m) as s:
            s.set_pose(synth.start_theta(m))
            alone.append([s.track_frame(f) for f in frames])
    sessions = [trk.Session(m) for m, _ in data]
    for (m, _), s in zip(data, sessions):
        s.set_pose(synth.start_theta(m))
    with trk.Server(1 << 40, max_inflight=3, dispatch=dispatch) as sv:
        for s in sessions:
            sv.attach(s)
        tickets = []
        for f in range(3):  # frames of all sessions interleaved; each session's in order
            for i, s in enumerate(sessions):
                tickets.append((i, f, sv.submit(s, data[i][1][f])))
        got = {}
        for i, f, t in tickets:
            got[(i, f)] = sv.wait(sessions[i], t)
        st = sv.stats()
        assert st["frames_done"] == 15 and st["in_flight"] == 0
        assert 0 < st["latency_p50_us"] <= st["latency_p99_us"] <= st["latency_max_us"]
        for i in range(5):
            for f in range(3):
                a, b = alone[i][f], got[(i, f)]
                assert np.array_equal(a["theta"], b["theta"])
                assert np.array_equal(a["offsets"], b["offsets"])
                assert np.array_equal(a["energy"], b["energy"])
                assert a["n_assoc_px"] == b["n_assoc_px"]
        for s in sessions:
            sv.detach(s)
    for s in sessions:
        s.close()


def test_admission_by_hbm_budget():
    """The budget counts a session's arena and the batched steps' buffers (per step slot, twice the step
    tables of the attached sessions), both in 2 MiB units; a second session that does not fit is refused
    until the first leaves."""
    (m, _), = _models(1)
    a, b = trk.Session(m), trk.Session(m)
    need = a.info()["device_bytes"]
    assert need % (2 << 20) == 0
    with trk.Server(1 << 40, max_inflight=4) as probe:  # what one attached session counts
        probe.attach(a)
        one = probe.stats()["hbm_used_bytes"]
        probe.detach(a)
    assert one >= need
    with trk.Server(one + need // 2, max_inflight=4) as sv:
        sv.attach(a)
        with pytest.raises(trk.TrkError) as e:
            sv.attach(b)
        assert e.value.status == trk.TRK_ERR_NO_CAPACITY
        assert sv.stats()["hbm_used_bytes"] == one
        sv.detach(a)
        assert sv.stats()["hbm_used_bytes"] == one - need  # the step buffers' reservation stays
        sv.attach(b)  # the budget freed by the detach admits the other session
        assert sv.stats()["sessions"] == 1
        sv.detach(b)
    a.close()
    b.close()


def test_wait_times_out_and_unknown_tickets_are_rejected():
    (m, frames), = _models(1)
    s = trk.Session(m)
    with trk.Server(1 << 40, max_inflight=0) as sv:  # admits frames, never launches them
        sv.attach(s)
        t = sv.submit(s, frames[0])
        with pytest.raises(trk.TrkError) as e:
            sv.wait(s, t, timeout_us=2000)
        assert e.value.status == trk.TRK_ERR_TIMEOUT
        with pytest.raises(trk.TrkError) as e:
            sv.wait(s, t + 12345, timeout_us=0)
        assert e.value.status == trk.TRK_ERR_INVALID_ARG
        with pytest.raises(trk.TrkError) as e:
            sv.detach(s)  # still has a queued frame
        assert e.value.status == trk.TRK_ERR_INVALID_ARG
    s.close()  # the server freed the uncollected frame on destruction


def _used():
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    return total - free


def test_budget_bounds_device_memory_while_sessions_come_and_go():
    """More sessions than the budget holds, created evicted (no device memory): each is admitted when the
    budget allows, tracks its frames through batched steps, and leaves; the device memory in use (read
    with cudaMemGetInfo) never exceeds the budget beyond the server's own step buffers, and every
    session's results are bitwise those it computes alone."""
    data = []
    for k in range(8):
        m = synth.make_model(2, session=k, V=12000 + 3000 * k, width=320)
        with trk.Session(m) as r:
            rng = np.random.default_rng(40 + k)
            frames = [synth.add_noise(r.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 2, rng)
                      for f in range(3)]
            r.set_pose(synth.gt_theta(m, 0.0))
            alone = [r.track_frame(d) for d in frames]
        data.append((m, frames, alone))
    base = _used()
    sessions = [trk.Session(m, evicted=True) for m, _, _ in data]
    for (m, _, _), s in zip(data, sessions):
        s.set_pose(synth.gt_theta(m, 0.0))
    need = [s.info()["device_bytes"] for s in sessions]
    budget = int(2.5 * max(need))
    # the library counts what it holds (the arenas of the admitted sessions, the step buffers) at the 2 MiB
    # allocation granularity, so what it holds never exceeds the budget; the device use read by
    # cudaMemGetInfo adds the runtime's own state (kernels loaded on first launch): 16 MiB allowed
    slack = 16 << 20
    peak = peak_pool = 0
    with trk.Server(budget, max_inflight=8) as sv:
        waiting = list(range(len(sessions)))
        active = {}
        done = 0
        while waiting or active:
            while waiting:  # admit in arrival order while the budget allows
                try:
                    sv.attach(sessions[waiting[0]])
                except trk.TrkError as e:
                    assert e.status == trk.TRK_ERR_NO_CAPACITY
                    break
                k = waiting.pop(0)
                active[k] = [sv.submit(sessions[k], d) for d in data[k][1]]
            assert active, "the budget admits at least one session"
            peak = max(peak, _used() - base)
            st = sv.stats()
            peak_pool = max(peak_pool, st["device_bytes_reserved"])
            assert st["hbm_used_bytes"] <= budget
            k = min(active)
            got = [sv.wait(sessions[k], t) for t in active.pop(k)]
            for a, b in zip(data[k][2], got):
                assert np.array_equal(a["theta"], b["theta"]) and np.array_equal(a["offsets"], b["offsets"])
                assert np.array_equal(a["energy"], b["energy"])
            sv.detach(sessions[k])
            assert not sessions[k].resident
            done += 1
        st = sv.stats()
        assert done == len(sessions) and st["frames_done"] == 3 * len(sessions)
        assert st["mean_frames_per_step"] >= 1.0
    print(f"budget {budget / 2**20:.1f} MiB, sessions {[round(n / 2**20, 1) for n in need]} MiB, "
          f"peak device use {peak / 2**20:.1f} MiB (held by the library: {peak_pool / 2**20:.1f} MiB)")
    assert sum(need) > budget  # more sessions than fit at once
    assert peak_pool <= budget
    assert peak <= budget + slack
    for s in sessions:
        s.close()


def test_tensor_core_sessions_are_served_batched():
    """Sessions in the 3xTF32 precision mode go through batched steps like FP32 ones and give bitwise
    their results alone."""
    data = []
    for k in range(3):
        m = synth.make_model(1, session=k, V=2000 + 500 * k, width=96, precision=trk.PRECISION_TF32X3)
        o = oracle.Oracle(m)
        d = synth.add_noise(o.render(synth.gt_theta(m, 0.0), synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(k))
        with trk.Session(m) as r:
            r.set_pose(synth.start_theta(m))
            data.append((m, d, r.track_frame(d)))
    sessions = [trk.Session(m, evicted=True) for m, _, _ in data]
    for (m, _, _), s in zip(data, sessions):
        s.set_pose(synth.start_theta(m))
    with trk.Server(1 << 40, max_inflight=8) as sv:
        for s in sessions:
            sv.attach(s)
        tickets = [sv.submit(s, d) for s, (_, d, _) in zip(sessions, data)]
        for s, t, (_, _, a) in zip(sessions, tickets, data):
            b = sv.wait(s, t)
            assert np.array_equal(a["theta"], b["theta"]) and np.array_equal(a["offsets"], b["offsets"])
        assert sv.stats()["steps"] >= 1
        for s in sessions:
            sv.detach(s)
    for s in sessions:
        s.close()
