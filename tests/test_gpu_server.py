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


def test_each_result_is_the_same_alone_and_in_the_mix():
    data = _models(5)
    alone = []
    for m, frames in data:
        with trk.Session(m) as s:
            s.set_pose(synth.start_theta(m))
            alone.append([s.track_frame(f) for f in frames])
    sessions = [trk.Session(m) for m, _ in data]
    for (m, _), s in zip(data, sessions):
        s.set_pose(synth.start_theta(m))
    with trk.Server(1 << 40, max_inflight=3) as sv:
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
    (m, _), = _models(1)
    a, b = trk.Session(m), trk.Session(m)
    need = a.info()["device_bytes"]
    with trk.Server(int(need * 1.5), max_inflight=4) as sv:
        sv.attach(a)
        with pytest.raises(trk.TrkError) as e:
            sv.attach(b)
        assert e.value.status == trk.TRK_ERR_NO_CAPACITY
        assert sv.stats()["hbm_used_bytes"] == need
        sv.detach(a)
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
