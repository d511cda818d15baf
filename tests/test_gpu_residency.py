"""Device residency of a session (trk_create_evicted, trk_session_evict, trk_session_restore): an evicted
session holds no device memory, and a session evicted and restored between frames tracks bit for bit as
one that stayed resident."""
import numpy as np
import pytest

from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _frames(m, n, seed=3):
    rng = np.random.default_rng(seed)
    with trk.Session(m) as r:
        return [synth.add_noise(r.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 2, rng)
                for f in range(n)]


def _used():
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    return total - free


def test_evicted_session_holds_no_device_memory_and_tracks_identically():
    m = synth.make_model(2, V=20000, width=320)
    frames = _frames(m, 4)
    th0 = synth.gt_theta(m, 0.0)
    with trk.Session(m) as ref:
        ref.set_pose(th0)
        want = [ref.track_frame(d) for d in frames]
    base = _used()
    s = trk.Session(m, evicted=True)
    try:
        assert not s.resident
        need = s.info()["device_bytes"]
        assert need > 10 << 20
        assert _used() - base < 4 << 20  # nothing of the session's state on the device
        s.set_pose(th0)  # kept on the host while evicted
        with pytest.raises(trk.TrkError) as e:
            s.track_frame(frames[0])
        assert e.value.status == trk.TRK_ERR_INVALID_ARG
        s.restore()
        assert s.resident
        grown = _used() - base
        assert need <= grown <= need + (64 << 20)
        got = [s.track_frame(frames[0]), s.track_frame(frames[1])]
        blob = s.export_state()
        s.evict()  # between frames: the state goes to the host, the device memory is returned
        assert not s.resident
        assert _used() - base < 4 << 20
        assert s.export_state() == blob  # the host copy is the state
        s.restore()
        got += [s.track_frame(frames[2]), s.track_frame(frames[3])]
    finally:
        s.close()
    for a, b in zip(want, got):
        assert np.array_equal(a["theta"], b["theta"])
        assert np.array_equal(a["offsets"], b["offsets"])
        assert np.array_equal(a["energy"], b["energy"])


def test_batch_refuses_members_evicted_after_it_was_built():
    ms = [synth.make_model(4, session=k) for k in (0, 1)]
    sessions = [trk.Session(m) for m in ms]
    try:
        for m, s in zip(ms, sessions):
            s.set_pose(synth.gt_theta(m, 0.0))
        dev = [torch.zeros((s.H, s.W), device="cuda") for s in sessions]
        b = trk.Batch(sessions)
        try:
            sessions[1].evict()
            with pytest.raises(trk.TrkError) as e:
                b.track_device([x.data_ptr() for x in dev])
            assert e.value.status == trk.TRK_ERR_INVALID_ARG
            sessions[1].restore()
            with pytest.raises(trk.TrkError):  # restored memory is new memory: the batch must be rebuilt
                b.track_device([x.data_ptr() for x in dev])
        finally:
            b.close()
        with pytest.raises(trk.TrkError):
            sessions[0].evict() or trk.Batch(sessions)
    finally:
        for s in sessions:
            s.close()
