"""Checkpoint and resume (trk_session_export / trk_session_import): a second session created from the
same model resumes from the exported state and tracks the following frames bit for bit as the exporting
session does (the kernels are deterministic, and Theta, Phi, the LM damping and the frame count are all a
frame hands to the next); damaged or foreign blobs are refused and leave the state as it was."""
import struct

import numpy as np
import pytest

from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402

HEADER = 24  # "TRKSTATE", version, n_links, n_verts, frames_done


def _frames(m, s, n, seed):
    rng = np.random.default_rng(seed)
    return [synth.add_noise(s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 1, rng)
            for f in range(n)]


@pytest.mark.parametrize("mode", [trk.MODE_TRACK, trk.MODE_SHAPE_MATCH])
def test_resumed_session_tracks_like_the_uninterrupted_one(mode):
    m = synth.make_model(1, mode=mode)
    with trk.Session(m) as a, trk.Session(m) as b:
        frames = _frames(m, a, 5, seed=11)
        a.set_pose(synth.start_theta(m))
        for f in range(2):
            a.track_frame(frames[f])
        blob = a.export_state()
        assert len(blob) == HEADER + 8 * (a.L + 1) + 16 * a.V
        ref = [a.track_frame(frames[f]) for f in range(2, 5)]
        b.import_state(blob)
        got = [b.track_frame(frames[f]) for f in range(2, 5)]
    for r, g in zip(ref, got):
        assert np.array_equal(r["theta"], g["theta"])
        assert np.array_equal(r["offsets"], g["offsets"])
        assert np.array_equal(r["energy"], g["energy"], equal_nan=True)
        assert r["n_assoc_px"] == g["n_assoc_px"]


def test_import_refuses_foreign_or_damaged_blobs():
    m = synth.make_model(1)
    with trk.Session(m) as a, trk.Session(synth.make_model(1, V=500, width=48)) as small:
        frames = _frames(m, a, 1, seed=12)
        a.set_pose(synth.start_theta(m))
        a.track_frame(frames[0])
        blob = a.export_state()
        nan_theta = bytearray(blob)
        struct.pack_into("<d", nan_theta, HEADER, float("nan"))
        bad_magic = bytearray(blob)
        bad_magic[:8] = b"NOTSTATE"
        cases = [(small, blob, trk.TRK_ERR_INVALID_ARG), (a, blob[:-16], trk.TRK_ERR_INVALID_ARG),
                 (a, bytes(bad_magic), trk.TRK_ERR_INVALID_ARG), (a, bytes(nan_theta), trk.TRK_ERR_NUMERIC)]
        for sess, b, status in cases:
            with pytest.raises(trk.TrkError) as e:
                sess.import_state(b)
            assert e.value.status == status
        assert a.export_state() == blob
