"""The paper's experiment conditions (Sec. 5) as session modes: shape-match (the shape is fitted on the
first frame after trk_set_pose and frozen afterwards) and smooth-bind (no shape estimation), against the
oracle driven the same way (an oracle without shape iterations takes over the state after frame 0)."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _depth(m, o, seed):
    return synth.add_noise(o.render(synth.gt_theta(m, 0.0), synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(seed))


def test_smooth_bind_keeps_phi_and_matches_a_pose_only_oracle():
    m = synth.make_model(1, mode=trk.MODE_SMOOTH_BIND)
    o = oracle.Oracle(dict(m, params=dict(m["params"], shape_iters=0)))
    depth = _depth(m, o, 3)
    th0 = synth.start_theta(m)
    P, S = m["params"]["pose_iters"], m["params"]["shape_iters"]
    with trk.Session(m) as s:
        s.set_pose(th0)
        o.set_state(th0, None)
        for f in range(3):
            g = s.track_frame(depth)
            e_ref, _, _ = o.track_frame(depth)
            assert np.all(g["offsets"] == 0.0)
            assert np.all(np.isnan(g["energy"][P:P + S]))
            assert np.max(np.abs(g["energy"][:P] - e_ref[:P]) / e_ref[:P]) < 1e-2
    th_ref, _, _ = o.get_state()
    assert np.abs(g["theta"] - th_ref).max() < 1e-3


def test_shape_match_fits_once_then_freezes_phi():
    m = synth.make_model(1, mode=trk.MODE_SHAPE_MATCH)
    o_full = oracle.Oracle(m)
    o_pose = oracle.Oracle(dict(m, params=dict(m["params"], shape_iters=0)))
    depth = _depth(m, o_full, 5)
    th0 = synth.start_theta(m)
    P, S = m["params"]["pose_iters"], m["params"]["shape_iters"]
    with trk.Session(m) as s:
        s.set_pose(th0)
        o_full.set_state(th0, None)
        g0 = s.track_frame(depth)
        o_full.track_frame(depth)
        th, phi, lam = o_full.get_state()
        o_pose.set_state(th, phi, lam)
        assert np.all(np.isfinite(g0["energy"]))
        for f in range(1, 4):
            g = s.track_frame(depth)
            o_pose.track_frame(depth)
            assert np.array_equal(g["offsets"], g0["offsets"])  # frozen after the first frame
            assert np.all(np.isnan(g["energy"][P:P + S]))
        th_ref, phi_ref, _ = o_pose.get_state()
        assert np.abs(g["theta"] - th_ref).max() < 1e-3
        H.assert_free_running_offsets(g0["offsets"], phi_ref)
        # a new sequence (trk_set_pose) fits the shape again on its first frame
        s.set_pose(th0)
        g = s.track_frame(depth)
        assert np.all(np.isfinite(g["energy"]))


def test_batches_take_tracking_mode_sessions_only():
    a = trk.Session(synth.make_model(1, V=500, width=48))
    b = trk.Session(synth.make_model(1, V=500, width=48, mode=trk.MODE_SMOOTH_BIND))
    with pytest.raises(trk.TrkError) as e:
        trk.Batch([a, b])
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
    a.close()
    b.close()
