"""The raster-ID association (reading R23: the nearest corner of the triangle the z-buffer holds at the
pixel) on the GPU against the oracle's: the correspondence map bit-exact except where the oracle flags a
tie (a marginal z-buffer decision, two corners or a corner and the cutoff within 1e-5 m), the per-vertex
sums of the map, whole frames, and batches."""
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


def _scene(seed=0, **over):
    m = synth.make_model(1, association=1, **over)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 7)
    th = gt + np.radians(2.0) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
    phi = (synth.gt_offsets(m, 0.0) * 0.5).astype(np.float32).astype(np.float64)
    return m, o, depth, th, phi


def test_map_bit_exact_except_ties():
    m, o, depth, th, phi = _scene()
    with trk.Session(m) as s:
        s.set_pose(th, phi)
        s.set_depth(depth)
        for st in ("skin", "raster", "visibility", "associate"):
            s.step(st)
        corr = s.read("CORR").reshape(depth.shape)
        acc = s.read("ACC")
        v = s.read("VERTS")[:, :3].astype(np.float64)
    v_ref, _ = o.skin(th, phi)
    _, ztri, amb = o.raster(v_ref, with_amb=True)
    ref, _, _, tie = o.associate_rid(v_ref, ztri, depth, zamb=amb, with_tie=True)
    diff = corr != ref
    assert (ref >= 0).sum() > 500  # only pixels the model covers can get a correspondence
    assert not (diff & ~(tie > 0)).any(), np.argwhere(diff & ~(tie > 0))[:5]
    assert (tie > 0).mean() < 0.05
    acc_ref, cnt_ref = o.accumulate(v, depth, corr)
    assert np.array_equal(acc[:, 3], cnt_ref)
    assert np.all(np.abs(acc[:, :3] / 2.0 ** 30 - acc_ref) <= 5e-7 * np.maximum(cnt_ref, 1)[:, None])


def test_frames_with_raster_id_association():
    m, o, depth, th, phi = _scene(seed=3)
    th0 = synth.start_theta(m)
    with trk.Session(m) as s:
        s.set_pose(th0)
        o.set_state(th0, None)
        for f in range(3):
            g = s.track_frame(depth)
            e_ref, _, _ = o.track_frame(depth)
    th_ref, phi_ref, _ = o.get_state()
    assert np.abs(g["theta"] - th_ref).max() < 1e-3
    H.assert_free_running_offsets(g["offsets"], phi_ref)
    assert np.max(np.abs(g["energy"] - e_ref) / e_ref) < 1e-2


def test_batch_with_raster_id_association_equals_alone():
    ms = [synth.make_model(4, session=k, association=1) for k in (1, 4)]
    alone, frames = [], []
    for i, m in enumerate(ms):
        with trk.Session(m) as s:
            rng = np.random.default_rng(40 + i)
            fr = [synth.add_noise(s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 4, rng)
                  for f in range(2)]
            frames.append(fr)
            s.set_pose(synth.gt_theta(m, 0.0))
            alone.append([s.track_frame(f) for f in fr])
    ss = [trk.Session(m) for m in ms]
    for m, s in zip(ms, ss):
        s.set_pose(synth.gt_theta(m, 0.0))
    dev = [[torch.from_numpy(f).cuda() for f in fr] for fr in frames]
    st = torch.cuda.Stream()
    with trk.Batch(ss) as b:
        for f in range(2):
            b.track_device([dev[i][f].data_ptr() for i in range(len(ss))], st.cuda_stream)
            st.synchronize()
            for i, s in enumerate(ss):
                r = s.read_result()
                assert np.array_equal(r["theta"], alone[i][f]["theta"]) and np.array_equal(r["offsets"], alone[i][f]["offsets"])
    for s in ss:
        s.close()
