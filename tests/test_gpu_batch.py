"""Batches (trk_batch_*): every stage of a frame as one launch over the blocks of many uneven sessions.
Each member's results must be bitwise those it computes alone (same kernels' arithmetic per block, fixed
reduction orders, order-independent integer sums), so the comparison is exact."""
import numpy as np
import pytest

from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _frames(m, s, n, seed):
    rng = np.random.default_rng(seed)
    return [synth.add_noise(s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 4, rng)
            for f in range(n)]


def _run(models, prec, n_frames):
    ms = [synth.make_model(4, session=k, precision=prec) if isinstance(k, int) else k for k in models]
    alone, frames = [], []
    for i, m in enumerate(ms):
        with trk.Session(m) as s:
            fr = _frames(m, s, n_frames, 50 + i)
            frames.append(fr)
            s.set_pose(synth.gt_theta(m, 0.0))
            alone.append([s.track_frame(f) for f in fr])
    sessions = [trk.Session(m) for m in ms]
    for m, s in zip(ms, sessions):
        s.set_pose(synth.gt_theta(m, 0.0))
    dev = [[torch.from_numpy(f).cuda() for f in fr] for fr in frames]
    st = torch.cuda.Stream()
    got = [[] for _ in ms]
    with trk.Batch(sessions) as b:
        for f in range(n_frames):
            b.track_device([dev[i][f].data_ptr() for i in range(len(ms))], st.cuda_stream)
            st.synchronize()
            for i, s in enumerate(sessions):
                got[i].append(s.read_result())
    for s in sessions:
        s.close()
    return alone, got


def _assert_same(alone, got):
    for i, (a_i, g_i) in enumerate(zip(alone, got)):
        for f, (a, g) in enumerate(zip(a_i, g_i)):
            assert np.array_equal(a["theta"], g["theta"]), (i, f)
            assert np.array_equal(a["offsets"], g["offsets"]), (i, f)
            assert np.array_equal(a["energy"], g["energy"]), (i, f)
            assert a["n_assoc_px"] == g["n_assoc_px"] and a["n_assoc_verts"] == g["n_assoc_verts"], (i, f)


def test_uneven_batch_equals_each_session_alone():
    # sizes 6k-160k vertices, 26-70 links, all three image sizes
    alone, got = _run([0, 1, 4, 5, 6, 7], trk.PRECISION_FP32, 3)
    _assert_same(alone, got)


def test_batch_on_the_tensor_cores_equals_alone():
    alone, got = _run([1, 4, 7], trk.PRECISION_TF32X3, 2)
    _assert_same(alone, got)


def test_single_member_batch_and_small_meshes():
    m = synth.make_model(1, V=400, width=48)
    alone, got = _run([m, synth.make_model(1, session=2, V=2000, width=64)], trk.PRECISION_FP32, 2)
    _assert_same(alone, got)
    alone, got = _run([synth.make_model(1, session=3, V=900, width=40)], trk.PRECISION_FP32, 2)
    _assert_same(alone, got)


def test_members_must_share_schedule_and_precision():
    a = trk.Session(synth.make_model(1, V=500, width=48))
    b = trk.Session(synth.make_model(1, V=500, width=48, pose_iters=5))
    c = trk.Session(synth.make_model(1, V=500, width=48, precision=trk.PRECISION_TF32X3))
    for group in ([a, b], [a, c], [a, a]):
        with pytest.raises(trk.TrkError) as e:
            trk.Batch(group)
        assert e.value.status == trk.TRK_ERR_INVALID_ARG
    for s in (a, b, c):
        s.close()


def test_members_with_different_jtj_groups():
    # the same kind of session with 1, 2 and 4 vertex blocks per [J r] block, in one batch
    ms = [synth.make_model(1, session=10 + G, V=6000, width=96, jtj_group=G) for G in (1, 2, 4)]
    alone, got = _run(ms, trk.PRECISION_FP32, 2)
    _assert_same(alone, got)
