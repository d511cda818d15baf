"""Schedules and the autotuner (trk_schedule_*): every grouping of the sessions gives each session bitwise
its results alone; the autotuner's choice is stored and read back from its cache."""
import numpy as np
import pytest

from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402

IDS = [1, 4, 7, 9, 12]


def _setup(ids):
    ms = [synth.make_model(4, session=k) for k in ids]
    ss = [trk.Session(m) for m in ms]
    frames = []
    for i, (m, s) in enumerate(zip(ms, ss)):
        rng = np.random.default_rng(70 + i)
        frames.append([torch.from_numpy(synth.add_noise(
            s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 4, rng)).cuda()
            for f in range(3)])
        s.set_pose(synth.gt_theta(m, 0.0))
    return ms, ss, frames


def _alone(ms, frames):
    out = []
    for m, fr in zip(ms, frames):
        with trk.Session(m) as s:
            s.set_pose(synth.gt_theta(m, 0.0))
            out.append([s.track_frame(f.cpu().numpy()) for f in fr])
    return out


@pytest.mark.parametrize("groups", [1, 2, 5])
def test_every_grouping_equals_each_session_alone(groups):
    ms, ss, frames = _setup(IDS)
    alone = _alone(ms, frames)
    st = torch.cuda.Stream()
    with trk.Schedule(ss, dict(groups=groups, assoc_blocks=304, tail_blocks=152)) as sc:
        assert sc.config()["groups"] == groups
        for f in range(3):
            sc.track_device([fr[f].data_ptr() for fr in frames], st.cuda_stream)
            st.synchronize()
            for i, s in enumerate(ss):
                g = s.read_result()
                a = alone[i][f]
                assert np.array_equal(a["theta"], g["theta"]) and np.array_equal(a["offsets"], g["offsets"]), (i, f)
                assert np.array_equal(a["energy"], g["energy"]), (i, f)
    for s in ss:
        s.close()


def test_autotune_picks_a_schedule_and_caches_it(tmp_path):
    ms, ss, frames = _setup(IDS[:3])
    cache = str(tmp_path / "tune.json")
    ptrs = [fr[0].data_ptr() for fr in frames]
    with trk.Schedule(ss) as sc:
        cfg, ms_step = sc.autotune(ptrs, reps=1, cache_path=cache)
        assert 1 <= cfg["groups"] <= 3 and ms_step > 0
        assert sc.config() == cfg
    sig = trk.Schedule.signature(ss)
    assert trk.tuning_cache_lookup(cache, sig)[0] == cfg
    with trk.Schedule(ss, cache_path=cache) as sc2:  # a later schedule of the same size class reads it
        assert sc2.config() == cfg
    with pytest.raises(trk.TrkError):
        trk.Schedule(ss, dict(groups=4, assoc_blocks=304, tail_blocks=152))  # more groups than sessions
    for s in ss:
        s.close()
