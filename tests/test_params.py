"""trk_create rejects parameters outside their documented ranges before it touches the device (host logic:
runs with or without a GPU)."""
import pytest

from paper_1711_07999_gb300 import synth, trk


@pytest.mark.parametrize("kw, msg", [
    (dict(jtj_group=3), "jtj_group 3"),
    (dict(jtj_group=-1), "jtj_group -1"),
    (dict(jtj_group=8), "jtj_group 8"),
    (dict(precision=7), "precision 7"),
    (dict(shape_solver=2), "shape_solver 2"),
    (dict(mode=9), "mode 9"),
    (dict(association=2), "association 2"),
    (dict(knn=5), "bad params"),
    (dict(shape_sweeps=0), "bad params"),
])
def test_out_of_range_parameters_are_rejected(kw, msg):
    with pytest.raises(trk.TrkError) as e:
        trk.Session(synth.make_model(1, V=500, width=48, **kw))
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
    assert msg in str(e.value)
