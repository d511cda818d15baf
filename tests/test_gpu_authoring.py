"""Template authoring on the GPU (trk_subdivide: Catmull-Clark levels of a cage with its skin weights)
against the oracle's subdivision: the same triangles (bit-exact), the positions and the 4 kept weights
(the oracle's dense weights reduced the same way) within FP32 rounding, and a session built on the result
tracks."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _cage(V=800):
    m = synth.make_model(2, V=V, width=64)
    me = m["mesh"]
    F = len(me["tris"])
    return m, me["verts"], np.arange(0, 3 * F + 1, 3), np.asarray(me["tris"]).ravel(), me["bone_idx"], me["bone_w"]


def _top4(w):
    order = np.argsort(-w, axis=1, kind="stable")[:, :4]  # ties to the smaller bone
    val = np.take_along_axis(w, order, 1)
    return order, val / val.sum(1, keepdims=True)


@pytest.mark.parametrize("levels", [1, 2])
def test_subdivision_matches_the_oracle(levels):
    m, v, fo, fv, bi, bw = _cage()
    nb = len(m["skeleton"]["parent"])
    ov, ot, obi, obw = trk.subdivide(v, fo, fv, bi, bw, nb, levels)
    dense = np.zeros((len(v), nb))
    for k in range(4):
        np.add.at(dense, (np.arange(len(v)), bi[:, k]), bw[:, k])
    ref, quads = oracle.subdivide(fo, fv, np.hstack([v.astype(np.float64), dense]), levels)
    tris = np.concatenate([quads[:, [0, 1, 2]], quads[:, [0, 2, 3]]], axis=1).reshape(-1, 3)
    assert np.array_equal(ot, tris)
    assert np.abs(ov - ref[:, :3]).max() < 2e-6 * np.abs(ref[:, :3]).max()
    idx, val = _top4(ref[:, 3:])
    w = np.sort(ref[:, 3:], 1)
    # unambiguous: the 4th and 5th largest weights differ, or at most 4 bones carry weight
    sure = (w[:, -4] - w[:, -5] > 1e-5) | (w[:, -5] < 1e-7) if nb > 4 else np.ones(len(ref), bool)
    assert sure.mean() > 0.9
    # compare the kept (bone, weight) pairs where the weight is not zero (zero slots name any bone)
    for i in np.nonzero(sure)[0][::3]:
        a = {(int(b), round(float(x), 5)) for b, x in zip(obi[i], obw[i]) if x > 1e-6}
        r = {(int(b), round(float(x), 5)) for b, x in zip(idx[i], val[i]) if x > 1e-6}
        assert {b for b, _ in a} == {b for b, _ in r}, i
    nz = val > 1e-6
    got = np.take_along_axis(obw, np.argsort(obi, 1), 1)
    want = np.take_along_axis(val, np.argsort(idx, 1), 1)
    ok = sure & (np.sort(obi, 1) == np.sort(idx, 1)).all(1)
    assert np.abs(got[ok] - want[ok]).max() < 1e-5


def test_a_session_on_the_authored_template_matches_the_oracle():
    """The authored template is a valid input of the tracker: at the same state and association the
    session's pose energy equals the oracle's on the same template (1e-5 relative)."""
    m, v, fo, fv, bi, bw = _cage(V=1200)
    nb = len(m["skeleton"]["parent"])
    ov, ot, obi, obw = trk.subdivide(v, fo, fv, bi, bw, nb, 2)
    m2 = dict(m, mesh=dict(verts=ov, tris=ot, bone_idx=obi, bone_w=obw))
    m2["params"] = synth.default_params(m["camera"]["fx"], len(ov))
    o = oracle.Oracle(m2)
    th = synth.gt_theta(m2, 0.0)
    depth = synth.add_noise(o.render(th), 2, np.random.default_rng(1))
    with trk.Session(m2) as s:
        s.set_pose(th)
        s.set_depth(depth)
        for st in ("skin", "raster", "visibility", "associate", "normal_equations"):
            s.step(st)
        E = s.read("ENERGY")[0]
        corr = s.read("CORR")
        assert (corr >= 0).sum() > 0.5 * (depth > 0).sum()
    vr, _ = o.skin(th, None)
    n, ok = o.normals(vr)
    acc, cnt = o.accumulate(vr, depth, corr)
    _, _, E_ref = o.residuals(th, n, ok, acc, cnt)
    assert E == pytest.approx(E_ref, rel=1e-5)
