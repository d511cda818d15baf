"""Grouped [J r] blocks (trk_params.jtj_group = 1, 2, 4): each block adds the rows of G consecutive
256-vertex blocks into one partial and writes a record per row for the candidate energies.  Whatever the
grouping, the normal equations, the energy and the LM step match the FP64 oracle at the GPU's own
association (the tolerances of the FP32 path: 1e-5 of the matrix scale, 1e-5 relative energy, the
oracle's LM decision and its step within 1e-6 rad)."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def _scene(G, V=4700, seed=0, prec=0):
    # 4700 vertices: 19 blocks of 256, so groups of 2 and 4 end with a partial group and a ragged block
    m = synth.make_model(1, V=V, jtj_group=G, precision=prec)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 7)
    th = gt + np.radians(2.0) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
    phi = (synth.gt_offsets(m, 0.0) * 0.5).astype(np.float32).astype(np.float64)
    return m, o, depth, th, phi


U = {trk.PRECISION_FP32: 0.0, trk.PRECISION_BF16X3: 2.0 ** -8, trk.PRECISION_TF32X3: 2.0 ** -11}


@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("prec", [trk.PRECISION_FP32, trk.PRECISION_TF32X3, trk.PRECISION_BF16X3])
def test_grouped_blocks_match_the_oracle(G, prec):
    """In the tensor-core modes the rows of a block's G vertex blocks accumulate in one TMEM accumulator;
    the normal equations are then checked within the split bound (3 u^2 + 770 2^-24) sum_k |x_ka x_kb|
    on top of the FP32 tolerance (the precision tests' bound)."""
    m, o, depth, th, phi = _scene(G, prec=prec)
    with trk.Session(m) as s:
        assert s.info()["jtj_group"] == G
        s.set_pose(th, phi)
        s.set_depth(depth)
        for st in ("skin", "raster", "visibility", "associate", "normal_equations"):
            s.step(st)
        A = s.read("NORMAL_EQ")
        E = s.read("ENERGY")[0]
        lam0 = s.read("LAMBDA")[0]
        corr = s.read("CORR")
        s.step("lm")
        trials = s.read("LM_TRIALS")
        th_gpu = s.read("THETA")
        lam_gpu = s.read("LAMBDA")[0]
    v, _ = o.skin(th, phi)
    n, ok = o.normals(v)
    acc, cnt = o.accumulate(v, depth, corr)
    r, inA, E_ref = o.residuals(th, n, ok, acc, cnt)
    assert inA.sum() > 500
    J = o.jacobian(th, phi, n, inA)
    JTJ, JTr = oracle.normal_eq(J, r, inA)
    L = o.L
    R = np.column_stack([J, r])[inA.astype(bool)]
    split = (3 * U[prec] ** 2 + 770 * 2.0 ** -24) * (np.abs(R).T @ np.abs(R)) if prec else 0.0
    ref = np.zeros((L + 1, L + 1))
    ref[:L, :L], ref[:L, L], ref[L, :L] = JTJ, JTr, JTr
    err = np.abs(A - ref)
    err[L, L] = 0.0
    tol = np.zeros_like(err)
    tol[:L, :L] = 1e-5 * np.abs(JTJ).max()
    tol[:L, L] = tol[L, :L] = 1e-4 * np.abs(JTr).max() + 1e-9
    assert (err <= tol + split).all(), (err / (tol + split)).max()
    assert E == pytest.approx(E_ref, rel=1e-5)
    o.set_state(th, phi)
    a_ref, th_ref, lam_ref, Ec = o.lm_step(A[:L, :L], A[:L, L], trials[6], v, n, acc, cnt, inA, th, lam0)
    assert int(trials[7]) == a_ref
    assert np.abs(th_gpu - th_ref).max() < 1e-6
    assert lam_gpu == pytest.approx(lam_ref, rel=1e-12)
    both = np.isfinite(Ec) & np.isfinite(trials[:6])
    assert both.any() and np.allclose(trials[:6][both], Ec[both], rtol=1e-5)


def _auto_group(m):
    """The grouping trk_create picks: the larger of the choice by mesh size and by the expected rows per
    256 vertices, r = 128 c / V with c the distinct pixels the template's vertices round to."""
    v = np.asarray(m["mesh"]["verts"], np.float32).astype(np.float64).reshape(-1, 3)  # as the C ABI gets them
    c = {k: float(np.float32(x)) if isinstance(x, float) else x for k, x in m["camera"].items()}
    V, W, H = len(v), c["width"], c["height"]
    nblk = -(-V // 256)
    by_size = 1 if nblk <= 304 else 2 if nblk <= 608 else 4
    z = v[:, 2]
    ok = z > float(np.float32(m["params"]["z_near"]))
    u = np.floor(c["fx"] * v[ok, 0] / z[ok] + c["cx"] + 0.5)
    w = np.floor(c["fy"] * v[ok, 1] / z[ok] + c["cy"] + 0.5)
    ins = (u >= 0) & (w >= 0) & (u < W) & (w < H)
    covered = len(np.unique((w[ins] * W + u[ins]).astype(np.int64)))
    rows = 256 * 0.5 * covered / V
    return max(by_size, 4 if rows < 18 else 2 if rows < 30 else 1)


def test_group_chosen_from_the_mesh_and_its_image_coverage():
    seen = set()
    for m in (synth.make_model(2), synth.make_model(1, V=5000, width=640), synth.make_model(4, session=3),
              synth.make_model(4, session=5), synth.make_model(3)):
        with trk.Session(m) as s:
            assert s.info()["jtj_group"] == _auto_group(m)
            seen.add(s.info()["jtj_group"])
    assert seen == {1, 2, 4}, seen
    m = synth.make_model(4, session=5, precision=trk.PRECISION_TF32X3)  # the tensor-core modes choose alike
    with trk.Session(m) as s:
        assert s.info()["jtj_group"] == _auto_group(m)


@pytest.mark.parametrize("kw", [dict(jtj_group=3), dict(jtj_group=-1), dict(jtj_group=8)])
def test_invalid_group_is_rejected(kw):
    with pytest.raises(trk.TrkError) as e:
        trk.Session(synth.make_model(1, V=500, width=64, **kw))
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
