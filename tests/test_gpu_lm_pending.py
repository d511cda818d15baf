"""The LM candidates scored in two passes (Sec. 4.2): the first launch scores lambda and 10 lambda and
accepts one of them when it does not raise E; otherwise the second scores the other four and decides over
all six.  From a far start with almost no damping (lambda_k0 = 1e-7, 25 degrees off) the undamped steps
overshoot, so the second pass and the no-acceptance case are reached; at every iteration the decision,
the step and lambda match the FP64 oracle's LM on the GPU's own normal equations and association."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1711_07999_gb300 import trk  # noqa: E402


def test_decisions_of_both_passes_match_the_oracle():
    decisions = []
    for seed in range(3):
        m = synth.make_model(1, V=3000, lambda_k0=1e-7)
        o = oracle.Oracle(m)
        gt = synth.gt_theta(m, 0.0)
        depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(seed))
        rng = np.random.default_rng(100 + seed)
        th0 = gt + np.radians(25.0) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
        L = o.L
        with trk.Session(m) as s:
            s.set_pose(th0)
            s.set_depth(depth)
            for it in range(6):
                th_g = s.read("THETA")
                lam0 = s.read("LAMBDA")[0]
                for st in ("skin", "raster", "visibility", "associate", "normal_equations"):
                    s.step(st)
                A = s.read("NORMAL_EQ")
                corr = s.read("CORR")
                s.step("lm")
                trials = s.read("LM_TRIALS")
                th_gpu = s.read("THETA")
                lam_gpu = s.read("LAMBDA")[0]
                zero = np.zeros((o.V, 3))
                v, _ = o.skin(th_g, zero)
                n, ok = o.normals(v)
                acc, cnt = o.accumulate(v, depth, corr)
                _, inA, _ = o.residuals(th_g, n, ok, acc, cnt)
                o.set_state(th_g, None)
                a_ref, th_ref, lam_ref, Ec = o.lm_step(A[:L, :L], A[:L, L], trials[6], v, n, acc, cnt, inA, th_g,
                                                       lam0)
                a = int(trials[7])
                decisions.append(a)
                assert a == a_ref, (seed, it)
                assert np.abs(th_gpu - th_ref).max() < 1e-6, (seed, it)
                assert lam_gpu == pytest.approx(lam_ref, rel=1e-12), (seed, it)
                both = np.isfinite(Ec) & np.isfinite(trials[:6])
                assert np.allclose(trials[:6][both], Ec[both], rtol=1e-5), (seed, it)
                hi = a + 1 if a >= 0 else 6  # every candidate up to the decision was scored
                for c in range(hi):
                    if np.isfinite(Ec[c]):
                        assert np.isfinite(trials[c]), (seed, it, c)
    print("decisions", decisions)
    assert any(a >= 2 or a < 0 for a in decisions), decisions
