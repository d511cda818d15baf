"""The coupled shape step (reading R22: the shape energy's damped Gauss-Newton system over all vertices,
block-Jacobi-preconditioned conjugate gradients) on the GPU against the oracle's, and in batches.

Tolerance: the iteration runs on FP32 vectors with FP64 dot products, the oracle entirely in FP64; r_i and
g_i agree to the Jacobi step's tolerances, and the offsets after k iterations to 5e-7 m, the Jacobi
step's (measured 6.5e-8 m for 1, 5 and 20 iterations, on steps of ~3 cm)."""
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


def _scene(iters, seed=9):
    m = synth.make_model(1, shape_solver=1, shape_sweeps=iters)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 7)
    th = gt + np.radians(2.0) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
    phi = (synth.gt_offsets(m, 0.0) * 0.5).astype(np.float32).astype(np.float64)
    return m, o, depth, th, phi


@pytest.mark.parametrize("iters", [1, 5, 20])
def test_coupled_shape_step_matches_the_oracle(iters):
    m, o, depth, th, phi = _scene(iters)
    with trk.Session(m) as s:
        s.set_pose(th, phi)
        s.set_depth(depth)
        for st in ("skin", "raster", "visibility", "associate", "shape"):
            s.step(st)
        phi_g = s.read("PHI")[:, :3].astype(np.float64)
        rg = s.read("SHAPE_RG")
        E_g = s.read("ENERGY")[m["params"]["pose_iters"]]
        corr = s.read("CORR")
    v, _ = o.skin(th, phi)
    n, ok = o.normals(v)
    acc, cnt = o.accumulate(v, depth, corr)
    _, inA, _ = o.residuals(th, n, ok, acc, cnt)
    E, phi_ref, r_ref, g_ref = o.shape_step(th, phi, n, acc, cnt, inA)
    A = inA > 0
    assert np.abs(rg[A, 3] - r_ref[A]).max() < 5e-6
    assert np.abs(rg[A, :3] - g_ref[A]).max() < 1e-4
    assert E_g == pytest.approx(E, rel=1e-5)
    d = np.abs(phi_g - phi_ref).max()
    print(f"iters {iters}: max |dphi| {d:.3e} m, step {np.abs(phi_ref - phi).max():.3e} m")
    assert d < 5e-7


def test_frames_with_the_coupled_shape_step():
    m, o, depth, th, phi = _scene(10, seed=3)
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


def test_batch_with_the_coupled_shape_step_equals_alone():
    ms = [synth.make_model(4, session=k, shape_solver=1, shape_sweeps=8) for k in (1, 4, 7)]
    alone, frames = [], []
    for i, m in enumerate(ms):
        with trk.Session(m) as s:
            rng = np.random.default_rng(90 + i)
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
                assert np.array_equal(r["theta"], alone[i][f]["theta"]), (i, f)
                assert np.array_equal(r["offsets"], alone[i][f]["offsets"]), (i, f)
                assert np.array_equal(r["energy"], alone[i][f]["energy"]), (i, f)
    for s in ss:
        s.close()
