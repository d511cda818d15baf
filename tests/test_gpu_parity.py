"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and per frame.

Tolerances (FP32 GPU vs FP64 oracle):
  positions 3e-6 m (a few FP32 ulps of ~3 m coordinates); normals and g = dr/dphi 1e-4 (a position error
  of ~3e-7 m over edges of ~5 mm tilts a face normal by ~1e-4); depths 2e-6 relative;
  correspondences bit-exact except where the oracle flags a tie (two candidates, the cutoff or a
  visibility / bucket decision within 1e-5 m, or a z-buffer coverage decision within 1e-3 px);
  per-iteration energy 1e-5 relative at the same state and association; J^T J, J^T r 1e-5 relative to
  the matrix scale; final joint values 1e-3 rad; offsets 0.05 mm.
"""
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


def _scene(cfg=1, V=None, width=None, seed=0, pert=2.0, phi_scale=0.5):
    m = synth.make_model(cfg, V=V, width=width)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    phi_gt = synth.gt_offsets(m, 0.0)
    depth = synth.add_noise(o.render(gt, phi_gt), cfg, np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 7)
    th = gt + np.radians(pert) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
    phi = (phi_gt * phi_scale).astype(np.float32).astype(np.float64)
    return m, o, depth, th, phi


def _gpu_pass(s, th, phi, depth):
    s.set_pose(th, phi)
    s.set_depth(depth)
    for st in ("skin", "raster", "visibility", "associate"):
        s.step(st)


@pytest.fixture(scope="module")
def cfg1():
    m, o, depth, th, phi = _scene(1)
    s = trk.Session(m)
    _gpu_pass(s, th, phi, depth)
    yield m, o, depth, th, phi, s
    s.close()


def test_derived_model_data_match(cfg1):
    m, o, depth, th, phi, s = cfg1
    bind, S, nbr = o.derived()
    assert np.array_equal(s.read("NEIGHBOURS")[:, :m["params"]["knn"]], nbr)
    prior2 = (float(np.float32(m["params"]["lambda_s"])) * S) ** 2
    assert np.allclose(s.read("PRIOR"), prior2, rtol=1e-6, atol=0)


def test_skinning(cfg1):
    m, o, depth, th, phi, s = cfg1
    v_ref, _ = o.skin(th, phi)
    v = s.read("VERTS")[:, :3].astype(np.float64)
    assert np.abs(v - v_ref).max() < 3e-6


def test_raster_on_the_same_vertices(cfg1):
    m, o, depth, th, phi, s = cfg1
    v = s.read("VERTS")[:, :3].astype(np.float64)
    z_ref, zt_ref, amb = o.raster(v, with_amb=True)
    key = s.read("ZBUF")
    empty = key == np.uint64(0xFFFFFFFFFFFFFFFF)
    zg = (key >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    zg[empty] = np.inf
    zg = zg.reshape(z_ref.shape)
    ok = ~amb.astype(bool)
    assert np.array_equal(np.isfinite(zg)[ok], np.isfinite(z_ref)[ok])
    both = ok & np.isfinite(z_ref)
    assert both.sum() > 500
    assert np.abs(zg[both] - z_ref[both]).max() <= 2e-6 * z_ref[both].max()


def test_normals_and_visibility(cfg1):
    m, o, depth, th, phi, s = cfg1
    v = s.read("VERTS")[:, :3].astype(np.float64)
    n_ref, ok_ref = o.normals(v)
    n4 = s.read("NORMALS")
    assert np.array_equal(n4[:, 3] > 0, ok_ref > 0)
    assert np.abs(n4[:, :3] - n_ref).max() < 1e-4
    z_ref, _, amb = o.raster(v, with_amb=True)
    vis_ref, pix_ref, marg = o.visibility(v, n_ref, ok_ref, z_ref, amb, with_marg=True)
    vp = s.read("VISPIX")
    sure = marg == 0
    assert np.array_equal((vp >= 0)[sure], (vis_ref > 0)[sure])
    both = sure & (vp >= 0)
    assert np.array_equal(vp[both], pix_ref[both])
    assert (vis_ref > 0).sum() > 1000


def test_association_bit_exact_except_ties(cfg1):
    m, o, depth, th, phi, s = cfg1
    ref = o.pass_at(th, phi, depth, with_ties=True)
    corr = s.read("CORR").reshape(ref["corr"].shape)
    tie = ref["tie"] > 0
    diff = corr != ref["corr"]
    assert (ref["corr"] >= 0).sum() > 1000
    assert not (diff & ~tie).any(), np.argwhere(diff & ~tie)[:5]
    assert tie.mean() < 0.05
    # the per-vertex sums of the GPU's own map equal the oracle's sums for that map
    v = s.read("VERTS")[:, :3].astype(np.float64)
    acc_ref, cnt_ref = o.accumulate(v, depth, corr)
    acc = s.read("ACC")
    assert np.array_equal(acc[:, 3], cnt_ref)
    # each term carries the FP32 rounding of v and p at ~3 m (<= 2.5e-7 m) and the 2^-30 m quantum
    assert np.all(np.abs(acc[:, :3] / 2.0 ** 30 - acc_ref) <= 5e-7 * np.maximum(cnt_ref, 1)[:, None])


def _oracle_at_gpu_association(o, s, th, phi, depth):
    """The oracle's residuals, Jacobian and normal equations on the GPU's own correspondence map
    (so that both sides see the same association)."""
    v_ref, _ = o.skin(th, phi)
    n_ref, ok_ref = o.normals(v_ref)
    corr = s.read("CORR")
    acc, cnt = o.accumulate(v_ref, depth, corr)
    r, inA, E = o.residuals(th, n_ref, ok_ref, acc, cnt)
    J = o.jacobian(th, phi, n_ref, inA)
    JTJ, JTr = oracle.normal_eq(J, r, inA)
    return dict(v=v_ref, n=n_ref, acc=acc, cnt=cnt, r=r, inA=inA, E=E, J=J, JTJ=JTJ, JTr=JTr)


def test_normal_equations_and_energy(cfg1):
    m, o, depth, th, phi, s = cfg1
    s.step("normal_equations")
    R = _oracle_at_gpu_association(o, s, th, phi, depth)
    A = s.read("NORMAL_EQ")
    L = o.L
    scale = np.sqrt(np.outer(np.diag(R["JTJ"]), np.diag(R["JTJ"]))) + 1e-12
    assert np.abs(A[:L, :L] - R["JTJ"]).max() / np.abs(R["JTJ"]).max() < 1e-5
    assert (np.abs(A[:L, :L] - R["JTJ"]) / scale).max() < 1e-4
    assert np.abs(A[:L, L] - R["JTr"]).max() <= 1e-4 * np.abs(R["JTr"]).max() + 1e-9
    E = s.read("ENERGY")[0]
    assert E == pytest.approx(R["E"], rel=1e-5)


def test_lm_step_matches_fp64_solve_of_the_same_system(cfg1):
    m, o, depth, th, phi, s = cfg1
    s.step("normal_equations")
    A = s.read("NORMAL_EQ")
    lam0 = s.read("LAMBDA")[0]
    s.step("lm")
    trials = s.read("LM_TRIALS")
    a = int(trials[7])
    th_gpu = s.read("THETA")
    # the oracle's LM on the GPU's normal equations and association gives the same decision and step
    R = _oracle_at_gpu_association(o, s, th, phi, depth)
    L = o.L
    o.set_state(th, phi)
    a_ref, th_ref, lam_ref, Ec = o.lm_step(A[:L, :L], A[:L, L], trials[6], R["v"], R["n"], R["acc"], R["cnt"],
                                           R["inA"], th, lam0)
    assert a == a_ref
    assert np.abs(th_gpu - th_ref).max() < 1e-6
    assert s.read("LAMBDA")[0] == pytest.approx(lam_ref, rel=1e-12)
    tried = np.isfinite(Ec)
    assert np.allclose(trials[:6][tried], Ec[tried], rtol=1e-5)


def test_shape_step(cfg1):
    m, o, depth, th, phi, s = cfg1
    _gpu_pass(s, th, phi, depth)
    s.step("shape")
    R = _oracle_at_gpu_association(o, s, th, phi, depth)
    E_ref, phi_ref, r_ref, g_ref = o.shape_step(th, phi, R["n"], R["acc"], R["cnt"], R["inA"])
    rg = s.read("SHAPE_RG")
    A = R["inA"] > 0
    assert np.abs(rg[A, 3] - r_ref[A]).max() < 5e-6
    assert np.abs(rg[A, :3] - g_ref[A]).max() < 1e-4
    assert np.abs(s.read("PHI")[:, :3] - phi_ref).max() < 5e-7
    assert s.read("ENERGY")[m["params"]["pose_iters"]] == pytest.approx(E_ref, rel=1e-5)


def test_render_depth_matches_oracle(cfg1):
    m, o, depth, th, phi, s = cfg1
    state = [s.read(f) for f in ("THETA", "PHI", "LAMBDA")]
    d_gpu = s.render_depth(th, phi).astype(np.float64)
    v = o.skin(th, phi)[0]
    z_ref, _, amb = o.raster(v, with_amb=True)
    ok = ~amb.astype(bool)
    ref = np.where(np.isfinite(z_ref), z_ref, 0.0)
    both = ok & (ref > 0) & (d_gpu > 0)
    assert np.array_equal((d_gpu > 0)[ok], (ref > 0)[ok]) or ((d_gpu > 0) != (ref > 0))[ok].sum() < 5
    assert np.abs(d_gpu[both] - ref[both]).max() < 1e-5
    # rendering leaves the tracking state (Theta, Phi, the LM damping) bit for bit alone
    for f, before in zip(("THETA", "PHI", "LAMBDA"), state):
        assert np.array_equal(s.read(f), before), f


_assert_offsets_close = H.assert_free_running_offsets


def _track_both(m, o, depth, th0, frames=1):
    with trk.Session(m) as s:
        s.set_pose(th0)
        o.set_state(th0, None)
        outs = []
        for f in range(frames):
            d = depth[f] if isinstance(depth, list) else depth
            g = s.track_frame(d)
            e_ref, acc_ref, na_ref = o.track_frame(d)
            th_ref, phi_ref, lam_ref = o.get_state()
            outs.append((g, e_ref, th_ref, phi_ref, na_ref))
    return outs


def test_frame_config1_end_to_end():
    # config 1 starts 10 degrees off; the first frame's 10 iterations do not converge, so the final
    # state is compared after three frames on the same depth image (30 pose iterations)
    m, o, depth, th, phi = _scene(1, seed=3)
    th0 = synth.start_theta(m)
    outs = _track_both(m, o, depth, th0, frames=3)
    g, e_ref, th_ref, phi_ref, na_ref = outs[-1]
    assert np.abs(g["theta"] - th_ref).max() < 1e-3
    _assert_offsets_close(g["offsets"], phi_ref)
    assert abs(g["n_assoc_px"] - na_ref) <= max(5, 0.01 * na_ref)
    g0, e0_ref = outs[0][0], outs[0][1]
    rel = np.abs(g0["energy"] - e0_ref) / e0_ref
    assert rel.max() < 1e-2, rel  # free-running first frame: paths differ by tie flips and rounding


def test_energy_per_iteration_at_matched_state():
    """Per-iteration energy parity (1e-5 relative): at each pose iteration, the oracle's E_pose at the
    GPU's own state and association equals the GPU's."""
    m, o, depth, th, phi = _scene(1, seed=4)
    th0 = synth.start_theta(m)
    with trk.Session(m) as s:
        s.set_pose(th0)
        s.set_depth(depth)
        for it in range(m["params"]["pose_iters"]):
            th_g = s.read("THETA")
            for st in ("skin", "raster", "visibility", "associate", "normal_equations"):
                s.step(st)
            E_g = s.read("ENERGY")[0]
            R = _oracle_at_gpu_association(o, s, th_g, np.zeros((o.V, 3)), depth)
            assert E_g == pytest.approx(R["E"], rel=1e-5), it
            s.step("lm")


def test_frame_sequence_config2_full_size():
    """The 50k-vertex / 640x480 workload, two frames of its sequence, free-running through the same graph
    the benchmark times (the lockstep comparison of every frame is in test_gpu_sequence.py)."""
    m = synth.make_model(2)
    o = oracle.Oracle(m)
    rng = np.random.default_rng(11)
    frames = []
    for f in range(2):
        t = f / 30.0
        frames.append(synth.add_noise(o.render(synth.gt_theta(m, t), synth.gt_offsets(m, t)), 2, rng))
    outs = _track_both(m, o, frames, synth.start_theta(m), frames=2)
    for g, e_ref, th_ref, phi_ref, na_ref in outs:
        assert np.abs(g["theta"] - th_ref).max() < 1e-3
        _assert_offsets_close(g["offsets"], phi_ref)
        # free-running energies: each association tie flip moves a pixel between two vertices
        assert np.max(np.abs(g["energy"] - e_ref) / e_ref) < 1e-2


def test_device_entry_point_on_a_torch_stream():
    m, o, depth, th, phi = _scene(1, seed=5)
    th0 = synth.start_theta(m)
    with trk.Session(m) as a, trk.Session(m) as b:
        a.set_pose(th0)
        b.set_pose(th0)
        ra = a.track_frame(depth)
        dt = torch.from_numpy(depth).cuda()
        st = torch.cuda.Stream()
        b.track_frame_device(dt.data_ptr(), st.cuda_stream)
        rb = b.read_result()
    assert np.array_equal(ra["theta"], rb["theta"])
    assert np.array_equal(ra["offsets"], rb["offsets"])
    assert np.array_equal(ra["energy"], rb["energy"])


def test_results_are_deterministic():
    m, o, depth, th, phi = _scene(1, seed=6)
    th0 = synth.start_theta(m)
    res = []
    for _ in range(2):
        with trk.Session(m) as s:
            s.set_pose(th0)
            res.append(s.track_frame(depth))
    assert np.array_equal(res[0]["theta"], res[1]["theta"])
    assert np.array_equal(res[0]["offsets"], res[1]["offsets"])


def test_edge_cases():
    m, o, depth, th, phi = _scene(1, seed=8)
    with trk.Session(m) as s:
        s.set_pose(th)
        # an empty depth image: nothing is associated, the pose does not move (prior only on non-root)
        out = s.track_frame(np.zeros_like(depth))
        assert out["n_assoc_px"] == 0 and out["n_assoc_verts"] == 0
        assert np.isfinite(out["theta"]).all()
        with pytest.raises(trk.TrkError) as e:
            s.set_pose(np.full(o.L, np.nan))
        assert e.value.status == trk.TRK_ERR_NUMERIC
    bad = synth.make_model(1, V=500)
    bad["mesh"]["tris"] = bad["mesh"]["tris"].copy()
    bad["mesh"]["tris"][0, 0] = 10 ** 6
    with pytest.raises(trk.TrkError) as e:
        trk.Session(bad)
    assert e.value.status == trk.TRK_ERR_INVALID_ARG
    big = synth.make_model(1, V=500)
    L = 80
    big["skeleton"] = dict(parent=np.arange(-1, L - 1, dtype=np.int32), type=np.zeros(L, np.int32),
                           axis=np.tile([1, 0, 0], (L, 1)).astype(np.float32),
                           offset_dq=np.tile([1, 0, 0, 0, 0, 0, 0, 0], (L, 1)).astype(np.float32),
                           prior_mask=np.ones(L, np.float32))
    with pytest.raises(trk.TrkError) as e:
        trk.Session(big)
    assert e.value.status == trk.TRK_ERR_NO_CAPACITY


def test_smallest_meshes_and_ragged_sizes():
    # a mesh smaller than one block, an image that is not a multiple of the 16x16 pixel tile
    m = synth.make_model(1, V=300, width=37, height=29)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0)
    depth = o.render(gt).astype(np.float32)
    (g, e_ref, th_ref, phi_ref, na_ref), = _track_both(m, o, depth, gt)
    assert np.abs(g["theta"] - th_ref).max() < 1e-3
    _assert_offsets_close(g["offsets"], phi_ref)

