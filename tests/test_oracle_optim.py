"""Pins of the oracle's residual (Eq. residual), pose Jacobian (Sec. 4.2 chain rule, R12), normal
equations (Eqs. JTJ, JTr, prior), damped least squares (R13, R14), shape step (Eq. r_warp, R15) and the
frame schedule, against finite differences, explicit products, closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth
from tests import helpers as H


def _scene(cfg=1, V=2000, width=96, pert_deg=2.0, seed=0, phi_scale=0.5):
    m = synth.make_model(cfg, V=V, width=width)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    phi = synth.gt_offsets(m, 0.0)
    z = o.render(gt, phi)
    depth = synth.add_noise(z, 1, np.random.default_rng(seed))
    rng = np.random.default_rng(seed + 100)
    th = gt + np.radians(pert_deg) * rng.normal(size=o.L) * (m["skeleton"]["type"] == 0)
    return m, o, gt, phi * phi_scale, depth, th


def test_jacobian_matches_central_differences():
    m, o, gt, phi, depth, th = _scene()
    P = o.pass_at(th, phi, depth)
    J = o.jacobian(th, phi, P["n"], P["inA"])
    A = P["inA"] > 0
    assert A.sum() > 100
    pt = P["v"] + np.where(A[:, None], P["acc"] / np.maximum(P["cnt"], 1)[:, None], 0)

    def r_of(t):  # association, normals and p~ held fixed
        v, _ = o.skin(t, phi)
        return np.einsum("ij,ij->i", P["n"], pt - v)

    h = 1e-6
    for k in range(o.L):
        e = np.zeros(o.L)
        e[k] = h
        fd = (r_of(th + e) - r_of(th - e)) / (2 * h)
        err = np.abs(J[A, k] - fd[A]).max()
        assert err <= 1e-6 * max(1.0, np.abs(fd[A]).max()), (k, err)
    assert np.allclose(r_of(th)[A], P["r"][A], atol=1e-14)


def test_normal_equations_equal_explicit_products():
    m, o, gt, phi, depth, th = _scene(V=1200, width=80)
    P = o.pass_at(th, phi, depth)
    J = o.jacobian(th, phi, P["n"], P["inA"])
    JTJ, JTr = oracle.normal_eq(J, P["r"], P["inA"])
    A = P["inA"] > 0
    assert np.allclose(JTJ, J[A].T @ J[A], rtol=1e-12, atol=1e-14)
    assert np.allclose(JTr, J[A].T @ P["r"][A], rtol=1e-12, atol=1e-14)


def test_cholesky_solve_equals_gaussian_elimination():
    rng = np.random.default_rng(1)
    for n in (1, 5, 40, 72):
        B = rng.normal(size=(n, n))
        M = B @ B.T + n * np.eye(n)
        b = rng.normal(size=n)
        assert np.allclose(oracle.cholesky_solve(M, b), np.linalg.solve(M, b), rtol=1e-11, atol=1e-13)
    assert oracle.cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2)) is None


def test_solve3_equals_gaussian_elimination():
    rng = np.random.default_rng(2)
    for _ in range(20):
        M = rng.normal(size=(3, 3))
        b = rng.normal(size=3)
        assert np.allclose(oracle.solve3(M, b), np.linalg.solve(M, b), rtol=1e-10)


def test_planar_patch_at_its_own_pose_has_zero_residual():
    V, T = H.grid_patch(25, 25, -0.3, 0.3, -0.3, 0.3, 2.0)
    n = len(V)
    m = H.make_model([-1, 0, 0], [1, 0, 0], [[1, 0, 0], [0, 1, 0], [1, 0, 0]], [[0, 0, 0]] * 3, V, T,
                     [[1, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n, W=64, H=64, fx=90.0, fy=90.0, window_half=3)
    o = oracle.Oracle(m)
    th = np.zeros(3)
    depth = o.render(th).astype(np.float32)
    P = o.pass_at(th, None, depth)
    A = P["inA"] > 0
    assert A.sum() > 300
    assert np.abs(P["r"][A]).max() < 1e-6  # only the float32 storage of the depth remains


def test_gauss_newton_step_from_truth_is_negligible():
    # a planar patch on the 6-DoF root, rendered noise-free at its own pose: J^T r = 0 and the
    # (minimum-norm) Gauss-Newton step vanishes
    V, T = H.grid_patch(21, 21, -0.3, 0.3, -0.25, 0.25, 2.0)
    n = len(V)
    axes = [[1, 0, 0], [0, 1, 0], [0, 0, 1]] * 2
    m = H.make_model([-1, 0, 1, 2, 3, 4], [1, 1, 1, 0, 0, 0], axes, [[0, 0, 2.0]] + [[0, 0, 0]] * 5, V, T,
                     [[5, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n, W=80, H=64, fx=90.0, fy=90.0, window_half=3,
                     prior_mask=[0] * 6)
    o = oracle.Oracle(m)
    th = np.array([0.01, -0.02, 0.1, 0.2, -0.15, 0.05])
    depth = o.render(th).astype(np.float32)
    P = o.pass_at(th, None, depth)
    J = o.jacobian(th, None, P["n"], P["inA"])
    A = P["inA"] > 0
    x = np.linalg.lstsq(J[A], P["r"][A], rcond=1e-10)[0]
    assert np.abs(J[A].T @ P["r"][A]).max() < 1e-5 * np.sqrt((J[A] ** 2).sum())
    assert np.abs(x).max() < 1e-5


def test_residual_at_truth_is_bounded_by_the_sagitta():
    # curved capsules rendered at their own pose: the pixels lie on chords of the surface, so r_i is
    # bounded by the sagitta h^2 / (8 r) of the tessellation and biased inward (negative)
    m = synth.make_model(1, V=3000, width=160)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    depth = o.render(gt).astype(np.float32)
    P = o.pass_at(gt, None, depth)
    A = P["inA"] > 0
    v0 = m["mesh"]["verts"].astype(np.float64)
    tri = m["mesh"]["tris"]
    h = max(np.linalg.norm(v0[tri[:, 0]] - v0[tri[:, 1]], axis=1).max(),
            np.linalg.norm(v0[tri[:, 1]] - v0[tri[:, 2]], axis=1).max())
    rmin = min(b["radius"] for b in m["bones"])
    assert np.abs(P["r"][A]).max() <= h * h / (8 * rmin) * 4 + 1e-6
    assert np.median(P["r"][A]) < 0


def test_energy_invariant_under_global_rigid_motion():
    m, o, gt, phi, depth, th = _scene(V=1500, width=80)
    P = o.pass_at(th, phi, depth)
    # move the whole model by G (rotation Rg, translation tg) through the root's fixed offset
    Rg = H.rot_matrix([0.3, -0.5, 0.8], 0.4)
    tg = np.array([0.05, -0.02, 0.1])
    w, x, y, z = _rot_to_quat(Rg)
    m2 = {k: (dict(v) if isinstance(v, dict) else v) for k, v in m.items()}
    sk = dict(m["skeleton"])
    off = np.array(sk["offset_dq"], np.float64)
    G = np.array([w, x, y, z, *(_qmul([0, *tg], [w, x, y, z]) * 0.5)])
    off[0] = _dqmul(G, off[0])
    sk["offset_dq"] = off.astype(np.float32)
    m2["skeleton"] = sk
    me = dict(m["mesh"])  # the template (bind pose, world frame) moves with the skeleton
    me["verts"] = (me["verts"].astype(np.float64) @ Rg.T + tg).astype(np.float32)
    m2["mesh"] = me
    o2 = oracle.Oracle(m2)
    v2, _ = o2.skin(th, phi @ Rg.T)
    # skinning is equivariant: v2 = G v (up to the float32 storage of the moved offset)
    assert np.abs(v2 - (P["v"] @ Rg.T + tg)).max() < 1e-6
    n2, ok2 = o2.normals(v2)
    assert np.allclose(n2[ok2 > 0], (P["n"] @ Rg.T)[ok2 > 0], atol=1e-4)  # float32 template storage
    acc2 = P["acc"] @ Rg.T  # the same association, data moved with the model
    r2, inA2, E2 = o2.residuals(th, n2, ok2, acc2, P["cnt"])
    assert np.array_equal(inA2, P["inA"])
    assert E2 == pytest.approx(P["E"], rel=1e-4)


def _qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


def _dqmul(A, B):
    return np.concatenate([_qmul(A[:4], B[:4]), _qmul(A[:4], B[4:]) + _qmul(A[4:], B[:4])])


def _rot_to_quat(R):
    w = math.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    return w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)


def test_lm_accepts_only_descent_and_updates_lambda():
    m, o, gt, phi, depth, th = _scene(V=1500, width=96, pert_deg=4)
    o.set_state(th, phi)
    P = o.pass_at(th, phi, depth)
    J = o.jacobian(th, phi, P["n"], P["inA"])
    JTJ, JTr = oracle.normal_eq(J, P["r"], P["inA"])
    lam0 = 1e-3
    a, th1, lam1, Ec = o.lm_step(JTJ, JTr, P["E"], P["v"], P["n"], P["acc"], P["cnt"], P["inA"], th, lam0)
    assert a >= 0 and Ec[a] <= P["E"]
    assert all(Ec[t] > P["E"] for t in range(a))
    assert lam1 == pytest.approx(max(lam0 * 10 ** a / 10, 1e-7))
    # the accepted step solves the damped, prior-augmented system of R13
    _, S, _ = o.derived()
    s2 = (m["params"]["lambda_s"] * S) ** 2
    A_ = JTJ + np.diag(s2)
    x = np.linalg.solve(A_ + lam0 * 10 ** a * np.diag(np.diag(A_)), JTr + s2 * th)
    assert np.allclose(th1, th - x, atol=1e-10)
    # an energy nothing can beat forces every attempt to be rejected
    a2, th2, lam2, Ec2 = o.lm_step(JTJ, JTr, -1.0, P["v"], P["n"], P["acc"], P["cnt"], P["inA"], th, lam0)
    assert a2 == -1 and np.array_equal(th2, th) and lam2 == pytest.approx(lam0 * 1e6)


def test_lm_lambda_stays_within_its_bounds():
    # R14: lambda is clamped to [1e-7, 1e7]: a step accepted at once from 1e-7 keeps 1e-7, six rejections
    # from 1e6 stop at 1e7
    m, o, gt, phi, depth, th = _scene(V=1500, width=96, pert_deg=4)
    P = o.pass_at(th, phi, depth)
    J = o.jacobian(th, phi, P["n"], P["inA"])
    JTJ, JTr = oracle.normal_eq(J, P["r"], P["inA"])
    a, _, lam1, _ = o.lm_step(JTJ, JTr, P["E"], P["v"], P["n"], P["acc"], P["cnt"], P["inA"], th, 1e-7)
    assert a == 0 and lam1 == 1e-7
    a2, _, lam2, _ = o.lm_step(JTJ, JTr, -1.0, P["v"], P["n"], P["acc"], P["cnt"], P["inA"], th, 1e6)
    assert a2 == -1 and lam2 == 1e7


def test_single_rigid_link_converges_to_truth():
    # one capsule on the 6-DoF root: point-to-plane Gauss-Newton on noise-free data
    # two capsules in an L, both on the root's last link: a rigid body with no symmetry axis
    bones = [synth._bone("b", -1, (0, 0, 0), (-0.15, 0.0, 0.0), (0.15, 0.05, 0.02), 0.08, synth.ROOT_DOFS),
             synth._bone("c", 0, (0.15, 0, 0), (0.15, 0.05, 0.0), (0.2, 0.3, -0.05), 0.05, [("h", synth.X)])]
    sk, lob, fl = synth.build_skeleton(bones[:1], (0, 0, 2.0))
    verts, tris, n0, bo = synth.tessellate(bones, (0, 0, 2.0), 1500)
    nV = len(verts)
    m = dict(skeleton=sk, mesh=dict(verts=verts.astype(np.float32), tris=tris.astype(np.int32),
                                    bone_idx=np.array([[5, 0, 0, 0]] * nV, np.uint8),
                                    bone_w=np.array([[1, 0, 0, 0]] * nV, np.float32)),
             camera=dict(width=120, height=90, fx=120.0, fy=120.0, cx=60.0, cy=45.0),
             params=synth.default_params(120.0, nV, pose_iters=15, shape_iters=0))
    o = oracle.Oracle(m)
    gt = np.array([0.01, -0.02, 0.015, 0.05, -0.04, 0.03])
    depth = o.render(gt).astype(np.float32)
    o.set_state(np.zeros(6), None)
    e, acc, na = o.track_frame(depth)
    th, _, _ = o.get_state()
    # converges to the truth up to the tessellation's chord bias (the pixels lie on chords) ...
    assert np.abs(th - gt).max() < 5e-3
    assert e[-1] < 1e-2 * e[0]
    # ... and the result is a fixed point of the iteration
    o.track_frame(depth)
    th2, _, _ = o.get_state()
    assert np.abs(th2 - th).max() < 1e-5


def test_shape_step_special_cases():
    V, T = H.grid_patch(8, 8, -0.2, 0.2, -0.2, 0.2, 2.0)
    n = len(V)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, T, [[0, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n,
                     W=40, H=40, fx=60.0, fy=60.0, window_half=3)
    o = oracle.Oracle(m)
    th = np.zeros(1)
    depth = o.render(th).astype(np.float32)
    P = o.pass_at(th, None, depth)
    # undisplaced flat patch at its own pose: zero Laplacian, zero update
    E, phi1, r, g = o.shape_step(th, np.zeros((n, 3)), P["n"], P["acc"], P["cnt"], P["inA"])
    assert np.abs(phi1).max() < 1e-6 and E < 1e-10
    # constant offsets with lambda_phi = 0: the smoothness gradient vanishes; an unassociated vertex stays
    m2 = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, T, [[0, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n,
                      W=40, H=40, fx=60.0, fy=60.0, window_half=3, lambda_phi=0.0)
    o2 = oracle.Oracle(m2)
    c = np.tile([0.001, -0.002, 0.0005], (n, 1))
    noA = np.zeros(n, np.int32)
    E2, phi2, _, _ = o2.shape_step(th, c, P["n"], P["acc"], P["cnt"], noA)
    assert np.allclose(phi2, c, atol=1e-15)


def test_shape_step_closed_form_without_smoothness():
    # lambda_N = 0: each vertex solves (M + lw diag M) d = -(g r + lp phi) with M = g g^T + lp I
    m = synth.make_model(1, V=1200, width=96)
    m["params"]["lambda_N"] = 0.0
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0)
    phi_gt = synth.gt_offsets(m, 0)
    depth = synth.add_noise(o.render(gt, phi_gt), 1, np.random.default_rng(3))
    phi = np.random.default_rng(4).normal(0, 0.002, (o.V, 3))
    P = o.pass_at(gt, phi, depth)
    E, phi1, r, g = o.shape_step(gt, phi, P["n"], P["acc"], P["cnt"], P["inA"])
    lp, lw = m["params"]["lambda_phi"], m["params"]["lambda_w"]
    for i in range(0, o.V, 11):
        gi = g[i]
        ri = r[i]
        Mx = np.outer(gi, gi) + lp * np.eye(3)
        Md = Mx + lw * np.diag(np.diag(Mx))
        d = -np.linalg.solve(Md, gi * ri + lp * phi[i])
        assert np.allclose(phi1[i], phi[i] + d, atol=1e-13)
    # g_i = dr_i/dphi_i by central differences on the skinning, p~ and n fixed
    A = np.nonzero(P["inA"])[0]
    pt = P["v"] + P["acc"] / np.maximum(P["cnt"], 1)[:, None]
    h = 1e-6
    for i in A[::23]:
        fd = np.zeros(3)
        for c in range(3):
            ph = phi.copy(); ph[i, c] += h
            vp, _ = o.skin(gt, ph)
            ph[i, c] -= 2 * h
            vm, _ = o.skin(gt, ph)
            fd[c] = (P["n"][i] @ (pt[i] - vp[i]) - P["n"][i] @ (pt[i] - vm[i])) / (2 * h)
        assert np.allclose(fd, g[i], atol=1e-8)


def _planar_root_model(**params):
    # a plane observes its own out-of-plane motion only: depth translation and tilts about x and y
    V, T = H.grid_patch(21, 21, -0.3, 0.3, -0.25, 0.25, 2.0)
    n = len(V)
    return H.make_model([-1, 0, 1], [1, 0, 0], [[0, 0, 1], [1, 0, 0], [0, 1, 0]], [[0, 0, 2.0]] + [[0, 0, 0]] * 2,
                        V, T, [[2, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n, W=80, H=64, fx=90.0, fy=90.0, window_half=3,
                        prior_mask=[0] * 3, **params)


def test_frame_at_own_pose_stays_put():
    # a planar patch rendered noise-free at its own pose: every residual is zero (up to the float32
    # depth), so neither the pose iterations nor the shape iterations move anything
    m = _planar_root_model()
    o = oracle.Oracle(m)
    th0 = np.array([0.1, 0.2, -0.15])
    depth = o.render(th0).astype(np.float32)
    o.set_state(th0, None)
    e, acc, na = o.track_frame(depth)
    th, phi, lam = o.get_state()
    assert na > 500
    assert np.abs(th - th0).max() < 1e-5
    assert np.abs(phi).max() < 1e-6
    assert max(e) < 1e-9


def test_frame_from_perturbed_start_reduces_energy():
    m = synth.make_model(1)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0.0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0.0)), 1, np.random.default_rng(0))
    o.set_state(synth.start_theta(m), None)
    e, acc, na = o.track_frame(depth)
    assert e[m["params"]["pose_iters"] - 1] < 0.6 * e[0]


def test_residual_averages_the_points_a_vertex_collects():
    # Eq. residual with p~_i the mean of the back-projected points assigned to vertex i: a coarse patch
    # (vertices 0.1 m apart) seen at ~5 px per vertex spacing collects ~25 pixels per vertex; the depth is
    # a tilted plane in front of it, so the residuals differ from vertex to vertex
    V, T = H.grid_patch(5, 5, -0.2, 0.2, -0.2, 0.2, 2.0)
    n = len(V)
    W = Hh = 64
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, T, [[0, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n,
                     W=W, H=Hh, fx=100.0, fy=100.0, window_half=4, cutoff=0.1)
    o = oracle.Oracle(m)
    fx, fy, cx, cy = (m["camera"][k] for k in ("fx", "fy", "cx", "cy"))
    ys, xs = np.mgrid[0:Hh, 0:W]
    depth = (2.02 + 0.1 * (xs - cx) / W + 0.05 * (ys - cy) / Hh).astype(np.float32)
    P = o.pass_at(np.zeros(1), None, depth)
    assert P["cnt"].max() >= 16
    sums = np.zeros((n, 3))
    cnt = np.zeros(n, np.int64)
    for py, px in zip(*np.nonzero(P["corr"] >= 0)):
        d = float(depth[py, px])
        i = P["corr"][py, px]
        sums[i] += [(px - cx) * d / fx, (py - cy) * d / fy, d]
        cnt[i] += 1
    A = cnt > 0
    r = np.zeros(n)
    r[A] = (P["n"][A] * (sums[A] / cnt[A, None] - P["v"][A])).sum(1)
    assert np.array_equal(P["inA"].astype(bool), A & P["nvalid"].astype(bool))
    assert np.allclose(P["r"], r, rtol=0, atol=1e-12)
    assert abs(P["E"] - (r ** 2).sum()) <= 1e-12 * (r ** 2).sum()


def test_smoothness_alone_moves_each_offset_to_its_neighbours_mean():
    # Sec. 4.3 with no data term (no associated vertex), lambda_phi = lambda_w = 0: a vertex's energy is
    # lambda_N sum_{n in N(i)} |phi_i - phi_n|^2 with the neighbours frozen, minimised at their mean; one
    # Jacobi sweep moves every vertex there at once
    V, T = H.grid_patch(6, 6, -0.2, 0.2, -0.2, 0.2, 2.0)
    n = len(V)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, T, [[0, 0, 0, 0]] * n, [[1, 0, 0, 0]] * n,
                     W=40, H=40, fx=60.0, fy=60.0, window_half=3, lambda_phi=0.0, lambda_w=0.0, shape_sweeps=1)
    o = oracle.Oracle(m)
    _, _, nbr = o.derived()
    phi = np.random.default_rng(9).normal(0, 0.003, (n, 3))
    zeros3 = np.zeros((n, 3))
    E, phi1, _, _ = o.shape_step(np.zeros(1), phi, zeros3, zeros3, np.zeros(n, np.int32), np.zeros(n, np.int32))
    assert np.allclose(phi1, phi[nbr].mean(axis=1), rtol=0, atol=1e-15)
    lN = m["params"]["lambda_N"]
    assert abs(E - lN * ((phi[:, None, :] - phi[nbr]) ** 2).sum()) <= 1e-12 * E


def test_energy_without_data_is_the_pose_prior():
    # no depth pixel: A is empty and E_pose = sum_k (lambda_s S_kk theta_k)^2 (Sec. 4.2 pose prior, R10)
    m = synth.make_model(1, V=800, width=48)
    o = oracle.Oracle(m)
    th = synth.start_theta(m) + 0.1
    P = o.pass_at(th, None, np.zeros((o.H, o.W), np.float32))
    assert not P["inA"].any()
    _, S, _ = o.derived()
    prior = ((m["params"]["lambda_s"] * S * th) ** 2).sum()
    assert prior > 0 and abs(P["E"] - prior) <= 1e-14 * prior


def test_jacobian_matches_central_differences_across_an_antipodal_bone():
    # R1: the child's hinge at 2 pi + 0.3 has a dual quaternion of the opposite sign to its parent's; the
    # blend and its derivative both carry the alignment sign, so the Jacobian still equals the central
    # differences of r_i = n_i.(p~_i - v_i(Theta)) (n, p~ fixed)
    parent, jtype = [-1, 0], [0, 0]
    axis, offs = [[0, 0, 1], [1, 0, 0]], [[0, 0, 2.0], [0.2, 0, 0]]
    verts = [[0.1, 0.05, 2.0], [0.3, -0.05, 2.1], [0.2, 0.1, 1.95]]
    m = H.make_model(parent, jtype, axis, offs, verts, [[0, 1, 2]], [[0, 1, 0, 0]] * 3, [[0.4, 0.6, 0, 0]] * 3)
    o = oracle.Oracle(m)
    th = np.array([0.4, 2 * math.pi + 0.3])
    _, Hd = o.fk(th)
    assert np.dot(Hd[0, :4], Hd[1, :4]) < 0
    rng = np.random.default_rng(2)
    n = rng.normal(size=(3, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    pt = rng.normal(0, 0.05, (3, 3)) + [0.2, 0, 2.0]
    inA = np.ones(3, np.int32)
    J = o.jacobian(th, None, n, inA)

    def r_of(t):
        v, _ = o.skin(t)
        return np.einsum("ij,ij->i", n, pt - v)

    h = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (r_of(th + e) - r_of(th - e)) / (2 * h)
        assert np.abs(J[:, k] - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max()), k


def test_second_sweep_is_a_fixed_point_without_smoothness_and_damping():
    # lambda_N = lambda_w = 0: a vertex's linearised energy (r_i + g_i.(phi_i - phi0_i))^2 + lp |phi_i|^2 is
    # quadratic and one Gauss-Newton sweep lands on its minimiser; a second sweep, with r re-linearised at
    # the new offsets, finds a zero gradient there and does not move
    m = synth.make_model(1, V=1200, width=96)
    m["params"].update(lambda_N=0.0, lambda_w=0.0)
    one = oracle.Oracle(dict(m, params=dict(m["params"], shape_sweeps=1)))
    two = oracle.Oracle(dict(m, params=dict(m["params"], shape_sweeps=2)))
    gt = synth.gt_theta(m, 0)
    depth = synth.add_noise(one.render(gt, synth.gt_offsets(m, 0)), 1, np.random.default_rng(3))
    phi = np.random.default_rng(4).normal(0, 0.002, (one.V, 3))
    P = one.pass_at(gt, phi, depth)
    assert P["inA"].sum() > 100
    _, phi1, _, _ = one.shape_step(gt, phi, P["n"], P["acc"], P["cnt"], P["inA"])
    _, phi2, _, _ = two.shape_step(gt, phi, P["n"], P["acc"], P["cnt"], P["inA"])
    assert np.abs(phi1 - phi).max() > 1e-4
    # rounding of the second 3x3 solve (condition ~ 1 / lambda_phi = 100): ~1e-15 on offsets of ~1e-2
    assert np.allclose(phi2, phi1, rtol=0, atol=1e-13)


def test_frame_is_the_schedule_of_its_steps():
    # R18: a frame is pose_iters LM iterations, each re-associating at the current state (skin, normals,
    # z-buffer, visibility, association, residuals, Jacobian, normal equations, LM step), then shape_iters
    # shape iterations, each re-associating too.  The frame equals those steps called one by one: the
    # same energies, accepted attempts, Theta, Phi and lambda, bit for bit.
    m, _, gt, phi0, depth, th0 = _scene(V=1500, width=96, pert_deg=3)
    m = dict(m, params=dict(m["params"], pose_iters=3, shape_iters=1, shape_sweeps=1))
    frame, steps = oracle.Oracle(m), oracle.Oracle(m)
    lam0 = 1e-3
    frame.set_state(th0, phi0, lam0)
    steps.set_state(th0, phi0, lam0)
    th, lam, E_ref, acc_ref = th0.copy(), lam0, [], []
    for _ in range(3):
        P = steps.pass_at(th, phi0, depth)
        E_ref.append(P["E"])
        J = steps.jacobian(th, phi0, P["n"], P["inA"])
        JTJ, JTr = oracle.normal_eq(J, P["r"], P["inA"])
        a, th, lam, _ = steps.lm_step(JTJ, JTr, P["E"], P["v"], P["n"], P["acc"], P["cnt"], P["inA"], th, lam)
        acc_ref.append(a)
    P = steps.pass_at(th, phi0, depth)
    E_shape, phi1, _, _ = steps.shape_step(th, phi0, P["n"], P["acc"], P["cnt"], P["inA"])
    e, acc, n_assoc = frame.track_frame(depth)
    th_f, phi_f, lam_f = frame.get_state()
    assert list(acc) == acc_ref and max(acc_ref) >= 0
    assert list(e) == E_ref + [E_shape]
    assert np.array_equal(th_f, th) and np.array_equal(phi_f, phi1) and lam_f == lam
    assert n_assoc == int((P["corr"] >= 0).sum())

