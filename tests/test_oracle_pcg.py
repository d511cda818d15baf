"""Pins of the oracle's coupled shape step (reading R22: the damped Gauss-Newton system of the whole shape
energy of Sec. 4.3, solved by block-Jacobi-preconditioned conjugate gradients)."""
import numpy as np

import oracle
from paper_1711_07999_gb300 import synth


def _setup(V=300, seed=5, **over):
    m = synth.make_model(1, V=V, width=64, **over)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0)), 1, np.random.default_rng(seed))
    phi = np.random.default_rng(seed + 1).normal(0, 0.002, (o.V, 3))
    P = o.pass_at(gt, phi, depth)
    return m, o, gt, phi, P


def _step(m, o, gt, phi, P, solver, iters, **over):
    m = dict(m, params=dict(m["params"], shape_solver=solver, shape_sweeps=iters, **over))
    o2 = oracle.Oracle(m)
    return o2.shape_step(gt, phi, P["n"], P["acc"], P["cnt"], P["inA"])


def _model_q(phi, r, g, inA, nbr, lp, lN):
    """The quadratic model of the shape energy (Sec. 4.3) with r_i linearised, written from the energy's
    terms: q(d) = sum_A (r_i + g_i.d_i)^2 + lp sum |phi_i + d_i|^2 + lN sum_i sum_{n in N(i)} |.|^2."""
    A = inA.astype(bool)
    src = np.repeat(np.arange(len(phi)), nbr.shape[1])
    dst = nbr.ravel()
    ok = dst >= 0
    src, dst = src[ok], dst[ok]

    def q(d):
        d = d.reshape(-1, 3)
        res = r[A] + (g[A] * d[A]).sum(1)
        y = phi + d
        e = y[src] - y[dst]
        return (res ** 2).sum() + lp * (y ** 2).sum() + lN * (e ** 2).sum()
    return q


def test_without_smoothness_one_pcg_iteration_is_the_per_vertex_solve():
    # lambda_N = 0 decouples the vertices: the block-Jacobi preconditioner is the exact inverse, so one
    # PCG iteration lands on the per-vertex damped solve that the Jacobi step (R15) computes.
    m, o, gt, phi, P = _setup(lambda_N=0.0)
    _, phi_cg, _, _ = _step(m, o, gt, phi, P, 1, 1)
    _, phi_j, _, _ = _step(m, o, gt, phi, P, 0, 1)
    assert np.abs(phi_cg - phi_j).max() < 1e-12


def test_converged_pcg_minimises_the_quadratic_model():
    # lambda_w = 0: the coupled step is the minimiser of the energy's quadratic model; its gradient, by
    # central differences of the model written from the energy's terms, vanishes there.
    m, o, gt, phi, P = _setup(lambda_w=0.0)
    _, phi1, r, g = _step(m, o, gt, phi, P, 1, 4 * o.V)
    _, _, nbr = o.derived()
    q = _model_q(phi, r, g, P["inA"], nbr, m["params"]["lambda_phi"], m["params"]["lambda_N"])
    x = (phi1 - phi).ravel()
    h = 1e-7

    def grad(x0, idx):
        out = np.empty(len(idx))
        for k, j in enumerate(idx):
            e = np.zeros_like(x0); e[j] = h
            out[k] = (q(x0 + e) - q(x0 - e)) / (2 * h)
        return out
    idx = np.arange(0, x.size, 7)
    g0 = grad(np.zeros_like(x), idx)
    g1 = grad(x, idx)
    assert np.abs(g1).max() < 1e-6 * np.abs(g0).max()
    assert q(x) < q(np.zeros_like(x))


def test_each_pcg_iteration_lowers_the_quadratic_model():
    # conjugate gradients decrease the (damped) quadratic model monotonically; with lambda_w = 0 that is
    # the energy's own quadratic model
    m, o, gt, phi, P = _setup(lambda_w=0.0)
    _, _, nbr = o.derived()
    qs = []
    for it in (1, 2, 4, 8, 16):
        _, phi1, r, g = _step(m, o, gt, phi, P, 1, it)
        q = _model_q(phi, r, g, P["inA"], nbr, m["params"]["lambda_phi"], m["params"]["lambda_N"])
        qs.append(q((phi1 - phi).ravel()))
    assert all(b < a for a, b in zip(qs, qs[1:])), qs


def test_energy_returned_is_the_same_for_both_solvers():
    m, o, gt, phi, P = _setup()
    E0, _, r0, g0 = _step(m, o, gt, phi, P, 0, 1)
    E1, _, r1, g1 = _step(m, o, gt, phi, P, 1, 5)
    assert E0 == E1 and np.array_equal(r0, r1) and np.array_equal(g0, g1)


def _damped_system(phi, r, g, inA, nbr, lp, lN, lw):
    """The coupled damped system of R22 assembled from the energy's terms: H = data blocks g g^T on A
    + lp I + lN (graph Laplacian of the neighbourhood edges, each directed edge once per direction),
    A = H + lw diag(H), right-hand side -b with b = [A] g r + lp phi + lN L phi."""
    V = len(phi)
    Hm = lp * np.eye(3 * V)
    for i in np.nonzero(inA)[0]:
        Hm[3 * i:3 * i + 3, 3 * i:3 * i + 3] += np.outer(g[i], g[i])
    Lap = np.zeros((V, V))
    for i in range(V):
        for q in nbr[i]:
            if q < 0:
                continue
            Lap[i, i] += 1; Lap[q, q] += 1; Lap[i, q] -= 1; Lap[q, i] -= 1
    Hm += lN * np.kron(Lap, np.eye(3))
    b = lp * phi.ravel() + lN * (np.kron(Lap, np.eye(3)) @ phi.ravel())
    b[np.repeat(inA.astype(bool), 3)] += (g * r[:, None])[inA.astype(bool)].ravel()
    return Hm + lw * np.diag(np.diag(Hm)), -b


def test_pcg_iterate_minimises_over_the_krylov_subspace():
    # After k iterations from 0, preconditioned CG minimises the A-norm error over the Krylov subspace
    # span{M^-1 c, (M^-1 A) M^-1 c, ...} (M the 3x3 diagonal blocks of A, c the right-hand side);
    # the minimiser there is Q (Q^T A Q)^-1 Q^T c for an orthonormal basis Q of the subspace.
    m, o, gt, phi, P = _setup(V=150)
    _, _, r, g = _step(m, o, gt, phi, P, 1, 1)
    _, _, nbr = o.derived()
    p = m["params"]
    A, c = _damped_system(phi, r, g, P["inA"], nbr, p["lambda_phi"], p["lambda_N"], p["lambda_w"])
    Minv = np.zeros_like(A)
    for i in range(o.V):
        Minv[3 * i:3 * i + 3, 3 * i:3 * i + 3] = np.linalg.inv(A[3 * i:3 * i + 3, 3 * i:3 * i + 3])
    for k in (1, 2, 3):
        u = [Minv @ c]
        for _ in range(k - 1):
            u.append(Minv @ (A @ u[-1]))
        Q, _ = np.linalg.qr(np.stack(u, 1))
        x = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ c)
        _, phik, _, _ = _step(m, o, gt, phi, P, 1, k)
        assert np.abs((phik - phi).ravel() - x).max() <= 1e-9 * np.abs(x).max(), k

