"""Pins of the oracle's kinematics and skinning (Sec. 3.1 forward kinematics, Eqs. H_hinge, H_prismatic,
H_Sigma, skin, deformation) against textbook 4x4 matrix chains and the special cases the paper fixes."""
import math

import numpy as np
import pytest

import oracle
from tests import helpers as H


def _tree_model(rng, L=6, V=None):
    parent, jtype, axis, offs = H.random_tree(rng, L)
    # one vertex per link, fully weighted to it, plus a few blended vertices
    verts, bidx, bw = [], [], []
    for j in range(L):
        verts.append(rng.uniform(-0.3, 0.3, 3) + [0, 0, 2.0])
        bidx.append([j, 0, 0, 0]); bw.append([1, 0, 0, 0])
    tris = [[0, 1, 2]]
    m = H.make_model(parent, jtype, axis, offs, verts, tris, bidx, bw)
    ax = np.asarray(m["skeleton"]["axis"], np.float64)
    ax = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    return m, parent, jtype, ax, [np.asarray(o, np.float64) for o in m["skeleton"]["offset_dq"][:, 5:] * 2]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fk_equals_homogeneous_matrix_chain(seed):
    rng = np.random.default_rng(seed)
    m, parent, jtype, axis, offs = _tree_model(rng, L=7)
    o = oracle.Oracle(m)
    theta = rng.uniform(-1.5, 1.5, o.L)
    H0, Hd = o.fk(theta)
    Ms = H.chain_matrices(parent, jtype, axis, offs, theta)
    M0 = H.chain_matrices(parent, jtype, axis, offs, np.zeros(o.L))
    for j in range(o.L):
        assert np.allclose(H.dq_to_matrix(H0[j]), Ms[j], atol=1e-12)
        # H_{j,Delta} = H_{0,j} (H^0_{0,j})^{-1}
        assert np.allclose(H.dq_to_matrix(Hd[j]), Ms[j] @ np.linalg.inv(M0[j]), atol=1e-12)


def test_bind_pose_offsets_are_identity():
    rng = np.random.default_rng(3)
    m, *_ = _tree_model(rng, L=5)
    o = oracle.Oracle(m)
    _, Hd = o.fk(np.zeros(o.L))
    ident = np.array([1, 0, 0, 0, 0, 0, 0, 0], float)
    assert np.allclose(Hd, ident[None], atol=1e-15)


@pytest.mark.parametrize("seed", [4, 5])
def test_single_bone_vertices_move_rigidly(seed):
    rng = np.random.default_rng(seed)
    m, parent, jtype, axis, offs = _tree_model(rng, L=6)
    o = oracle.Oracle(m)
    theta = rng.uniform(-2.0, 2.0, o.L)
    phi = rng.normal(0, 0.01, (o.V, 3))
    v, _ = o.skin(theta, phi)
    Ms = H.chain_matrices(parent, jtype, axis, offs, theta)
    M0 = H.chain_matrices(parent, jtype, axis, offs, np.zeros(o.L))
    x = m["mesh"]["verts"].astype(np.float64) + phi
    for i in range(o.V):
        j = int(m["mesh"]["bone_idx"][i, 0])
        D = Ms[j] @ np.linalg.inv(M0[j])
        assert np.allclose(v[i], D[:3, :3] @ x[i] + D[:3, 3], atol=1e-12)


def test_bind_pose_gives_template_plus_offsets():
    m = __import__("paper_1711_07999_gb300.synth", fromlist=["x"]).make_model(1)
    o = oracle.Oracle(m)
    phi = np.random.default_rng(0).normal(0, 0.003, (o.V, 3))
    v, _ = o.skin(np.zeros(o.L), phi)
    assert np.abs(v - (m["mesh"]["verts"].astype(np.float64) + phi)).max() < 1e-14


def _two_link(theta_child_extra=0.0):
    parent, jtype = [-1, 0], [0, 0]
    axis = [[0, 0, 1], [1, 0, 0]]
    offs = [[0, 0, 2.0], [0.2, 0, 0]]
    verts = [[0.1, 0.05, 2.0], [0.3, -0.05, 2.1], [0.2, 0.1, 1.95]]
    bidx = [[0, 1, 0, 0]] * 3
    bw = [[0.5, 0.5, 0, 0]] * 3
    return H.make_model(parent, jtype, axis, offs, verts, [[0, 1, 2]], bidx, bw), parent, jtype, axis, offs


def test_equal_bone_transforms_blend_to_that_transform():
    # child at theta = 0 has the same H_Delta as its parent; a 50/50 vertex then moves rigidly with it
    m, parent, jtype, axis, offs = _two_link()
    o = oracle.Oracle(m)
    th = np.array([0.7, 0.0])
    v, Hs = o.skin(th)
    M = H.chain_matrices(parent, jtype, axis, offs, th)[0] @ np.linalg.inv(H.chain_matrices(parent, jtype, axis, offs, [0, 0])[0])
    x = m["mesh"]["verts"].astype(np.float64)
    assert np.allclose(v, x @ M[:3, :3].T + M[:3, 3], atol=1e-12)


def test_antipodal_bone_is_sign_aligned():
    # a hinge at 2*pi is the identity rotation but its dual quaternion has the opposite sign; without
    # the alignment of R1 the blend would cancel.  The blend must equal the theta = 0 result.
    m, *_ = _two_link()
    o = oracle.Oracle(m)
    va, _ = o.skin(np.array([0.4, 0.0]))
    vb, Hs = o.skin(np.array([0.4, 2 * math.pi]))
    assert np.allclose(va, vb, atol=1e-12)
    _, Hd = o.fk(np.array([0.4, 2 * math.pi]))
    assert np.dot(Hd[0, :4], Hd[1, :4]) < 0  # the raw bone DQs are antipodal


def test_point_map_is_scale_invariant():
    # T(c H, x) = T(H, x): two bones with equal transforms and weights 0.3/0.7 give the rigid map
    parent, jtype = [-1, 0], [0, 1]
    axis = [[0, 1, 0], [0, 0, 1]]
    offs = [[0, 0, 2.0], [0, 0, 0]]
    verts = [[0.1, 0.05, 2.0], [0.3, -0.05, 2.1], [0.2, 0.1, 1.95]]
    m = H.make_model(parent, jtype, axis, offs, verts, [[0, 1, 2]], [[0, 1, 0, 0]] * 3, [[0.3, 0.7, 0, 0]] * 3)
    o = oracle.Oracle(m)
    v, Hs = o.skin(np.array([0.9, 0.0]))
    R = H.rot_matrix([0, 1, 0], 0.9)
    c = np.array([0, 0, 2.0])
    x = m["mesh"]["verts"].astype(np.float64)
    assert np.allclose(v, (x - c) @ R.T + c, atol=1e-12)


def test_blend_of_coaxial_rotations_turns_by_the_blended_half_angle():
    # Bones 0 and 1 turn about the same axis line (y through (0, 0, 2); link 1 has no offset) by 0.9 and
    # 0.9 - 1.2 = -0.3 rad.  Blended with weights 0.3 / 0.7 the dual quaternion is not unit (|a|^2 = 0.93);
    # the point map of R2 then gives the rotation about that line by phi, tan(phi / 2) =
    # (0.3 sin 0.45 + 0.7 sin -0.15) / (0.3 cos 0.45 + 0.7 cos -0.15) (the blend of coaxial rotations).
    parent, jtype = [-1, 0], [0, 0]
    axis = [[0, 1, 0], [0, 1, 0]]
    offs = [[0, 0, 2.0], [0, 0, 0]]
    verts = [[0.1, 0.05, 2.0], [0.3, -0.05, 2.1], [0.2, 0.1, 1.95]]
    m = H.make_model(parent, jtype, axis, offs, verts, [[0, 1, 2]], [[0, 1, 0, 0]] * 3, [[0.3, 0.7, 0, 0]] * 3)
    o = oracle.Oracle(m)
    v, _ = o.skin(np.array([0.9, -1.2]))
    h1, h2 = 0.45, -0.15
    phi = 2 * math.atan2(0.3 * math.sin(h1) + 0.7 * math.sin(h2), 0.3 * math.cos(h1) + 0.7 * math.cos(h2))
    R = H.rot_matrix([0, 1, 0], phi)
    c = np.array([0, 0, 2.0])
    x = m["mesh"]["verts"].astype(np.float64)
    assert np.allclose(v, (x - c) @ R.T + c, atol=1e-12)

