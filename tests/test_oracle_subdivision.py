"""Pins of the oracle's Catmull-Clark subdivision (the template construction: two levels of subdivision
of a low-resolution cage, the skin weights interpolated with the same scheme as the positions)."""
import numpy as np
import pytest

import oracle


def _cube():
    v = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    idx = {tuple(p): i for i, p in enumerate(v.astype(int))}
    faces = []
    for ax in range(3):
        for s in (-1, 1):
            quad = []
            for a, b in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                p = [0, 0, 0]
                p[ax] = s
                p[(ax + 1) % 3] = a
                p[(ax + 2) % 3] = b
                quad.append(idx[tuple(p)])
            faces.append(quad if s > 0 else quad[::-1])
    fo = np.arange(0, 4 * len(faces) + 1, 4)
    return v, fo, np.array(faces).ravel()


def test_cube_closed_forms():
    v, fo, fv = _cube()
    out, quads = oracle.subdivide(fo, fv, v, 1)
    assert len(out) == 8 + 12 + 6 and len(quads) == 24
    # corner (valence 3): F = (1,1,1)/3, R = (2,2,2)/3 -> (F + 2R + 0 P)/3 = (5,5,5)/9
    corner = np.where((v == [1, 1, 1]).all(1))[0][0]
    assert np.allclose(out[corner], [5 / 9] * 3, atol=1e-15)
    # face points are the face centres; an edge point is (v0 + v1 + fa + fb)/4, e.g. (3/4, 3/4, 0)
    assert np.allclose(np.sort(np.abs(out[20:]).sum(1)), 1.0)
    e_pts = out[8:20]
    assert any(np.allclose(p, [0.75, 0.75, 0.0]) for p in e_pts)


def test_counts_and_euler_characteristic():
    v, fo, fv = _cube()
    for levels in (1, 2, 3):
        out, quads = oracle.subdivide(fo, fv, v, levels)
        E = len({tuple(sorted((q[i], q[(i + 1) % 4]))) for q in quads for i in range(4)})
        assert len(out) - E + len(quads) == 2  # sphere topology kept
        assert len(quads) == 6 * 4 ** levels


def test_regular_flat_grid_interior_is_fixed_and_planar():
    n = 6
    g = np.array([[x, y, 0.0] for y in range(n) for x in range(n)])
    faces = [[y * n + x, y * n + x + 1, (y + 1) * n + x + 1, (y + 1) * n + x] for y in range(n - 1) for x in range(n - 1)]
    fo = np.arange(0, 4 * len(faces) + 1, 4)
    out, quads = oracle.subdivide(fo, np.array(faces).ravel(), g, 2)
    assert np.abs(out[:, 2]).max() == 0.0
    # an interior vertex of a uniform flat grid stays where it is (F = R = P)
    for y in range(2, n - 2):
        for x in range(2, n - 2):
            assert np.allclose(out[y * n + x], g[y * n + x], atol=1e-14)


def test_attributes_follow_the_position_stencils():
    # "the same scheme": an attribute equal to a linear function of the position is reproduced exactly;
    # weights that sum to one still do
    v, fo, fv = _cube()
    rng = np.random.default_rng(0)
    w = rng.random((8, 5))
    w /= w.sum(1, keepdims=True)
    lin = v @ np.array([0.3, -1.2, 2.0]) + 0.7
    attr = np.hstack([v, lin[:, None], w])
    out, _ = oracle.subdivide(fo, fv, attr, 2)
    assert np.allclose(out[:, 3], out[:, :3] @ np.array([0.3, -1.2, 2.0]) + 0.7, atol=1e-13)
    assert np.allclose(out[:, 4:].sum(1), 1.0, atol=1e-13)


def test_triangle_cage_and_open_boundary():
    # a single triangle: boundary rules (edge midpoints; corners (6P + two neighbours)/8)
    v = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0]], float)
    out, quads = oracle.subdivide([0, 3], [0, 1, 2], v, 1)
    assert len(out) == 3 + 3 + 1 and len(quads) == 3
    assert np.allclose(out[0], (6 * v[0] + v[1] + v[2]) / 8)
    assert np.allclose(out[3], [1, 0, 0]) and np.allclose(out[6], [2 / 3, 2 / 3, 0])
