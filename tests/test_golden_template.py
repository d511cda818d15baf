"""The one worked example the paper prints: the sizes of its template before and after two levels of
Catmull-Clark subdivision (Sec. 3.3; tests/golden/template_subdivision_counts.txt).  Any closed genus-0
cage with the printed vertex and face counts has the same counts after subdivision, so a latitude-longitude
sphere with those counts stands in for the paper's cage.  Host logic only (oracle and the library's
host-side counting)."""
import os

import numpy as np

import oracle
from paper_1711_07999_gb300 import trk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "template_subdivision_counts.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = int(v)
    return out


def _sphere_cage(segments, rings, n_split):
    """Closed genus-0 polygon cage: poles, `rings` latitude circles of `segments` vertices, triangle fans
    at the poles, quads between circles, and the first `n_split` quads of the middle band split into two
    triangles.  Faces are counter-clockwise seen from outside."""
    s, r = segments, rings
    th = np.pi * (np.arange(r) + 1) / (r + 1)
    ph = 2 * np.pi * np.arange(s) / s
    ring = np.stack([np.outer(np.sin(th), np.cos(ph)), np.outer(np.sin(th), np.sin(ph)),
                     np.outer(np.cos(th), np.ones(s))], -1).reshape(-1, 3)
    verts = np.vstack([[0, 0, 1], ring, [0, 0, -1]])
    north, south = 0, 1 + r * s
    at = lambda k, j: 1 + k * s + j % s
    faces = [[north, at(0, j), at(0, j + 1)] for j in range(s)]
    split = 0
    for k in range(r - 1):
        for j in range(s):
            q = [at(k, j), at(k + 1, j), at(k + 1, j + 1), at(k, j + 1)]
            if k == r // 2 and split < n_split:
                faces += [q[:3], [q[0], q[2], q[3]]]
                split += 1
            else:
                faces.append(q)
    faces += [[south, at(r - 1, j + 1), at(r - 1, j)] for j in range(s)]
    fo = np.cumsum([0] + [len(f) for f in faces])
    return verts, fo, np.concatenate(faces)


def _cage_like_the_papers(g):
    # V = 2 + rings * segments and F = segments * (rings + 1) + splits: 3460 = 2 + 247 * 14, 3476 = 14 * 248 + 4
    verts, fo, fv = _sphere_cage(14, 247, 4)
    assert len(verts) == g["cage_vertices"] and len(fo) - 1 == g["cage_faces"]
    return verts, fo, fv


def _edges(fo, fv):
    fv = fv.tolist()
    return [(fv[a + i], fv[a + (i + 1) % (b - a)]) for a, b in zip(fo[:-1].tolist(), fo[1:].tolist()) for i in range(b - a)]


def test_stand_in_cage_is_closed_genus_zero():
    g = _golden()
    verts, fo, fv = _cage_like_the_papers(g)
    d = _edges(fo, fv)
    sd = set(d)
    assert len(sd) == len(d)  # each directed edge once ...
    assert all((b, a) in sd for a, b in d)  # ... and its reverse once: closed, consistently oriented
    E = len(d) // 2
    assert len(verts) - E + (len(fo) - 1) == 2


def test_two_levels_give_the_printed_vertex_count():
    g = _golden()
    verts, fo, fv = _cage_like_the_papers(g)
    out, quads = oracle.subdivide(fo, fv, verts, g["levels"])
    assert len(out) == g["result_vertices"]
    # the library's host-side counting of the authoring call agrees
    nv, nt = trk.subdivide_counts(fo, fv, len(verts), g["levels"])
    assert nv == g["result_vertices"] and nt == 2 * len(quads)


def test_triangle_count_reading():
    """After two levels every face is a quad and the count is 4 x (sum of the level-1 face sizes) = 8 x (2E - E_b),
    so the triangulated count is a multiple of 8 for any cage.  The printed 110,994 is not; the count the
    printed vertex count implies (a closed cage, E = V + F - 2 = 6,934) is 16 E = 110,944, which is what
    the oracle gives."""
    g = _golden()
    assert g["result_triangles_printed"] % 8 != 0
    verts, fo, fv = _cage_like_the_papers(g)
    _, quads = oracle.subdivide(fo, fv, verts, g["levels"])
    E = g["cage_vertices"] + g["cage_faces"] - 2
    assert 2 * len(quads) == 16 * E == 110944
