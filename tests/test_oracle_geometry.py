"""Pins of the oracle's normals (R4), z-buffer (R5, R6), visibility (R7), projective association
(Sec. 4.1 with R8, R9), neighbourhoods N(i) (Sec. 4.3, R16) and prior weights S (Sec. 4.2, R10), against
brute force, closed forms and special cases."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import synth
from tests import helpers as H


def test_flat_grid_has_constant_normal():
    V, T = H.grid_patch(6, 5, -0.2, 0.2, -0.1, 0.1, 2.0)
    n, ok = oracle.normals(V, T)
    assert ok.all()
    assert np.allclose(n, [0, 0, -1], atol=1e-15)


def test_capsule_normals_are_radial_within_mesh_spacing():
    m = synth.make_model(1)
    v = m["mesh"]["verts"].astype(np.float64)
    n, ok = oracle.normals(v, m["mesh"]["tris"])
    n0 = m["motion"]["bind_normals"]
    cosang = np.einsum("ij,ij->i", n, n0)
    assert ok.all()
    # outward orientation everywhere, deviation of the order of the spacing / radius
    assert cosang.min() > 0.9
    assert np.median(cosang) > 0.995


def _mt_depth(orig_dir, A, B, C):
    """Moller-Trumbore: ray (0, d) against triangle ABC; returns hit distance along d or None."""
    d = orig_dir
    e1, e2 = B - A, C - A
    p = np.cross(d, e2)
    det = e1 @ p
    if abs(det) < 1e-15:
        return None
    inv = 1.0 / det
    s = -A
    u = (s @ p) * inv
    q = np.cross(s, e1)
    v = (d @ q) * inv
    if u < -1e-12 or v < -1e-12 or u + v > 1 + 1e-12:
        return None
    t = (e2 @ q) * inv
    return t if t > 0 else None


@pytest.mark.parametrize("seed", [0, 1])
def test_raster_equals_brute_force_ray_casting(seed):
    rng = np.random.default_rng(seed)
    W, Hh, fx, fy, cx, cy = 24, 18, 20.0, 20.0, 12.0, 9.0
    tris, verts = [], []
    for f in range(12):
        c = rng.uniform([-0.8, -0.6, 1.5], [0.8, 0.6, 3.0])
        pts = c + rng.normal(0, 0.25, (3, 3))
        verts.extend(pts)
        tris.append([3 * f, 3 * f + 1, 3 * f + 2])
    v = np.array(verts)
    z, zt, amb = oracle.raster(W, Hh, fx, fy, cx, cy, 0.05, v, tris, with_amb=True)
    assert amb.sum() <= 3
    for py in range(Hh):
        for px in range(W):
            d = np.array([(px - cx) / fx, (py - cy) / fy, 1.0])
            best, bt = math.inf, -1
            for f, (a, b, c) in enumerate(tris):
                t = _mt_depth(d, v[a], v[b], v[c])
                if t is not None and t < best:
                    best, bt = t, f
            if amb[py, px]:
                continue  # coverage decided at rounding level (flagged pixels: a handful at most)
            if bt < 0:
                assert not np.isfinite(z[py, px])
            else:
                assert z[py, px] == pytest.approx(best, rel=1e-12)
                assert zt[py, px] == bt


def test_zbuffer_flags_exactly_the_pixels_on_an_edge():
    # R6: a pixel centre within 1e-3 px of a triangle's edge (on the triangle's side of the other two
    # edges) has a coverage that rounding decides, and is flagged ambiguous; no other pixel is.  Camera
    # fx = fy = 20, principal point (10, 10), depth 2: u = 10 x + 10.  The triangle's corners project to
    # (5, 5), (15, 5), (5, 15), shifted by `off` pixels in u and v.
    def amb_at(off, corners=((5.0, 5.0), (15.0, 5.0), (5.0, 15.0))):
        uv = np.array(corners) + off
        v = np.array([[(u - 10.0) / 10.0, (w - 10.0) / 10.0, 2.0] for u, w in uv])
        _, _, amb = oracle.raster(20, 20, 20.0, 20.0, 10.0, 10.0, 0.05, v, [[0, 1, 2]], with_amb=True)
        return {(int(px), int(py)) for py, px in zip(*np.nonzero(amb))}
    edges = ({(px, 5) for px in range(5, 16)} | {(5, py) for py in range(5, 16)}
             | {(px, 20 - px) for px in range(5, 16)})
    assert len(edges) == 30
    assert amb_at(0.0) == edges        # the centres on the edges and corners
    assert amb_at(0.0005) == edges     # 0.5 mpx from them (0.7 mpx from the slanted edge)
    assert amb_at(0.005) == set()      # 5 mpx from them
    # corners (5, 5), (10, 8), (15, 15): the line of the edge (5, 5)-(10, 8) passes the centre (15, 11)
    # inside the bounding box but beyond the corner, outside the triangle: not flagged
    assert amb_at(0.0, ((5.0, 5.0), (10.0, 8.0), (15.0, 15.0))) == {(k, k) for k in range(5, 16)} | {(10, 8)}


def test_fronto_parallel_quad_has_constant_depth():
    V, T = H.grid_patch(2, 2, -0.5, 0.5, -0.4, 0.4, 2.5)
    z, zt, _ = oracle.raster(40, 30, 30.0, 30.0, 20.0, 15.0, 0.05, V, T)
    covered = np.isfinite(z)
    assert covered.sum() > 100
    assert np.all(z[covered] == 2.5)


def test_tilted_plane_depth_closed_form():
    # plane z = z0 + a x: along the ray (u, v, 1) s, depth = z0 / (1 - a u)
    z0, a = 2.0, 0.3
    V = np.array([[-0.6, -0.5, z0 - 0.6 * a], [0.6, -0.5, z0 + 0.6 * a], [-0.6, 0.5, z0 - 0.6 * a],
                  [0.6, 0.5, z0 + 0.6 * a]])
    T = [[0, 2, 1], [1, 2, 3]]
    W, Hh, f = 40, 30, 30.0
    z, _, _ = oracle.raster(W, Hh, f, f, 20.0, 15.0, 0.05, V, T)
    for py in range(Hh):
        for px in range(W):
            if np.isfinite(z[py, px]):
                u = (px - 20.0) / f
                assert z[py, px] == pytest.approx(z0 / (1 - a * u), rel=1e-12)


def test_visibility_occlusion_backface_and_image_bounds():
    front, Tf = H.grid_patch(5, 5, -0.2, 0.2, -0.2, 0.2, 2.0)
    back, Tb = H.grid_patch(5, 5, -0.2, 0.2, -0.2, 0.2, 2.5)
    away, Ta = H.grid_patch(3, 3, 0.3, 0.5, -0.1, 0.1, 2.0, facing_camera=False)
    outside = np.array([[5.0, 0, 2.0], [5.1, 0, 2.0], [5.0, 0.1, 2.0]])
    verts = np.concatenate([front, back, away, outside])
    tris = np.concatenate([Tf, Tb + 25, Ta + 50, [[59, 61, 60]]])
    nV = len(verts)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, tris, [[0, 0, 0, 0]] * nV, [[1, 0, 0, 0]] * nV,
                     W=40, H=40, fx=40.0, fy=40.0)
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    n, ok = o.normals(v)
    z, zt, _ = o.raster(v)
    vis, pix, _ = o.visibility(v, n, ok, z)
    assert vis[:25].all()                  # front plane visible
    assert not vis[25:50].any()            # hidden 0.5 m behind it (> eps_vis)
    assert not vis[50:59].any()            # facing away from the camera
    assert not vis[59:].any()              # projects outside the image


def test_triangle_crossing_the_near_plane_is_skipped():
    # R6: a triangle with a vertex at z <= z_near is not rasterised (no clipping); a background plane at
    # 3 m covers the whole image and keeps every pixel
    back, Tb = H.grid_patch(2, 2, -3.0, 3.0, -3.0, 3.0, 3.0)
    cross = [[0.0, 0.0, 1.0], [0.2, 0.0, 1.0], [0.1, 0.1, 0.01]]
    verts = np.concatenate([back, cross])
    tris = np.concatenate([Tb, [[4, 5, 6]]])
    nV = len(verts)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, tris, [[0, 0, 0, 0]] * nV, [[1, 0, 0, 0]] * nV)
    assert m["params"]["z_near"] > 0.01
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    z, zt, _ = o.raster(v)
    assert (zt >= 0).all() and (zt < 2).all()
    assert np.allclose(z, 3.0, rtol=0, atol=1e-12)


def test_coincident_triangles_keep_the_smaller_index():
    # R6: equal depths go to the smaller triangle; the quad's two triangles are duplicated with larger ids
    V, T = H.grid_patch(2, 2, -0.3, 0.3, -0.3, 0.3, 2.0)
    tris = np.concatenate([T, T])
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, tris, [[0, 0, 0, 0]] * 4, [[1, 0, 0, 0]] * 4)
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    z, zt, _ = o.raster(v)
    covered = zt >= 0
    assert covered.sum() > 50
    assert (zt[covered] < 2).all()


def test_back_face_is_judged_along_the_view_ray():
    # R7 front-facing means n . p < 0 for the camera-frame vertex p.  Two tiny triangles at p ~ (0.9, 0, 2):
    # one tilted so that n_z < 0 but n . p > 0 (it faces the optical axis, not the ray to it): hidden; one
    # with n . p < 0: visible
    def facing(p0, nrm, h=0.004):
        nrm = np.asarray(nrm, float) / np.linalg.norm(nrm)
        u1 = np.array([0.0, 1.0, 0.0])
        u2 = np.cross(nrm, u1)  # (h u1) x (h u2) points along nrm
        return [p0, p0 + h * u1, p0 + h * u2]
    p0 = np.array([0.9, 0.0, 2.0])
    away = facing(p0, [0.92, 0.0, -0.39])
    toward = facing(p0 + [0, 0.1, 0], [0.3, 0.0, -0.95])
    verts = np.concatenate([away, toward])
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 1, 2], [3, 4, 5]], [[0, 0, 0, 0]] * 6,
                     [[1, 0, 0, 0]] * 6, W=40, H=40, fx=40.0, fy=40.0, cx=20.0, cy=20.0)
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    n, ok = o.normals(v)
    assert ok.all() and (n[:, 2] < 0).all()
    assert ((n * v).sum(1)[:3] > 0).all() and ((n * v).sum(1)[3:] < 0).all()
    z, _, _ = o.raster(v)
    vis, pix, _ = o.visibility(v, n, ok, z)
    assert not vis[:3].any() and vis[3:].all()


def _tiny_triangle(x, y, z, h=0.004):
    # facing the camera (normal -z), too small to cover a pixel centre of the 40 x 40 camera below
    return [[x, y, z], [x, y + h, z], [x + h, y, z]]


def test_visibility_rounds_to_the_nearest_pixel_and_tolerates_eps_vis():
    # camera fx = fy = 40, principal point (20, 20), depth 2: u = 20 x + 20.  R7: a front-facing vertex is
    # visible in the pixel its projection rounds to, if that pixel is in the image and the vertex is at
    # most eps_vis (1 cm) behind the z-buffer there (or the pixel is empty)
    occluder, To = H.grid_patch(3, 3, 0.2, 0.6, 0.2, 0.6, 2.0)  # covers pixels 24..32 in u and v
    tiny = [_tiny_triangle(-0.48, 0.0, 2.0),   # u = 10.4: pixel 10
            _tiny_triangle(-0.47, 0.0, 2.0),   # u = 10.6: pixel 11
            _tiny_triangle(0.97, 0.0, 2.0),    # u = 39.4: pixel 39, the last column
            _tiny_triangle(0.98, 0.0, 2.0),    # u = 39.6: rounds to 40, outside
            _tiny_triangle(0.4, 0.4, 2.005),   # 5 mm behind the occluder: visible
            _tiny_triangle(0.3, 0.3, 2.02)]    # 2 cm behind it: hidden
    verts = np.concatenate([occluder, np.concatenate(tiny)])
    tris = np.concatenate([To, 9 + np.arange(18).reshape(6, 3)])
    nV = len(verts)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, tris, [[0, 0, 0, 0]] * nV, [[1, 0, 0, 0]] * nV,
                     W=40, H=40, fx=40.0, fy=40.0, cx=20.0, cy=20.0)
    assert m["params"]["eps_vis"] == 0.01
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    n, ok = o.normals(v)
    z, _, _ = o.raster(v)
    vis, pix, _ = o.visibility(v, n, ok, z)
    t = lambda k: slice(9 + 3 * k, 12 + 3 * k)
    assert vis[:9].all()
    assert vis[t(0)].all() and (pix[t(0)] == 20 * 40 + 10).all()
    assert vis[t(1)].all() and (pix[t(1)] == 20 * 40 + 11).all()
    assert vis[t(2)].all() and (pix[t(2)] == 20 * 40 + 39).all()
    assert not vis[t(3)].any() and (pix[t(3)] == -1).all()
    assert np.isfinite(z.ravel()[pix[t(4)]]).all() and vis[t(4)].all()
    assert not vis[t(5)].any()


def _bruteforce_assoc(o, v, vis, pix, depth, R):
    """Every pixel against every visible vertex whose bucket lies in the window (vectorised over vertices)."""
    W, Hh = o.W, o.H
    tau2 = o.params["cutoff"] ** 2
    corr = -np.ones((Hh, W), int)
    pu, pv = pix % W, pix // W
    idx = np.arange(o.V)
    for py in range(Hh):
        for px in range(W):
            d = float(depth[py, px])
            if d <= 0:
                continue
            p = np.array([(px - o.cx) * d / o.fx, (py - o.cy) * d / o.fy, d])
            cand = (vis > 0) & (np.abs(pu - px) <= R) & (np.abs(pv - py) <= R)
            if not cand.any():
                continue
            dd = ((p - v[cand]) ** 2).sum(1)
            ok = dd <= tau2
            if not ok.any():
                continue
            ii, dd = idx[cand][ok], dd[ok]
            corr[py, px] = ii[np.lexsort((ii, dd))[0]]
    return corr


@pytest.mark.parametrize("R", [1, 3, 50])
def test_association_equals_brute_force(R):
    m = synth.make_model(1, V=1500, width=64, height=48)
    m["params"]["window_half"] = R
    o = oracle.Oracle(m)
    th = synth.gt_theta(m, 0)
    z = o.render(th)
    depth = synth.add_noise(z, 1, np.random.default_rng(5))
    th2 = th + np.radians(1) * np.random.default_rng(6).normal(size=o.L)
    P = o.pass_at(th2, None, depth)
    ref = _bruteforce_assoc(o, P["v"], P["vis"], P["pix"], depth, R)
    assert np.array_equal(P["corr"], ref)
    assert (ref >= 0).sum() > 20
    # per-vertex sums of Sec. 4.1
    acc, cnt = o.accumulate(P["v"], depth, ref)
    assert np.array_equal(cnt, P["cnt"]) and np.allclose(acc, P["acc"], atol=1e-15)


def test_single_vertex_collects_every_pixel_within_cutoff():
    verts = np.array([[0.0, 0.0, 2.0], [0.01, 0.0, 2.0], [0.0, 0.01, 2.0]])
    # only vertex 0 is visible: give vertices 1, 2 a degenerate face so their normals are invalid
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3, [[1, 0, 0, 0]] * 3,
                     W=30, H=30, fx=200.0, fy=200.0, window_half=30, cutoff=0.05)
    o = oracle.Oracle(m)
    v, _ = o.skin([0.0])
    n, ok = o.normals(v)
    vis = np.array([1, 0, 0], np.int32)
    u = int(math.floor(200 * 0 / 2 + 15 + 0.5))
    pix = np.array([15 * 30 + u, -1, -1], np.int32)
    depth = np.full((30, 30), 2.02, np.float32)
    corr, acc, cnt, _ = o.associate(v, vis, pix, depth)
    for py in range(30):
        for px in range(30):
            p = np.array([(px - 15) * 2.02 / 200, (py - 15) * 2.02 / 200, 2.02])
            within = np.linalg.norm(p - v[0]) <= 0.05
            assert corr[py, px] == (0 if within else -1)
    assert cnt[0] == (corr == 0).sum()


def test_association_ties_go_to_smaller_index():
    verts = np.array([[-0.01, 0.0, 2.0], [0.01, 0.0, 2.0], [0.0, 0.2, 2.0]])
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3, [[1, 0, 0, 0]] * 3,
                     W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, window_half=5, cutoff=0.05)
    o = oracle.Oracle(m)
    v = verts.astype(np.float64)
    vis = np.array([1, 1, 0], np.int32)
    pix = np.array([15 * 31 + 15, 15 * 31 + 16, -1], np.int32)
    depth = np.zeros((31, 31), np.float32)
    depth[15, 15] = 2.0  # p = (0, 0, 2): equidistant from vertices 0 and 1
    corr, *_ = o.associate(v, vis, pix, depth)
    assert corr[15, 15] == 0


def test_near_ties_are_flagged():
    # the oracle flags a pixel whose two best candidates are within 1e-5 m of each other (a decision that
    # FP32 rounding may take either way); candidates 1 mm apart are not flagged
    def run(dx1):
        verts = np.array([[-0.01, 0.0, 2.0], [0.01 + dx1, 0.0, 2.0], [0.0, 0.2, 2.0]])
        m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3,
                         [[1, 0, 0, 0]] * 3, W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, window_half=5,
                         cutoff=0.05)
        o = oracle.Oracle(m)
        depth = np.zeros((31, 31), np.float32)
        depth[15, 15] = 2.0
        corr, _, _, tie = o.associate(verts, np.array([1, 1, 0], np.int32),
                                      np.array([15 * 31 + 15, 15 * 31 + 16, -1], np.int32), depth, with_tie=True)
        return corr[15, 15], tie[15, 15]
    assert run(4e-6) == (0, 1)
    assert run(1e-3) == (0, 0)


def test_cutoff_ties_are_those_of_the_nearest_candidate():
    # The cutoff can change a pixel's correspondence only through its nearest candidate: a pixel is a tie
    # where that candidate lies within 1e-5 m of the cutoff (5 cm), not where a farther one does.
    def run(d_near, d_far):
        verts = np.array([[d_near, 0.0, 2.0], [0.0, d_far, 2.0], [0.0, 0.3, 2.0]])
        m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3,
                         [[1, 0, 0, 0]] * 3, W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, window_half=5,
                         cutoff=0.05)
        o = oracle.Oracle(m)
        depth = np.zeros((31, 31), np.float32)
        depth[15, 15] = 2.0
        corr, _, _, tie = o.associate(verts, np.array([1, 1, 0], np.int32),
                                      np.array([15 * 31 + 15, 17 * 31 + 15, -1], np.int32), depth, with_tie=True)
        return int(corr[15, 15]), int(tie[15, 15])
    assert run(0.004, 0.05) == (0, 0)           # a farther candidate exactly at the cutoff
    assert run(0.004, 0.05 + 3e-6) == (0, 0)    # ... or just beyond it
    assert run(0.05 - 5e-6, 0.2) == (0, 1)      # the nearest 5 um inside the cutoff
    assert run(0.05 + 5e-6, 0.2) == (-1, 1)     # 5 um beyond it
    assert run(0.05 - 5e-5, 0.2) == (0, 0)      # 50 um inside it


def _facing_normal(p, s):
    """A unit normal whose dot product with the view ray p is s |p| (s = sine of its angle to the plane
    normal to the ray; negative: front-facing)."""
    ph = p / np.linalg.norm(p)
    e = np.cross(ph, [1.0, 0.0, 0.0])
    e /= np.linalg.norm(e)
    return math.sqrt(1.0 - s * s) * e + s * ph


def test_visibility_flags_exactly_its_marginal_decisions():
    # R7's decisions that an FP32 evaluation may take the other way are flagged marginal, and only those:
    # the facing test within 1e-4 rad (|n.p| < 1e-4 |p|), the pixel rounding within 1e-3 px of a pixel
    # edge, the depth test within 1e-5 m of Z + eps_vis, a pixel whose z-buffer winner is ambiguous.
    # Camera fx = fy = 40, principal point (20, 20), depth 2: u = 20 x + 20, v = 20 y + 20; each case in a
    # pixel of its own.
    cases = []  # (p, n, nvalid, Z at its pixel or inf, ambiguous pixel, expected vis, expected marg)
    def add(u, v, s=-1.0, z=2.0, Z=np.inf, amb=0, nvalid=1, vis=1, marg=0):
        p = np.array([(u - 20.0) * z / 40.0, (v - 20.0) * z / 40.0, z])
        cases.append((p, _facing_normal(p, s), nvalid, Z, amb, vis, marg))
    add(5, 5)                                  # plain front-facing, pixel centre
    add(7, 5, s=-0.7e-4, marg=1)               # facing within the band, front
    add(9, 5, s=+0.7e-4, vis=0, marg=1)        # facing within the band, back
    add(11, 5, s=-3e-4)                        # facing outside the band
    add(13, 5, s=+3e-4, vis=0)                 # back-facing outside the band
    add(15.4996, 5, marg=1)                    # 0.4 mpx below a pixel edge
    add(17.5004, 5, marg=1)                    # 0.4 mpx above one
    add(19.498, 5)                             # 2 mpx from it
    add(5, 9.5004, marg=1)                     # the same in v
    add(7, 9.498)
    add(5, 13, z=2.0, Z=2.0 - 0.01 - 0.5e-5, vis=0, marg=1)   # 5 um behind Z + eps_vis
    add(7, 13, z=2.0, Z=2.0 - 0.01 + 0.5e-5, vis=1, marg=1)   # 5 um in front of it
    add(9, 13, z=2.0, Z=2.0 - 0.01 - 3e-5, vis=0)             # 30 um behind
    add(11, 13, z=2.0, Z=2.0 - 0.01 + 3e-5, vis=1)            # 30 um in front
    add(13, 13, z=2.0, Z=1.5, vis=0)                          # well behind an occluder
    add(15, 13, Z=2.5, amb=1, marg=1)                         # ambiguous z-buffer winner
    add(17, 13, Z=2.5)                                        # the same pixel state, unambiguous
    add(5, 17, s=-0.7e-4, nvalid=0, vis=0)                    # no normal: never visible, never marginal
    add(7, 17, z=0.04, vis=0)                                 # before the near plane
    add(-0.6, 17, vis=0)                                      # rounds to pixel -1: outside the image
    add(39.4, 17, vis=1)                                      # the last column
    nV = len(cases)
    verts = np.array([c[0] for c in cases])
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 1, 2]], [[0, 0, 0, 0]] * nV,
                     [[1, 0, 0, 0]] * nV, W=40, H=40, fx=40.0, fy=40.0, cx=20.0, cy=20.0)
    assert m["params"]["eps_vis"] == 0.01 and m["params"]["z_near"] == 0.05
    o = oracle.Oracle(m)
    z = np.full((40, 40), np.inf)
    amb = np.zeros((40, 40), np.int32)
    for p, _, _, Z, a, _, _ in cases:
        if p[2] > 0.05:
            u, v = 40.0 * p[0] / p[2] + 20.0, 40.0 * p[1] / p[2] + 20.0
            k = (int(math.floor(v + 0.5)), int(math.floor(u + 0.5)))
            if 0 <= k[0] < 40 and 0 <= k[1] < 40:
                z[k], amb[k] = Z, a
    n = np.array([c[1] for c in cases])
    ok = np.array([c[2] for c in cases], np.int32)
    vis, pix, marg = o.visibility(verts, n, ok, z, amb, with_marg=True)
    assert list(vis) == [c[5] for c in cases]
    assert list(marg) == [c[6] for c in cases]
    assert (pix[vis == 0] == -1).all()
    # without the flags the decisions are the same
    vis2, pix2, _ = o.visibility(verts, n, ok, z, amb)
    assert np.array_equal(vis, vis2) and np.array_equal(pix, pix2)


def test_marginal_vertices_make_their_pixels_ties():
    # A pixel is a tie where a marginal vertex (visible or not, its bucket one pixel beyond the window
    # included) could be the argmin: within the cutoff + 1e-5 m and within 1e-5 m of the best distance.
    # Camera fx = fy = 100, principal point (15, 15), window 1 (1 px = 2 cm at depth 2); the pixel (15, 15)
    # at depth 2 has p = (0, 0, 2).
    verts = np.array([[0.004, 0.0, 2.0],     # 0: visible, 4 mm from p: the argmin
                      [0.0, 0.0035, 2.0],    # 1: marginal, hidden, nearer than 0
                      [0.0, -0.006, 2.0],    # 2: marginal, 2 mm farther than 0
                      [0.04, 0.0, 2.0]])     # 3: marginal, 2 px out (one beyond the window), 4 cm away
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 1, 2]], [[0, 0, 0, 0]] * 4,
                     [[1, 0, 0, 0]] * 4, W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, window_half=1,
                     cutoff=0.05)
    o = oracle.Oracle(m)
    depth = np.zeros((31, 31), np.float32)
    depth[15, 15] = 2.0
    pix = np.array([15 * 31 + 15, -1, -1, -1], np.int32)

    def tie_at(vis, marg):
        corr, _, _, tie = o.associate(verts, np.array(vis, np.int32), pix, depth, np.array(marg, np.int32),
                                      with_tie=True)
        return corr[15, 15], tie[15, 15]
    assert tie_at([1, 0, 0, 0], [0, 0, 0, 0]) == (0, 0)
    assert tie_at([1, 0, 0, 0], [0, 1, 0, 0]) == (0, 1)   # could be nearer than the argmin
    assert tie_at([1, 0, 0, 0], [0, 0, 1, 0]) == (0, 0)   # farther than the argmin by more than 1e-5 m
    assert tie_at([1, 0, 0, 0], [0, 0, 0, 1]) == (0, 0)
    assert tie_at([1, 0, 0, 0], [1, 0, 0, 0]) == (0, 1)   # the argmin itself marginal
    # no visible candidate: a marginal vertex within the cutoff makes the empty result a tie, also one
    # whose bucket lies one pixel beyond the window
    assert tie_at([0, 0, 0, 0], [0, 0, 0, 0]) == (-1, 0)
    assert tie_at([0, 0, 0, 0], [0, 0, 1, 0]) == (-1, 1)
    assert tie_at([0, 0, 0, 0], [0, 0, 0, 1]) == (-1, 1)


def test_knn_equals_brute_force():
    m = synth.make_model(1, V=800)
    o = oracle.Oracle(m)
    _, _, nbr = o.derived()
    v = m["mesh"]["verts"].astype(np.float64)
    for i in range(0, o.V, 7):
        d2 = ((v - v[i]) ** 2).sum(1)
        d2[i] = np.inf
        order = np.lexsort((np.arange(o.V), d2))[:4]
        assert list(nbr[i]) == list(order)


def test_knn_ties_on_a_regular_grid_go_to_smaller_index():
    V, T = H.grid_patch(4, 4, 0.0, 0.3, 0.0, 0.3, 2.0)
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], V, T, [[0, 0, 0, 0]] * 16, [[1, 0, 0, 0]] * 16)
    o = oracle.Oracle(m)
    _, _, nbr = o.derived()
    assert list(nbr[5]) == [1, 4, 6, 9]   # interior vertex: its four axis neighbours, by index
    assert list(nbr[0]) == [1, 4, 5, 2]   # corner: two at h, then sqrt(2) h, then 2h (index 2 < 8)


def test_prior_weights_count_subtree_vertices():
    m = synth.make_model(1, V=900)
    o = oracle.Oracle(m)
    _, S, _ = o.derived()
    sk = m["skeleton"]
    L, V = len(sk["parent"]), o.V
    anc = [[j] for j in range(L)]
    for j in range(L):
        k = sk["parent"][j]
        while k >= 0:
            anc[j].append(k)
            k = sk["parent"][k]
    for k in range(L):
        n_k = 0
        for i in range(V):
            links = {int(j) for j, w in zip(m["mesh"]["bone_idx"][i], m["mesh"]["bone_w"][i]) if w > 0}
            if any(k in anc[j] for j in links):
                n_k += 1
        assert S[k] == pytest.approx(float(sk["prior_mask"][k]) * n_k / V, rel=1e-15)
