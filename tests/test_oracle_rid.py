"""Pins of the oracle's raster-ID association (reading R23: a pixel takes the nearest corner of the
triangle the z-buffer holds there)."""
import numpy as np

import oracle
from tests import helpers as H
from paper_1711_07999_gb300 import synth


def _setup(seed=4, V=3000):
    m = synth.make_model(1, V=V, width=96)
    o = oracle.Oracle(m)
    gt = synth.gt_theta(m, 0)
    depth = synth.add_noise(o.render(gt, synth.gt_offsets(m, 0)), 1, np.random.default_rng(seed))
    P = o.pass_at(gt, None, depth)
    return m, o, gt, depth, P


def test_each_pixel_takes_the_nearest_corner_of_its_triangle():
    m, o, gt, depth, P = _setup()
    corr, acc, cnt, _ = o.associate_rid(P["v"], P["ztri"], depth)
    tri = np.asarray(m["mesh"]["tris"])
    H, W = depth.shape
    fx, fy, cx, cy = (m["camera"][k] for k in ("fx", "fy", "cx", "cy"))
    tau = m["params"]["cutoff"]
    ys, xs = np.nonzero(depth > 0)
    for py, px in list(zip(ys, xs))[::7]:
        t = P["ztri"][py, px]
        if t < 0:
            assert corr[py, px] == -1
            continue
        z = float(depth[py, px])
        p = np.array([(px - cx) * z / fx, (py - cy) * z / fy, z])
        d2 = ((P["v"][tri[t]] - p) ** 2).sum(1)
        c = [(d2[k], tri[t][k]) for k in range(3) if d2[k] <= tau * tau]
        assert corr[py, px] == (min(c)[1] if c else -1)
    # the sums are those of the map
    acc2, cnt2 = o.accumulate(P["v"], depth, corr)
    assert np.array_equal(cnt, cnt2) and np.allclose(acc, acc2, rtol=0, atol=1e-12)


def test_never_closer_than_the_window_search():
    # the window search returns the nearest visible vertex in the window; a corner of the rasterised
    # triangle that is visible and inside the window is one of its candidates, so the raster-ID
    # correspondence is never strictly closer than the window search's
    m, o, gt, depth, P = _setup(seed=6)
    corr_w = P["corr"]
    corr_r, _, _, _ = o.associate_rid(P["v"], P["ztri"], depth)
    H, W = depth.shape
    fx, fy, cx, cy = (m["camera"][k] for k in ("fx", "fy", "cx", "cy"))
    R = m["params"]["window_half"]
    n_equal = n_both = 0
    for py, px in zip(*np.nonzero((corr_w >= 0) & (corr_r >= 0))):
        i_r, i_w = corr_r[py, px], corr_w[py, px]
        pix = P["pix"][i_r]
        if not P["vis"][i_r] or abs(pix % W - px) > R or abs(pix // W - py) > R:
            continue
        z = float(depth[py, px])
        p = np.array([(px - cx) * z / fx, (py - cy) * z / fy, z])
        d_r = ((P["v"][i_r] - p) ** 2).sum()
        d_w = ((P["v"][i_w] - p) ** 2).sum()
        assert d_w <= d_r
        n_both += 1
        n_equal += i_r == i_w
    assert n_both > 200 and n_equal > 0.5 * n_both, (n_both, n_equal)


def test_uncovered_pixels_get_no_correspondence():
    m, o, gt, depth, P = _setup(seed=8)
    ztri = np.full_like(P["ztri"], -1)
    corr, acc, cnt, _ = o.associate_rid(P["v"], ztri, depth)
    assert np.all(corr == -1) and np.all(cnt == 0)


def test_equidistant_corners_go_to_the_smaller_index():
    # the pixel at the principal point back-projects to p = (0, 0, 2), inside the triangle and exactly as
    # far from corner 0 as from corner 1 (mirror images in x); corner 2 is farther
    verts = np.array([[-0.01, -0.01, 2.0], [0.01, -0.01, 2.0], [0.0, 0.02, 2.0]])
    m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3, [[1, 0, 0, 0]] * 3,
                     W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, cutoff=0.05)
    o = oracle.Oracle(m)
    v = verts.astype(np.float64)
    _, ztri, _ = o.raster(v)
    assert ztri[15, 15] == 0
    depth = np.zeros((31, 31), np.float32)
    depth[15, 15] = 2.0
    corr, _, cnt, _ = o.associate_rid(v, ztri, depth)
    assert corr[15, 15] == 0 and cnt[0] == 1 and cnt[1] == 0



def test_ties_are_flagged():
    # The raster-ID map is compared with the GPU's except where its decision is a rounding-level one:
    # two corners within 1e-5 m of each other (within the cutoff), a corner within 1e-5 m of the cutoff,
    # or a pixel whose z-buffer winner is ambiguous.  p = (0, 0, 2) as above; corner 0 is 14.14 mm away.
    def flags(dx1, cutoff, amb=0):
        verts = np.array([[-0.01, -0.01, 2.0], [0.01 + dx1, -0.01, 2.0], [0.0, 0.02, 2.0]])
        m = H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], verts, [[0, 2, 1]], [[0, 0, 0, 0]] * 3,
                         [[1, 0, 0, 0]] * 3, W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, cutoff=cutoff)
        o = oracle.Oracle(m)
        v = verts.astype(np.float64)
        _, ztri, _ = o.raster(v)
        assert ztri[15, 15] == 0
        depth = np.zeros((31, 31), np.float32)
        depth[15, 15] = 2.0
        zamb = np.zeros((31, 31), np.int32)
        zamb[15, 15] = amb
        corr, _, _, tie = o.associate_rid(v, ztri, depth, zamb=zamb, with_tie=True)
        assert tie.sum() == tie[15, 15]  # only the one pixel with a depth can be flagged
        return int(corr[15, 15]), int(tie[15, 15])
    d0 = float(np.hypot(0.01, 0.01))
    assert flags(0.0, 0.05) == (0, 1)           # corners 0 and 1 equidistant
    assert flags(4e-6, 0.05) == (0, 1)          # 2.8 um apart
    assert flags(1e-3, 0.05) == (0, 0)          # 0.7 mm apart
    assert flags(1e-3, d0 + 5e-6) == (0, 1)     # corner 0 5 um inside the cutoff
    assert flags(1e-3, d0 - 5e-6) == (-1, 1)    # 5 um outside it
    assert flags(1e-3, d0 + 5e-5) == (0, 0)     # 50 um inside it
    assert flags(1e-3, 0.05, amb=1) == (0, 1)   # an ambiguous z-buffer pixel
    assert flags(0.0, 0.01) == (-1, 0)          # equidistant corners both beyond the cutoff
