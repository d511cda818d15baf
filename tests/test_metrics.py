"""The evaluation measures of Sec. 5 (paper_1711_07999_gb300.metrics) against brute force, and the
library's host forward kinematics (trk_fk_joint_positions) against the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1711_07999_gb300 import metrics, synth


def test_accuracy_curve_and_auc():
    e = np.array([0.01, 0.02, 0.02, 0.05, 0.2])
    t = np.array([0.0, 0.01, 0.015, 0.02, 0.05, 0.1, 0.3])
    brute = np.array([(e <= x).mean() for x in t])
    assert np.array_equal(metrics.accuracy_curve(e, t), brute)
    assert metrics.auc(np.zeros(10), 0.1) == pytest.approx(1.0)
    assert metrics.auc(np.full(10, 1.0), 0.1) == pytest.approx(0.0)
    # uniform errors on [0, d]: the accuracy curve is x / d, area 1/2
    u = np.linspace(0, 0.1, 100001)
    assert metrics.auc(u, 0.1) == pytest.approx(0.5, abs=1e-4)


def test_reconstruction_error_is_the_nearest_observed_point():
    rng = np.random.default_rng(2)
    H, W, fx, fy, cx, cy = 24, 32, 30.0, 30.0, 16.0, 12.0
    depth = rng.uniform(1.0, 2.0, (H, W)) * (rng.random((H, W)) > 0.3)
    verts = rng.normal(0, 0.2, (50, 3)) + [0, 0, 1.5]
    vis = rng.random(50) > 0.4
    d = metrics.reconstruction_error(verts, vis, depth, fx, fy, cx, cy)
    pts = []
    for py in range(H):
        for px in range(W):
            z = depth[py, px]
            if z > 0:
                pts.append(((px - cx) * z / fx, (py - cy) * z / fy, z))
    pts = np.array(pts)
    brute = np.sqrt(((verts[vis][:, None, :] - pts[None]) ** 2).sum(-1)).min(1)
    assert np.allclose(d, brute, rtol=0, atol=1e-12)


def test_joint_links_are_the_bone_origins():
    m = synth.make_model(2, V=2000, width=64)
    j = metrics.joint_links(m["skeleton"])
    assert j[0] == 0 and len(j) == 22  # one per bone of the humanoid


@pytest.mark.parametrize("cfg", [1, 2])
def test_fk_joint_positions_match_the_oracle(cfg):
    from paper_1711_07999_gb300 import trk
    try:
        trk.lib()
    except Exception as e:
        pytest.skip(f"library unavailable: {e}")
    m = synth.make_model(cfg, V=1500, width=64)
    o = oracle.Oracle(m)
    rng = np.random.default_rng(cfg)
    for _ in range(3):
        th = synth.gt_theta(m, 0.3) + rng.normal(0, 0.2, o.L) * (m["skeleton"]["type"] == 0)
        p = trk.joint_positions(m["skeleton"], th)
        H0, _ = o.fk(th)
        r, dq = H0[:, :4], H0[:, 4:]
        # translation of the oracle's unit dual quaternions: 2 vec(d r*)
        rc = r * np.array([1, -1, -1, -1])
        t = np.stack([dq[:, 0] * rc[:, 1] + dq[:, 1] * rc[:, 0] + dq[:, 2] * rc[:, 3] - dq[:, 3] * rc[:, 2],
                      dq[:, 0] * rc[:, 2] - dq[:, 1] * rc[:, 3] + dq[:, 2] * rc[:, 0] + dq[:, 3] * rc[:, 1],
                      dq[:, 0] * rc[:, 3] + dq[:, 1] * rc[:, 2] - dq[:, 2] * rc[:, 1] + dq[:, 3] * rc[:, 0]], 1) * 2
        t /= (r ** 2).sum(1)[:, None]
        assert np.abs(p - t).max() < 1e-9
