"""The paper's evaluation measures (Sec. 5), computed on the host from tracked and ground-truth states:

- pose accuracy as a function of the distance threshold: the fraction of joints whose 3D position lies
  within d of the truth, for every d (instead of one threshold), summarised by the normalised area under
  that curve up to d_max;
- reconstruction error: for every visible model vertex, the distance to the nearest point of the
  observed depth (back-projected valid pixels).
"""
from __future__ import annotations

import numpy as np


def joint_links(skeleton: dict) -> np.ndarray:
    """Links that carry a joint: the root and every link whose fixed offset is not the identity (the other
    links of a multi-DoF joint share their predecessor's origin)."""
    off = np.asarray(skeleton["offset_dq"], np.float64)
    parent = np.asarray(skeleton["parent"])
    ident = np.all(np.abs(off - np.array([1, 0, 0, 0, 0, 0, 0, 0])) < 1e-12, axis=1)
    return np.nonzero((parent < 0) | ~ident)[0]


def joint_errors(p_est: np.ndarray, p_gt: np.ndarray) -> np.ndarray:
    """Euclidean distance of each estimated joint position to the truth (same shape but the last axis)."""
    return np.linalg.norm(np.asarray(p_est, np.float64) - np.asarray(p_gt, np.float64), axis=-1)


def accuracy_curve(errors, thresholds) -> np.ndarray:
    """Fraction of errors <= each threshold."""
    e = np.sort(np.asarray(errors, np.float64).ravel())
    if e.size == 0:
        return np.zeros(len(thresholds))
    return np.searchsorted(e, np.asarray(thresholds, np.float64), side="right") / e.size


def auc(errors, d_max: float, n: int = 1001) -> float:
    """Area under the accuracy curve on [0, d_max], normalised to [0, 1] (trapezoids on n thresholds)."""
    t = np.linspace(0.0, d_max, n)
    a = accuracy_curve(errors, t)
    return float(np.sum((a[1:] + a[:-1]) * 0.5 * np.diff(t)) / d_max)


def observed_points(depth: np.ndarray, fx: float, fy: float, cx: float, cy: float) -> np.ndarray:
    """Back-projection of the valid pixels: pixel (px, py) with depth z maps to ((px-cx) z/fx, (py-cy) z/fy, z)."""
    d = np.asarray(depth, np.float64)
    py, px = np.nonzero(d > 0)
    z = d[py, px]
    return np.stack([(px - cx) * z / fx, (py - cy) * z / fy, z], axis=1)


def reconstruction_error(verts: np.ndarray, visible: np.ndarray, depth: np.ndarray, fx: float, fy: float,
                         cx: float, cy: float) -> np.ndarray:
    """Distance from each visible vertex (camera frame) to the nearest observed point."""
    from scipy.spatial import cKDTree
    pts = observed_points(depth, fx, fy, cx, cy)
    v = np.asarray(verts, np.float64)[np.asarray(visible, bool)]
    if len(pts) == 0 or len(v) == 0:
        return np.zeros(0)
    dist, _ = cKDTree(pts).query(v, k=1)
    return dist
