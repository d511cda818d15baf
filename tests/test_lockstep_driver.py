"""The lockstep comparator (tests/sequence.py) on hand-built cases: which differences between the GPU's
correspondence map and the oracle's it accepts as tie flips, which it counts as mismatches, and the
session-state blob it imports.  CPU only (the oracle; no device)."""
import struct

import numpy as np

import oracle
from tests import helpers as H
from tests import sequence as seq

# camera fx = fy = 100, principal point (15, 15); the pixel (15, 15) at depth 2 has p = (0, 0, 2)
K = 15 * 31 + 15
VERTS = np.array([[0.004, 0.0, 2.0],          # 0: visible, 4 mm from p: the oracle's argmin
                  [0.0, 0.004 + 5e-6, 2.0],   # 1: visible, 5 um farther than 0
                  [0.0, -0.010, 2.0],         # 2: visible, 6 mm farther than 0
                  [-0.004 - 3e-6, 0.0, 2.0],  # 3: hidden but marginal, 3 um farther than 0
                  [0.004002 * 0.5 ** 0.5, -0.004002 * 0.5 ** 0.5, 2.0],  # 4: hidden, not marginal, 2 um farther
                  [0.0, 0.3, 2.0]])           # 5: far away


def _model(cutoff=0.05):
    n = len(VERTS)
    return H.make_model([-1], [0], [[0, 0, 1]], [[0, 0, 0]], VERTS, [[0, 1, 2]], [[0, 0, 0, 0]] * n,
                        [[1, 0, 0, 0]] * n, W=31, H=31, fx=100.0, fy=100.0, cx=15.0, cy=15.0, window_half=2,
                        cutoff=cutoff)


def _R(best, tie=1, vis=(1, 1, 1, 0, 0, 1), marg=(0, 0, 0, 1, 0, 0)):
    corr = -np.ones((31, 31), np.int32)
    corr.ravel()[K] = best
    t = np.zeros((31, 31), np.int32)
    t.ravel()[K] = tie
    return dict(corr=corr, tie=t, v=VERTS.astype(np.float64), vis=np.array(vis, np.int32),
                marg=np.array(marg, np.int32))


def _depth():
    d = np.zeros((31, 31), np.float32)
    d[15, 15] = 2.0
    return d


def _merge(o, R, gpu):
    g = R["corr"].copy()
    g.ravel()[K] = gpu
    merged, nontie, flips, invalid = seq.merge_association(o, _depth(), R, g)
    return int(merged.ravel()[K]), nontie, flips, invalid


def test_flips_at_ties_to_a_valid_near_argmin_are_taken():
    o = oracle.Oracle(_model())
    assert _merge(o, _R(0), 0) == (0, 0, 0, 0)   # the same choice
    assert _merge(o, _R(0), 1) == (1, 0, 1, 0)   # visible, 5 um farther: a valid flip, the oracle follows
    assert _merge(o, _R(0), 3) == (3, 0, 1, 0)   # hidden but marginal, 3 um farther: valid


def test_flips_that_no_rounding_explains_are_invalid():
    o = oracle.Oracle(_model())
    assert _merge(o, _R(0), 2)[1:] == (0, 1, 1)   # 6 mm farther
    assert _merge(o, _R(0), 4)[1:] == (0, 1, 1)   # as near, but neither visible nor marginal
    assert _merge(o, _R(0), 5)[1:] == (0, 1, 1)   # far away
    assert _merge(o, _R(0), -1)[1:] == (0, 1, 1)  # none, where the argmin is 4 mm away and not marginal


def test_a_marginal_argmin_excuses_any_choice_near_it_and_none():
    o = oracle.Oracle(_model())
    R = _R(3, vis=(1, 1, 1, 1, 0, 1))  # the oracle's argmin is vertex 3 itself, marginal
    assert _merge(o, R, -1)[1:] == (0, 1, 0)
    assert _merge(o, R, 2)[1:] == (0, 1, 0)
    assert _merge(o, R, 5)[1:] == (0, 1, 1)   # but not a vertex beyond the cutoff


def test_none_against_the_cutoff():
    # the oracle finds nothing within the cutoff; the GPU may take a vertex within 1e-5 m beyond it
    d0 = float(np.hypot(0.004, 0.0))
    o = oracle.Oracle(_model(cutoff=d0 - 5e-6))
    assert _merge(o, _R(-1), 0)[1:] == (0, 1, 0)
    o = oracle.Oracle(_model(cutoff=d0 - 5e-5))
    assert _merge(o, _R(-1), 0)[1:] == (0, 1, 1)


def test_differences_at_pixels_not_flagged_are_mismatches():
    o = oracle.Oracle(_model())
    assert _merge(o, _R(0, tie=0), 1) == (0, 1, 0, 0)   # counted, and the oracle keeps its own choice
    assert _merge(o, _R(0, tie=0), 0) == (0, 0, 0, 0)


def test_state_blob_layout():
    th = np.array([0.5, -1.25, 3.0])
    phi = np.array([[1e-3, 2e-3, 3e-3], [4e-3, 5e-3, 6e-3]], np.float32)
    b = seq.state_blob(th, 0.125, phi, frames_done=7)
    assert b[:8] == b"TRKSTATE"
    assert struct.unpack("<4i", b[8:24]) == (1, 3, 2, 7)
    assert np.array_equal(np.frombuffer(b[24:48], np.float64), th)
    assert struct.unpack("<d", b[48:56]) == (0.125,)
    p4 = np.frombuffer(b[56:], np.float32).reshape(2, 4)
    assert np.array_equal(p4[:, :3], phi) and not p4[:, 3].any()
    assert len(b) == 56 + 2 * 16


def test_summary_reports_the_largest_deviations():
    recs = [dict(nontie=0, flips=2, invalid_flips=0, tie_frac=0.01, E_gpu=1.0, E_matched=1.0 + 1e-6,
                 a_gpu=0, a_oracle=0),
            dict(nontie=1, flips=0, invalid_flips=0, tie_frac=0.03, E_gpu=2.0, E_matched=2.0, a_gpu=1,
                 a_oracle=0)]
    res = dict(records=recs, theta_gpu=np.array([0.0, 1e-4]), theta_oracle=np.array([0.0, 0.0]),
               phi_gpu=np.zeros((2, 3)), phi_oracle=np.array([[0.0, 0.0, 2e-7], [0.0, 0.0, 0.0]]),
               lam_gpu=1e-3, lam_oracle=1e-3)
    sm = seq.summary(res)
    assert sm["theta_rad_max"] == 1e-4
    assert abs(sm["offsets_mm_max"] - 2e-4) < 1e-12
    assert abs(sm["energy_rel_max_matched"] - 1e-6 / (1.0 + 1e-6)) < 1e-15
    assert sm["nontie_mismatches"] == 1 and sm["tie_flips"] == 2 and sm["invalid_flips"] == 0
    assert abs(sm["tie_flagged_frac"] - 0.02) < 1e-15
    assert not sm["lm_decisions_equal"] and sm["lambda_equal"]
