"""Frame-by-frame parity driver (test infrastructure): one frame of a GPU session, stepped through the
C ABI, in lockstep with the FP64 oracle from the same state.

Why lockstep.  The association is an argmin (Sec. 4.1); where the two best candidates of a pixel lie
within ~1e-7 m of each other, FP32 and FP64 distances can order them differently.  Both choices are
correct answers to within the tie tolerance of the correspondence maps (1e-5 m), but the frame's later
iterations start from the chosen one, and the method amplifies such a change: a pixel that moves to the
neighbouring vertex moves both vertices' residuals by up to the pixel spacing, and joint values the
energy barely constrains (a capsule's twist about its own axis) follow it by up to ~1e-2 rad within a
frame.  So at every iteration the oracle computes its own association with its tie flags; at pixels
where the GPU chose differently, the pixel must be a flagged tie and the GPU's vertex a valid near
argmin (see merge_association), and the oracle continues from the GPU's choice there.  Everything that is unique -- every other correspondence, the LM decisions,
the energies, Theta, Phi and lambda -- is then compared with the stated tolerances.

The GPU path is stepped with the step-level calls (the same kernels in the same order as the frame
graph); ``graph_frame`` checks that the frame graph gives bitwise the same results.
"""
from __future__ import annotations

import struct

import numpy as np

import oracle

TIE_M = 1e-5  # correspondence tie tolerance: two candidates closer than this are a tie (Sec. 4.1)


def state_blob(theta, lam, phi, frames_done=1) -> bytes:
    """A trk_session_import blob (format 1: 'TRKSTATE', version, links, vertices, frames since set_pose;
    Theta f64 [L], lambda f64, Phi float4 [V]) holding the given state."""
    th = np.ascontiguousarray(theta, np.float64)
    ph = np.asarray(phi, np.float32).reshape(-1, 3)
    p4 = np.zeros((len(ph), 4), np.float32)
    p4[:, :3] = ph
    head = b"TRKSTATE" + struct.pack("<4i", 1, len(th), len(ph), int(frames_done))
    return head + th.tobytes() + struct.pack("<d", float(lam)) + p4.tobytes()


def _pixel_points(o, depth, ks):
    """Back-projected points p_k of the pixels ks, exactly as the oracle forms them (FP64)."""
    W = o.W
    px, py = (ks % W).astype(np.float64), (ks // W).astype(np.float64)
    d = np.asarray(depth, np.float32).ravel()[ks].astype(np.float64)
    return np.stack([(px - o.cx) * d / o.fx, (py - o.cy) * d / o.fy, d], axis=1)


def merge_association(o, depth, R, corr_g):
    """The oracle's correspondence map (pass R of Oracle.pass_at with ties) with the GPU's choices taken
    at flagged ties.  Returns the merged map and (non-tie mismatches, tie flips, invalid flips).  A flip
    is valid when the GPU's vertex g is a candidate the oracle could have taken up to the tolerance:
    visible or marginally visible, within the cutoff + TIE_M, and within TIE_M of the oracle's best
    distance unless the oracle's vertex is itself marginal (its visibility or bucket decided within
    TIE_M); a pixel the GPU leaves unassociated needs the oracle's best within TIE_M of the cutoff or a
    marginal best vertex."""
    co, cg = R["corr"].ravel(), np.asarray(corr_g).ravel()
    tie = R["tie"].ravel() > 0
    v, vis, marg = R["v"], R["vis"] > 0, R["marg"] > 0
    mism = co != cg
    flips = np.flatnonzero(mism & tie)
    invalid = 0
    if flips.size:
        p = _pixel_points(o, depth, flips)
        g, b = cg[flips], co[flips]
        tau = float(o.params["cutoff"])
        gi, bi = np.maximum(g, 0), np.maximum(b, 0)
        dg = np.where(g >= 0, np.linalg.norm(p - v[gi], axis=1), np.inf)
        db = np.where(b >= 0, np.linalg.norm(p - v[bi], axis=1), tau)
        b_marg = (b >= 0) & marg[bi]
        ok_g = (g >= 0) & (vis[gi] | marg[gi]) & (dg <= tau + TIE_M) & ((dg <= db + TIE_M) | b_marg)
        ok_none = (g < 0) & ((db >= tau - TIE_M) | b_marg)
        invalid = int((~(ok_g | ok_none)).sum())
    merged = np.where(mism & tie, cg, co)
    return merged, int((mism & ~tie).sum()), int(flips.size), invalid


def follow_frame(o, s, depth, theta, phi, lam, frames_done=1, matched_energy=True):
    """One frame (R18: pose_iters LM iterations, then shape_iters shape iterations) of session s and of
    the oracle o from the state (theta, phi [V,3] float32, lam), the oracle following the GPU at flagged
    ties.  Returns per-iteration records and both final states."""
    P, S = o.params["pose_iters"], o.params["shape_iters"]
    phi32 = np.asarray(phi, np.float32).reshape(-1, 3)
    s.import_state(state_blob(theta, lam, phi32, frames_done))
    s.set_depth(depth)
    th_o, ph_o, lam_o = np.array(theta, np.float64), phi32.astype(np.float64), float(lam)
    recs = []
    for it in range(P + S):
        th_g, ph_g = s.read("THETA"), s.read("PHI")[:, :3].astype(np.float64)
        for st in ("skin", "raster", "visibility", "associate"):
            s.step(st)
        corr_g = s.read("CORR")
        R = o.pass_at(th_o, ph_o, depth, with_ties=True)
        corr, nontie, flips, invalid = merge_association(o, depth, R, corr_g)
        rec = dict(iteration=it, nontie=nontie, flips=flips, invalid_flips=invalid,
                   tie_frac=float((R["tie"] > 0).mean()), valid_px=int((np.asarray(depth) > 0).sum()))
        acc, cnt = o.accumulate(R["v"], depth, corr)
        r, inA, E_o = o.residuals(th_o, R["n"], R["nvalid"], acc, cnt)
        if matched_energy:  # the oracle at the GPU's own state and correspondence map
            v_m, _ = o.skin(th_g, ph_g)
            n_m, ok_m = o.normals(v_m)
            acc_m, cnt_m = o.accumulate(v_m, depth, corr_g)
            r_m, inA_m, E_m = o.residuals(th_g, n_m, ok_m, acc_m, cnt_m)
        if it < P:
            s.step("normal_equations")
            rec["E_gpu"] = float(s.read("ENERGY")[0])
            s.step("lm")
            rec["a_gpu"] = int(s.read("LM_TRIALS")[7])
            J = o.jacobian(th_o, ph_o, R["n"], inA)
            JTJ, JTr = oracle.normal_eq(J, r, inA)
            o.set_state(th_o, ph_o, lam_o)
            a_o, th_o, lam_o, _ = o.lm_step(JTJ, JTr, E_o, R["v"], R["n"], acc, cnt, inA, th_o, lam_o)
            rec["a_oracle"] = int(a_o)
            if matched_energy:
                rec["E_matched"] = float(E_m)
        else:
            s.step("shape")
            rec["E_gpu"] = float(s.read("ENERGY")[P])
            E_s, ph_o, _, _ = o.shape_step(th_o, ph_o, R["n"], acc, cnt, inA)
            if matched_energy:
                rec["E_matched"] = float(o.shape_step(th_g, ph_g, n_m, acc_m, cnt_m, inA_m)[0])
        rec["E_oracle"] = float(E_o) if it < P else float(E_s)
        recs.append(rec)
    return dict(records=recs, theta_gpu=s.read("THETA"), phi_gpu=s.read("PHI")[:, :3].astype(np.float64),
                lam_gpu=float(s.read("LAMBDA")[0]), theta_oracle=th_o, phi_oracle=ph_o, lam_oracle=lam_o)


def graph_frame(s, depth, theta, phi, lam, frames_done=1):
    """The same frame through the frame graph (trk_track_frame) from the same imported state."""
    s.import_state(state_blob(theta, lam, phi, frames_done))
    return s.track_frame(depth)


def summary(res):
    """Largest deviations of one followed frame (the figures the tests bound and the benchmark reports)."""
    recs = res["records"]
    dth = np.abs(res["theta_gpu"] - res["theta_oracle"])
    dphi = np.abs(res["phi_gpu"] - res["phi_oracle"]).max(axis=1)
    em = [abs(r["E_gpu"] - r["E_matched"]) / r["E_matched"] for r in recs if "E_matched" in r]
    return dict(theta_rad_max=float(dth.max()), offsets_mm_max=float(1e3 * dphi.max()),
                energy_rel_max_matched=float(max(em)) if em else float("nan"),
                nontie_mismatches=int(sum(r["nontie"] for r in recs)),
                tie_flips=int(sum(r["flips"] for r in recs)),
                invalid_flips=int(sum(r["invalid_flips"] for r in recs)),
                tie_flagged_frac=float(np.mean([r["tie_frac"] for r in recs])),
                lm_decisions_equal=all(r["a_gpu"] == r["a_oracle"] for r in recs if "a_gpu" in r),
                lambda_equal=res["lam_gpu"] == res["lam_oracle"])
