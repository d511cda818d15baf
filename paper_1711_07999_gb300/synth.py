"""Seeded synthetic inputs: capsule bodies, kinematic trees, skin weights, motion and sensor noise.

These stand in for the paper's Kinect-v2 recordings and its hand-built 55k-vertex template (Sec. 3.3,
Sec. 5.1), which are not available.  The module builds the *inputs* of the tracker only: a kinematic
tree of 1-DoF links (Sec. 3.1: multi-DoF joints are chains of hinges), a triangle mesh of capsules in
the bind pose (Theta = 0, Sec. 3.2), sparse skin weights (<= 4 bones per vertex), ground-truth joint
trajectories and surface offsets, and the sensor noise applied to a rendered depth image.  It contains
none of the tracker's arithmetic (no skinning, rendering, association or solving): depth images are
rendered by whichever side consumes the model.

Workloads (seed = 17110799 + 1000 * config + session):
  config 1  12-bone tree (root 6-DoF + 11 revolute/ball joints), capsules of radius 3-8 cm and length
            10-40 cm, 5k vertices, 160x120 depth (fx = fy = 140), noise 1 mm quantised to 1 mm.
  config 2  22-bone humanoid (55 DoF), 50k vertices, 640x480 (fx = fy = 525), 300 frames at 30 fps of
            sinusoidal joint motion with a 1 m root translation, wrinkle offsets of 2-8 mm, depth noise
            1.5 mm * (z / 3 m)^2 and 2 % invalid pixels.
  config 3  the humanoid at 200k vertices, 1280x720 (fx = fy = 920).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 17110799


def seed_for(config: int, session: int = 0) -> int:
    return SEED_BASE + 1000 * config + session


# ------------------------------------------------------------------------------------------------
# parameters of the method (the readings of the paper's unstated constants)
# ------------------------------------------------------------------------------------------------
def default_params(fx: float, n_verts: int, tau: float = 0.05, z_min: float = 2.0, **over) -> dict:
    """lambda values, cutoff tau, window W = ceil(fx * tau / z_min) and the iteration schedule.
    The pose-prior weight grows with sqrt(|V|) (S_kk = n_k/|V| is a fraction, while the data term of
    J^T J grows with the number of vertices), so that the prior has the same relative strength at
    every mesh resolution: it dominates only directions the data do not observe (e.g. capsule twist)."""
    p = dict(pose_iters=10, shape_iters=2, shape_sweeps=1, window_half=int(math.ceil(fx * tau / z_min)), knn=4,
             lambda_k0=1e-3, lambda_s=0.005 * math.sqrt(n_verts), lambda_phi=1e-2, lambda_N=1e-1, lambda_w=1e-1,
             cutoff=tau,
             eps_vis=0.01, z_near=0.05)
    p.update(over)
    return p


# ------------------------------------------------------------------------------------------------
# bodies
# ------------------------------------------------------------------------------------------------
X, Y, Z = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)
ROOT_DOFS = [("p", X), ("p", Y), ("p", Z), ("h", X), ("h", Y), ("h", Z)]
BALL = [("h", X), ("h", Y), ("h", Z)]


def _bone(name, parent, pivot, p0, p1, radius, dofs):
    return dict(name=name, parent=parent, pivot=np.array(pivot, float), p0=np.array(p0, float),
                p1=np.array(p1, float), radius=float(radius), dofs=list(dofs))


def humanoid_bones() -> list:
    """22 bones; coordinates relative to the root pivot; camera frame: x right, y down, z forward."""
    b = [
        _bone("pelvis", -1, (0, 0, 0), (-0.09, 0, 0), (0.09, 0, 0), 0.09, ROOT_DOFS),
        _bone("spine1", 0, (0, -0.08, 0), (0, -0.08, 0), (0, -0.20, 0), 0.10, BALL),
        _bone("spine2", 1, (0, -0.22, 0), (0, -0.22, 0), (0, -0.34, 0), 0.11, BALL),
        _bone("chest", 2, (0, -0.36, 0), (-0.08, -0.45, 0), (0.08, -0.45, 0), 0.12, BALL),
        _bone("neck", 3, (0, -0.55, 0), (0, -0.55, 0), (0, -0.62, 0), 0.05, BALL),
        _bone("head", 4, (0, -0.64, 0), (0, -0.70, 0), (0, -0.80, 0), 0.09, BALL),
    ]
    for s in (-1.0, 1.0):  # left (x < 0), right
        side = "L" if s < 0 else "R"
        c0 = len(b)
        b += [
            _bone(side + "clavicle", 3, (0.04 * s, -0.50, 0), (0.04 * s, -0.50, 0), (0.16 * s, -0.50, 0), 0.05,
                  [("h", Y), ("h", Z)]),
            _bone(side + "upperarm", c0, (0.19 * s, -0.50, 0), (0.19 * s, -0.48, 0), (0.19 * s, -0.22, 0), 0.05, BALL),
            _bone(side + "forearm", c0 + 1, (0.19 * s, -0.20, 0), (0.19 * s, -0.20, 0), (0.19 * s, 0.04, 0), 0.04,
                  [("h", X), ("p", Y)]),
            _bone(side + "hand", c0 + 2, (0.19 * s, 0.06, 0), (0.19 * s, 0.06, 0), (0.19 * s, 0.14, 0), 0.035,
                  [("h", X), ("h", Z)]),
        ]
    for s in (-1.0, 1.0):
        side = "L" if s < 0 else "R"
        c0 = len(b)
        b += [
            _bone(side + "thigh", 0, (0.09 * s, 0.05, 0), (0.09 * s, 0.08, 0), (0.09 * s, 0.45, 0), 0.075, BALL),
            _bone(side + "shin", c0, (0.09 * s, 0.48, 0), (0.09 * s, 0.48, 0), (0.09 * s, 0.86, 0), 0.055,
                  [("h", X), ("p", Y)]),
            _bone(side + "foot", c0 + 1, (0.09 * s, 0.88, 0), (0.09 * s, 0.90, -0.02), (0.09 * s, 0.90, -0.14), 0.04,
                  [("h", X), ("h", Z)]),
            _bone(side + "toe", c0 + 2, (0.09 * s, 0.90, -0.15), (0.09 * s, 0.90, -0.15), (0.09 * s, 0.90, -0.20),
                  0.03, [("h", X)]),
        ]
    return b


def small_tree_bones(rng) -> list:
    """12 bones: root 6-DoF + 11 revolute / ball joints; radius U[3,8] cm, length U[10,40] cm."""
    L = lambda: rng.uniform(0.10, 0.40)
    R = lambda: rng.uniform(0.03, 0.08)
    b = []
    w = L()
    b.append(_bone("pelvis", -1, (0, 0, 0), (-w / 2, 0, 0), (w / 2, 0, 0), R(), ROOT_DOFS))
    top = np.zeros(3)
    chest_end = top
    for name in ("spine", "chest", "head"):
        l = L()
        b.append(_bone(name, len(b) - 1, top, top, top + (0, -l, 0), R(), BALL))
        top = top + (0, -l, 0)
        if name == "chest":
            chest_end = top
    for s in (-1.0, 1.0):
        d = np.array([0.3 * s, 1.0, 0.0]); d /= np.linalg.norm(d)
        piv = chest_end + np.array([0.12 * s, 0.10, 0])
        l1, l2 = L(), L()
        b.append(_bone(("L" if s < 0 else "R") + "upperarm", 2, piv, piv, piv + d * l1, R(), BALL))
        b.append(_bone(("L" if s < 0 else "R") + "forearm", len(b) - 1, piv + d * l1, piv + d * l1,
                       piv + d * (l1 + l2), R(), [("h", X)]))
    for s in (-1.0, 1.0):
        piv = np.array([w / 2 * s, 0.0, 0.0])
        l1, l2 = L(), L()
        b.append(_bone(("L" if s < 0 else "R") + "thigh", 0, piv, piv, piv + (0, l1, 0), R(), BALL))
        b.append(_bone(("L" if s < 0 else "R") + "shin", len(b) - 1, piv + (0, l1, 0), piv + (0, l1, 0),
                       piv + (0, l1 + l2, 0), R(), [("h", X)]))
    return b


def random_tree_bones(rng, n_bones: int, max_dof: int = 72) -> list:
    """n_bones capsules in a random tree: a 6-DoF root, then bones hung from the end of a random earlier
    bone (chains at most 5 deep) in a direction turned up to 60 degrees from the parent's, mostly in
    the image plane; each joint a ball (3 DoF), 2-DoF or hinge, with the total held to max_dof;
    radius U[2,6] cm, length U[6,18] cm."""
    w = rng.uniform(0.10, 0.20)
    b = [_bone("root", -1, (0, 0, 0), (-w / 2, 0, 0), (w / 2, 0, 0), rng.uniform(0.04, 0.07), ROOT_DOFS)]
    ends, dirs, depth = [np.zeros(3)], [np.array([0.0, -1.0, 0.0])], [0]
    budget = max_dof - 6
    for k in range(1, n_bones):
        cand = [i for i in range(len(b)) if depth[i] < 5]
        pa = int(rng.choice(cand))
        ang = rng.uniform(-math.pi / 3, math.pi / 3)
        d0 = dirs[pa] if pa > 0 else np.array([math.cos(rng.uniform(0, 2 * math.pi)), math.sin(rng.uniform(0, 2 * math.pi)), 0.0])
        c, s_ = math.cos(ang), math.sin(ang)
        d = np.array([c * d0[0] - s_ * d0[1], s_ * d0[0] + c * d0[1], rng.uniform(-0.2, 0.2)])
        d /= np.linalg.norm(d)
        length = rng.uniform(0.06, 0.18)
        piv = ends[pa]
        left = n_bones - 1 - k  # bones still to place after this one need at least one DoF each
        r = rng.random()
        nd = 3 if r < 0.4 else (2 if r < 0.7 else 1)
        nd = max(1, min(nd, budget - left))
        dofs = BALL if nd == 3 else ([("h", X), ("h", Z)] if nd == 2 else [("h", Z)])
        budget -= nd
        b.append(_bone(f"b{k}", pa, piv, piv, piv + d * length, rng.uniform(0.02, 0.06), dofs))
        ends.append(piv + d * length)
        dirs.append(d)
        depth.append(depth[pa] + 1)
    return b


def build_skeleton(bones: list, root_pos) -> tuple:
    """Links: one per DoF.  The first link of a bone carries the fixed offset H_{P(j),j} (a pure
    translation from the parent bone's pivot); the others have identity offsets.  The bone's capsule
    is attached to its last link.  Offsets are unit dual quaternions (1,0,0,0 | 0, t/2)."""
    parent, jtype, axis, offs, mask, link_of_bone, first_link = [], [], [], [], [], [], []
    for bi, bn in enumerate(bones):
        pb = bn["parent"]
        t = bn["pivot"] + (np.asarray(root_pos, float) if pb < 0 else -bones[pb]["pivot"])
        first_link.append(len(parent))
        for d, (kind, ax) in enumerate(bn["dofs"]):
            j = len(parent)
            parent.append((link_of_bone[pb] if pb >= 0 else -1) if d == 0 else j - 1)
            jtype.append(0 if kind == "h" else 1)
            axis.append(ax)
            tt = t if d == 0 else np.zeros(3)
            offs.append([1.0, 0.0, 0.0, 0.0, 0.0, tt[0] / 2, tt[1] / 2, tt[2] / 2])
            mask.append(0.0 if pb < 0 else 1.0)  # no pose prior on the root's 6 DoF
        link_of_bone.append(len(parent) - 1)
    sk = dict(parent=np.array(parent, np.int32), type=np.array(jtype, np.int32), axis=np.array(axis, np.float32),
              offset_dq=np.array(offs, np.float32), prior_mask=np.array(mask, np.float32))
    return sk, np.array(link_of_bone), np.array(first_link)


def _capsule(p0, p1, r, h):
    """Hemisphere-capped cylinder from p0 to p1, radius r, spacing ~h.  Returns (verts, tris, normals,
    axial coordinate from p0).  Triangles are counter-clockwise seen from outside."""
    d = p1 - p0
    length = float(np.linalg.norm(d))
    dirn = d / length
    hv = np.array(X) if abs(dirn[0]) < 0.9 else np.array(Y)
    e1 = hv - hv.dot(dirn) * dirn
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(dirn, e1)  # (e1, e2, dirn) right-handed
    S = max(8, int(round(2 * math.pi * r / h)))
    Lp = length + math.pi * r
    K = max(4, int(round(Lp / h)))
    verts, nrm, ax = [p0 - r * dirn], [-dirn], [-r]
    beta = 2 * math.pi * np.arange(S) / S
    radial = np.cos(beta)[:, None] * e1 + np.sin(beta)[:, None] * e2
    q = 0.5 * math.pi * r
    for k in range(1, K):
        s = k * Lp / K
        if s < q:
            a = s / r
            axial, rad, nd, nr = -r * math.cos(a), r * math.sin(a), -math.cos(a), math.sin(a)
        elif s < q + length:
            axial, rad, nd, nr = s - q, r, 0.0, 1.0
        else:
            a = (s - q - length) / r
            axial, rad, nd, nr = length + r * math.sin(a), r * math.cos(a), math.sin(a), math.cos(a)
        verts.extend(p0 + axial * dirn + rad * radial)
        nrm.extend(nd * dirn + nr * radial)
        ax.extend([axial] * S)
    verts.append(p1 + r * dirn)
    nrm.append(dirn)
    ax.append(length + r)
    tris = []
    ring = lambda k, m: 1 + (k - 1) * S + (m % S)
    for m in range(S):
        tris.append((0, ring(1, m + 1), ring(1, m)))
    for k in range(1, K - 1):
        for m in range(S):
            tris.append((ring(k, m), ring(k, m + 1), ring(k + 1, m)))
            tris.append((ring(k, m + 1), ring(k + 1, m + 1), ring(k + 1, m)))
    last = 1 + (K - 1) * S
    for m in range(S):
        tris.append((last, ring(K - 1, m), ring(K - 1, m + 1)))
    return np.array(verts), np.array(tris), np.array(nrm), np.array(ax), length, dirn


def _count(bones, h):
    n = 0
    for bn in bones:
        r = bn["radius"]
        length = float(np.linalg.norm(bn["p1"] - bn["p0"]))
        S = max(8, int(round(2 * math.pi * r / h)))
        K = max(4, int(round((length + math.pi * r) / h)))
        n += 2 + S * (K - 1)
    return n


def tessellate(bones: list, root_pos, target_V: int):
    """Capsule per bone at the bind pose, spacing chosen so that |V| is within 2 % of target_V."""
    lo, hi = 1e-4, 1.0
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if _count(bones, mid) > target_V:
            lo = mid
        else:
            hi = mid
    h = lo if abs(_count(bones, lo) - target_V) < abs(_count(bones, hi) - target_V) else hi
    V, T, N, B, A = [], [], [], [], []
    for bi, bn in enumerate(bones):
        rp = np.asarray(root_pos, float)
        v, t, n, a, length, dirn = _capsule(bn["p0"] + rp, bn["p1"] + rp, bn["radius"], h)
        T.append(t + sum(len(x) for x in V))
        V.append(v); N.append(n); B.append(np.full(len(v), bi)); A.append(a)
    return np.concatenate(V), np.concatenate(T), np.concatenate(N), np.concatenate(B)


def skin_weights(bones, root_pos, verts, bone_of, link_of_bone):
    """Own bone weight 1; the parent bone and each child bone get exp(-s^2 / (2 sigma^2)) with s the
    axial distance (along the bone's capsule axis) to the shared joint and sigma = 0.15 * capsule
    length.  The 4 largest are kept and renormalised."""
    rp = np.asarray(root_pos, float)
    children = {i: [c for c, b in enumerate(bones) if b["parent"] == i] for i in range(len(bones))}
    V = len(verts)
    idx = np.zeros((V, 4), np.uint8)
    w = np.zeros((V, 4), np.float32)
    for bi, bn in enumerate(bones):
        sel = np.nonzero(bone_of == bi)[0]
        x = verts[sel]
        d = bn["p1"] - bn["p0"]
        length = float(np.linalg.norm(d))
        dirn = d / length
        sigma = 0.15 * length
        cand = [(np.ones(len(sel)), link_of_bone[bi])]
        if bn["parent"] >= 0:
            s = (x - (bn["pivot"] + rp)) @ dirn
            cand.append((np.exp(-s * s / (2 * sigma * sigma)), link_of_bone[bn["parent"]]))
        for c in children[bi]:
            s = (x - (bones[c]["pivot"] + rp)) @ dirn
            cand.append((np.exp(-s * s / (2 * sigma * sigma)), link_of_bone[c]))
        ws = np.stack([c[0] for c in cand], 1)
        ls = np.array([c[1] for c in cand])
        order = np.argsort(-ws, axis=1, kind="stable")[:, :4]
        top = np.take_along_axis(ws, order, 1)
        top = top / top.sum(1, keepdims=True)
        k = top.shape[1]
        w[sel, :k] = top.astype(np.float32)
        idx[sel, :k] = ls[order].astype(np.uint8)
    # renormalise in float32 so the stored weights sum to 1 within float rounding
    w = (w / w.sum(1, keepdims=True)).astype(np.float32)
    return idx, w


# ------------------------------------------------------------------------------------------------
# workloads
# ------------------------------------------------------------------------------------------------
CONFIGS = {
    1: dict(width=160, height=120, fx=140.0, fy=140.0, cx=80.0, cy=60.0, V=5000, root_z=2.5, body="small"),
    2: dict(width=640, height=480, fx=525.0, fy=525.0, cx=320.0, cy=240.0, V=50000, root_z=3.0, body="humanoid"),
    3: dict(width=1280, height=720, fx=920.0, fy=920.0, cx=640.0, cy=360.0, V=200000, root_z=3.0, body="humanoid"),
}
# the uneven batch: per session, |V| ~ U[5k, 200k], bones ~ U{12..40} (DoF <= 72), one of three images
BATCH_IMAGES = [dict(width=320, height=240, fx=262.5, fy=262.5, cx=160.0, cy=120.0),
                dict(width=640, height=480, fx=525.0, fy=525.0, cx=320.0, cy=240.0),
                dict(width=1280, height=720, fx=920.0, fy=920.0, cx=640.0, cy=360.0)]


def batch_session_config(session: int) -> dict:
    """Size class of session `session` of the uneven batch (seeded per session)."""
    rng = np.random.default_rng(seed_for(4, session))
    c = dict(BATCH_IMAGES[int(rng.integers(0, 3))])
    c.update(V=int(rng.integers(5000, 200001)), bones=int(rng.integers(12, 41)), root_z=3.0, body="random")
    return c


def make_model(config: int = 1, session: int = 0, V: int | None = None, width: int | None = None,
               height: int | None = None, **param_over) -> dict:
    """Template model + camera + parameters + ground-truth motion description for one session."""
    c = dict(CONFIGS[config]) if config != 4 else batch_session_config(session)
    if width is not None:
        s = width / c["width"]
        c.update(width=width, height=height if height is not None else int(round(c["height"] * s)),
                 fx=c["fx"] * s, fy=c["fy"] * s)
        c.update(cx=c["width"] / 2.0, cy=c["height"] / 2.0)
    if V is not None:
        c["V"] = V
    seed = seed_for(config, session)
    rng = np.random.default_rng(seed)
    if c["body"] == "small":
        bones = small_tree_bones(rng)
    elif c["body"] == "random":
        bones = random_tree_bones(rng, c["bones"])
    else:
        bones = humanoid_bones()
    root = (0.0, 0.2 if c["body"] == "small" else 0.0, c["root_z"])
    sk, link_of_bone, first_link = build_skeleton(bones, root)
    verts, tris, nrm0, bone_of = tessellate(bones, root, c["V"])
    bidx, bw = skin_weights(bones, root, verts, bone_of, link_of_bone)
    L = len(sk["parent"])
    # motion: per link, 3 sinusoids (Hz in [0.2, 2]); amplitudes by joint kind
    amp = np.zeros((L, 3))
    twist = np.zeros(L, bool)  # a hinge about the capsule's own axis moves nothing the camera can see
    for bi, bn in enumerate(bones):
        cd = (bn["p1"] - bn["p0"]) / np.linalg.norm(bn["p1"] - bn["p0"])
        for d, (kind, ax) in enumerate(bn["dofs"]):
            j = first_link[bi] + d
            twist[j] = kind == "h" and abs(float(np.dot(ax, cd))) > 0.9 and bn["parent"] >= 0
            if twist[j]:
                continue
            if bn["parent"] < 0:
                amp[j] = rng.uniform(0, math.radians(4), 3) if kind == "h" else rng.uniform(0, 0.01, 3)
            else:
                amp[j] = rng.uniform(0, math.radians(15), 3) if kind == "h" else rng.uniform(0, 0.004, 3)
    freq = rng.uniform(0.2, 2.0, (L, 3))
    phase = rng.uniform(0, 2 * math.pi, (L, 3))
    # wrinkles: delta_i = sum_m a_m sin(2 pi <d_m, v0_i> / lambda_m + psi_m + 2 pi f'_m t)
    amin, amax = (0.002, 0.005) if config == 1 else (0.002, 0.008)
    dm = rng.normal(size=(3, 3))
    dm /= np.linalg.norm(dm, axis=1, keepdims=True)
    wr = dict(a=rng.uniform(amin, amax, 3), d=dm, lam=rng.uniform(0.05, 0.20, 3), psi=rng.uniform(0, 2 * math.pi, 3),
              f=rng.uniform(0.2, 2.0, 3) if config != 1 else np.zeros(3))
    # config 1: one static pose, hinges U[+-30 deg]
    static_theta = np.zeros(L)
    for j in range(L):
        if sk["type"][j] == 0 and not twist[j]:
            static_theta[j] = rng.uniform(-math.radians(30), math.radians(30))
    start_pert = np.zeros(L)
    for j in range(L):
        if sk["type"][j] == 0 and not twist[j]:
            start_pert[j] = rng.uniform(-math.radians(10), math.radians(10))
    root_links = [first_link[0] + d for d in range(len(bones[0]["dofs"]))]
    camera = dict(width=c["width"], height=c["height"], fx=c["fx"], fy=c["fy"], cx=c["cx"], cy=c["cy"])
    params = default_params(c["fx"], len(verts), **param_over)
    mesh = dict(verts=verts.astype(np.float32), tris=tris.astype(np.int32), bone_idx=bidx, bone_w=bw)
    motion = dict(config=config, amp=amp, freq=freq, phase=phase, wrinkle=wr, static_theta=static_theta,
                  start_pert=start_pert, root_links=root_links, bind_normals=nrm0, seed=seed)
    return dict(skeleton=sk, mesh=mesh, camera=camera, params=params, motion=motion, bones=bones)


def gt_theta(model: dict, t: float) -> np.ndarray:
    """Ground-truth joint values at time t (s)."""
    mo = model["motion"]
    if mo["config"] == 1:
        return mo["static_theta"].copy()
    th = (mo["amp"] * np.sin(2 * math.pi * mo["freq"] * t + mo["phase"])).sum(1)
    th = np.clip(th, -math.radians(45), math.radians(45))
    tx = mo["root_links"][0]
    th[tx] = -0.5 + t / 10.0  # the root translates 1 m along +x over 10 s
    return th


def gt_offsets(model: dict, t: float) -> np.ndarray:
    """Ground-truth surface offsets phi_i = delta_i(t) n0_i (bind-pose normal of the capsule)."""
    wr = model["motion"]["wrinkle"]
    v0 = model["mesh"]["verts"].astype(np.float64)
    arg = 2 * math.pi * (v0 @ wr["d"].T) / wr["lam"] + wr["psi"] + 2 * math.pi * wr["f"] * t
    delta = (wr["a"] * np.sin(arg)).sum(1)
    return delta[:, None] * model["motion"]["bind_normals"]


def start_theta(model: dict) -> np.ndarray:
    """Tracking start: config 1 = ground truth + U[+-10 deg] on each hinge; otherwise the frame-0 truth."""
    th = gt_theta(model, 0.0)
    if model["motion"]["config"] == 1:
        th = th + model["motion"]["start_pert"]
    return th


def add_noise(depth: np.ndarray, config: int, rng) -> np.ndarray:
    """Sensor model applied to a rendered depth image (0 = no return)."""
    d = np.array(depth, np.float64)
    valid = d > 0
    if config == 1:
        d = np.where(valid, np.round((d + rng.normal(0, 0.001, d.shape)) * 1000.0) / 1000.0, 0.0)
    else:
        sig = 0.0015 * (d / 3.0) ** 2
        d = np.where(valid, d + rng.normal(size=d.shape) * sig, 0.0)
        drop = rng.random(d.shape) < 0.02
        d[drop] = 0.0
    d[d < 0] = 0.0
    return d.astype(np.float32)
