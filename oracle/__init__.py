"""FP64 CPU oracle of the per-frame tracker (Walsman et al., 3DV 2017, Secs. 3-4).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The product path (``paper_1711_07999_gb300``) never imports this
package.  The arithmetic lives in ``oracle.c`` (plain C, FP64, single-threaded); this module compiles
it with gcc and marshals numpy arrays through ctypes.

Functions with no pin other than agreement with a second computation are listed as "parity unpinned"
in the repository's design notes; every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, IEEE FP64: no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("pose_iters", C.c_int32), ("shape_iters", C.c_int32), ("shape_sweeps", C.c_int32),
                ("window_half", C.c_int32), ("knn", C.c_int32), ("shape_solver", C.c_int32),
                ("lambda_k0", C.c_double), ("lambda_s", C.c_double), ("lambda_phi", C.c_double),
                ("lambda_N", C.c_double), ("lambda_w", C.c_double), ("cutoff", C.c_double),
                ("eps_vis", C.c_double), ("z_near", C.c_double), ("association", C.c_int32), ("pad2_", C.c_int32)]


def _P(t):
    return np.ctypeslib.ndpointer(dtype=t, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        f64, f32, i32, u8 = _P(np.float64), _P(np.float32), _P(np.int32), _P(np.uint8)
        vp, ci, cd = C.c_void_p, C.c_int, C.c_double
        sig = {
            "orc_create": (vp, [ci, i32, i32, f32, f32, f32, ci, f32, ci, i32, u8, f32, ci, ci, cd, cd, cd, cd,
                                C.POINTER(Params)]),
            "orc_destroy": (None, [vp]),
            "orc_set_state": (None, [vp, f64, f64, cd]),
            "orc_get_state": (None, [vp, f64, f64, C.POINTER(C.c_double)]),
            "orc_get_derived": (None, [vp, f64, f64, i32]),
            "orc_fk": (None, [vp, f64, f64, f64]),
            "orc_skin": (None, [vp, f64, f64, f64, f64]),
            "orc_normals": (None, [ci, ci, i32, f64, f64, i32]),
            "orc_raster": (None, [ci, ci, cd, cd, cd, cd, cd, ci, f64, ci, i32, f64, i32, vp]),
            "orc_visibility": (None, [vp, f64, f64, i32, f64, vp, i32, i32, vp]),
            "orc_associate": (None, [vp, f64, i32, i32, vp, f32, i32, f64, i32, vp]),
            "orc_associate_rid": (None, [vp, f64, i32, vp, f32, i32, f64, i32, vp]),
            "orc_subdivide_counts": (None, [ci, ci, i32, i32, ci, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
            "orc_subdivide": (None, [ci, ci, i32, i32, ci, f64, ci, f64, i32]),
            "orc_accumulate": (None, [vp, f64, f32, i32, f64, i32]),
            "orc_residuals": (cd, [vp, f64, f64, i32, f64, i32, f64, i32]),
            "orc_jacobian": (None, [vp, f64, f64, f64, i32, f64]),
            "orc_normal_eq": (None, [ci, ci, f64, f64, i32, f64, f64]),
            "orc_cholesky_solve": (ci, [ci, f64, f64, f64]),
            "orc_solve3": (ci, [f64, f64, f64]),
            "orc_lm_step": (ci, [vp, f64, f64, cd, f64, f64, f64, i32, i32, f64, C.POINTER(C.c_double), f64]),
            "orc_shape_step": (cd, [vp, f64, f64, f64, f64, i32, i32, vp, vp]),
            "orc_render": (None, [vp, f64, f64, f64]),
            "orc_track_frame": (ci, [vp, f32, f64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def raster(W, H, fx, fy, cx, cy, znear, v, tris, with_amb=False):
    """Z-buffer (R5, R6): returns (z [H,W] with +inf where empty, tri id [H,W] with -1, ambiguity or None)."""
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    z = np.empty(W * H, np.float64)
    zt = np.empty(W * H, np.int32)
    amb = np.empty(W * H, np.int32) if with_amb else None
    lib().orc_raster(W, H, fx, fy, cx, cy, znear, len(v), v, len(tris), tris, z, zt, _ptr(amb))
    return z.reshape(H, W), zt.reshape(H, W), None if amb is None else amb.reshape(H, W)


def normals(v, tris):
    v = np.ascontiguousarray(v, np.float64).reshape(-1, 3)
    tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    n = np.empty_like(v)
    ok = np.empty(len(v), np.int32)
    lib().orc_normals(len(v), len(tris), tris, v, n, ok)
    return n, ok


def cholesky_solve(M, b):
    M = np.ascontiguousarray(M, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    rc = lib().orc_cholesky_solve(len(b), M, b, x)
    return x if rc == 0 else None


def solve3(M, b):
    x = np.zeros(3)
    rc = lib().orc_solve3(np.ascontiguousarray(M, np.float64).ravel(), np.ascontiguousarray(b, np.float64), x)
    return x if rc == 0 else None


def subdivide(face_off, face_vert, attr, levels):
    """Catmull-Clark subdivision (the paper's template construction) of the polygons (CSR face_off /
    face_vert) carrying per-vertex attributes attr [V][A]; returns (attributes [V'][A], quads [Q][4])."""
    fo = np.ascontiguousarray(face_off, np.int32)
    fv = np.ascontiguousarray(face_vert, np.int32)
    a = np.ascontiguousarray(attr, np.float64)
    V, A = a.shape
    F = len(fo) - 1
    nv, nq = C.c_int32(), C.c_int32()
    lib().orc_subdivide_counts(V, F, fo, fv, levels, C.byref(nv), C.byref(nq))
    out = np.empty((nv.value, A))
    quads = np.empty((nq.value, 4), np.int32)
    lib().orc_subdivide(V, F, fo, fv, A, a, levels, out, quads)
    return out, quads


def normal_eq(J, r, inA):
    J = np.ascontiguousarray(J, np.float64)
    V, L = J.shape
    JTJ = np.empty((L, L))
    JTr = np.empty(L)
    lib().orc_normal_eq(V, L, J, np.ascontiguousarray(r, np.float64), np.ascontiguousarray(inA, np.int32), JTJ, JTr)
    return JTJ, JTr


class Oracle:
    """One tracking session of the FP64 oracle.  ``model`` is a dict as produced by
    ``paper_1711_07999_gb300.synth`` (skeleton, mesh, camera, params)."""

    def __init__(self, model):
        sk, me, cam, pr = model["skeleton"], model["mesh"], model["camera"], model["params"]
        self.L = int(len(sk["parent"]))
        self.V = int(len(me["verts"]))
        self.F = int(len(me["tris"]))
        self.W, self.H = int(cam["width"]), int(cam["height"])
        self.fx, self.fy, self.cx, self.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
        self.params = pr
        p = Params(pose_iters=pr["pose_iters"], shape_iters=pr["shape_iters"], shape_sweeps=pr["shape_sweeps"],
                   window_half=pr["window_half"], knn=pr["knn"], shape_solver=pr.get("shape_solver", 0),
                   lambda_k0=pr["lambda_k0"],
                   lambda_s=pr["lambda_s"], lambda_phi=pr["lambda_phi"], lambda_N=pr["lambda_N"],
                   lambda_w=pr["lambda_w"], cutoff=pr["cutoff"], eps_vis=pr["eps_vis"], z_near=pr["z_near"],
                   association=pr.get("association", 0), pad2_=0)
        self._keep = dict(
            parent=np.ascontiguousarray(sk["parent"], np.int32), type=np.ascontiguousarray(sk["type"], np.int32),
            axis=np.ascontiguousarray(sk["axis"], np.float32), off=np.ascontiguousarray(sk["offset_dq"], np.float32),
            mask=np.ascontiguousarray(sk["prior_mask"], np.float32), verts=np.ascontiguousarray(me["verts"], np.float32),
            tris=np.ascontiguousarray(me["tris"], np.int32), bidx=np.ascontiguousarray(me["bone_idx"], np.uint8),
            bw=np.ascontiguousarray(me["bone_w"], np.float32))
        k = self._keep
        self.tris = k["tris"]
        self.h = lib().orc_create(self.L, k["parent"], k["type"], k["axis"], k["off"], k["mask"], self.V, k["verts"],
                                  self.F, k["tris"], k["bidx"], k["bw"], self.W, self.H, self.fx, self.fy, self.cx,
                                  self.cy, C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the model")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # state -----------------------------------------------------------------------------------------
    def set_state(self, theta, phi=None, lam=None):
        th = np.ascontiguousarray(theta, np.float64)
        ph = np.zeros((self.V, 3)) if phi is None else np.ascontiguousarray(phi, np.float64).reshape(self.V, 3)
        lib().orc_set_state(self.h, th, np.ascontiguousarray(ph), self.params["lambda_k0"] if lam is None else lam)

    def get_state(self):
        th = np.empty(self.L)
        ph = np.empty((self.V, 3))
        lam = C.c_double()
        lib().orc_get_state(self.h, th, ph, C.byref(lam))
        return th, ph, lam.value

    def derived(self):
        bind = np.empty((self.L, 8))
        S = np.empty(self.L)
        nbr = np.empty((self.V, max(self.params["knn"], 1)), np.int32)
        lib().orc_get_derived(self.h, bind, S, nbr)
        return bind, S, nbr[:, :self.params["knn"]]

    # steps -----------------------------------------------------------------------------------------
    def fk(self, theta):
        H0 = np.empty((self.L, 8))
        Hd = np.empty((self.L, 8))
        lib().orc_fk(self.h, np.ascontiguousarray(theta, np.float64), H0, Hd)
        return H0, Hd

    def skin(self, theta, phi=None):
        v = np.empty((self.V, 3))
        Hs = np.empty((self.V, 8))
        ph = np.zeros((self.V, 3)) if phi is None else np.ascontiguousarray(phi, np.float64).reshape(self.V, 3)
        lib().orc_skin(self.h, np.ascontiguousarray(theta, np.float64), ph, v, Hs)
        return v, Hs

    def normals(self, v):
        return normals(v, self.tris)

    def raster(self, v, with_amb=False):
        return raster(self.W, self.H, self.fx, self.fy, self.cx, self.cy, self.params["z_near"], v, self.tris, with_amb)

    def visibility(self, v, n, nvalid, z, zamb=None, with_marg=False):
        vis = np.empty(self.V, np.int32)
        pix = np.empty(self.V, np.int32)
        marg = np.empty(self.V, np.int32) if with_marg else None
        za = None if zamb is None else np.ascontiguousarray(zamb, np.int32).ravel()
        lib().orc_visibility(self.h, np.ascontiguousarray(v, np.float64), np.ascontiguousarray(n, np.float64),
                             np.ascontiguousarray(nvalid, np.int32), np.ascontiguousarray(z, np.float64).ravel(),
                             _ptr(za), vis, pix, _ptr(marg))
        return vis, pix, marg

    def associate(self, v, vis, pix, depth, marg=None, with_tie=False):
        corr = np.empty(self.W * self.H, np.int32)
        acc = np.empty((self.V, 3))
        cnt = np.empty(self.V, np.int32)
        tie = np.empty(self.W * self.H, np.int32) if with_tie else None
        mg = None if marg is None else np.ascontiguousarray(marg, np.int32)
        lib().orc_associate(self.h, np.ascontiguousarray(v, np.float64), np.ascontiguousarray(vis, np.int32),
                            np.ascontiguousarray(pix, np.int32), _ptr(mg),
                            np.ascontiguousarray(depth, np.float32).ravel(), corr, acc, cnt, _ptr(tie))
        return corr.reshape(self.H, self.W), acc, cnt, None if tie is None else tie.reshape(self.H, self.W)

    def associate_rid(self, v, ztri, depth, zamb=None, with_tie=False):
        """Raster-ID association (R23): nearest corner of the triangle the z-buffer holds at the pixel."""
        corr = np.empty(self.W * self.H, np.int32)
        acc = np.empty((self.V, 3))
        cnt = np.empty(self.V, np.int32)
        tie = np.empty(self.W * self.H, np.int32) if with_tie else None
        za = None if zamb is None else np.ascontiguousarray(zamb, np.int32).ravel()
        lib().orc_associate_rid(self.h, np.ascontiguousarray(v, np.float64), np.ascontiguousarray(ztri, np.int32).ravel(),
                                _ptr(za), np.ascontiguousarray(depth, np.float32).ravel(), corr, acc, cnt, _ptr(tie))
        return corr.reshape(self.H, self.W), acc, cnt, None if tie is None else tie.reshape(self.H, self.W)

    def accumulate(self, v, depth, corr):
        acc = np.empty((self.V, 3))
        cnt = np.empty(self.V, np.int32)
        lib().orc_accumulate(self.h, np.ascontiguousarray(v, np.float64), np.ascontiguousarray(depth, np.float32).ravel(),
                             np.ascontiguousarray(corr, np.int32).ravel(), acc, cnt)
        return acc, cnt

    def residuals(self, theta, n, nvalid, acc, cnt):
        r = np.empty(self.V)
        inA = np.empty(self.V, np.int32)
        E = lib().orc_residuals(self.h, np.ascontiguousarray(theta, np.float64), np.ascontiguousarray(n, np.float64),
                                np.ascontiguousarray(nvalid, np.int32), np.ascontiguousarray(acc, np.float64),
                                np.ascontiguousarray(cnt, np.int32), r, inA)
        return r, inA, E

    def jacobian(self, theta, phi, n, inA):
        J = np.empty((self.V, self.L))
        ph = np.zeros((self.V, 3)) if phi is None else np.ascontiguousarray(phi, np.float64).reshape(self.V, 3)
        lib().orc_jacobian(self.h, np.ascontiguousarray(theta, np.float64), ph, np.ascontiguousarray(n, np.float64),
                           np.ascontiguousarray(inA, np.int32), J)
        return J

    def lm_step(self, JTJ, JTr, E, v, n, acc, cnt, inA, theta, lam):
        th = np.array(theta, np.float64)
        lm = C.c_double(lam)
        Ec = np.empty(6)
        a = lib().orc_lm_step(self.h, np.ascontiguousarray(JTJ, np.float64), np.ascontiguousarray(JTr, np.float64),
                              float(E), np.ascontiguousarray(v, np.float64), np.ascontiguousarray(n, np.float64),
                              np.ascontiguousarray(acc, np.float64), np.ascontiguousarray(cnt, np.int32),
                              np.ascontiguousarray(inA, np.int32), th, C.byref(lm), Ec)
        return a, th, lm.value, Ec

    def shape_step(self, theta, phi, n, acc, cnt, inA):
        ph = np.array(phi, np.float64).reshape(self.V, 3).copy()
        r = np.empty(self.V)
        g = np.empty((self.V, 3))
        E = lib().orc_shape_step(self.h, np.ascontiguousarray(theta, np.float64), ph, np.ascontiguousarray(n, np.float64),
                                 np.ascontiguousarray(acc, np.float64), np.ascontiguousarray(cnt, np.int32),
                                 np.ascontiguousarray(inA, np.int32), _ptr(r), _ptr(g))
        return E, ph, r, g

    def render(self, theta, phi=None):
        z = np.empty(self.W * self.H)
        ph = np.zeros((self.V, 3)) if phi is None else np.ascontiguousarray(phi, np.float64).reshape(self.V, 3)
        lib().orc_render(self.h, np.ascontiguousarray(theta, np.float64), ph, z)
        return z.reshape(self.H, self.W)

    def track_frame(self, depth):
        """One frame at the carried state; returns (energies, accepted attempts, associated pixels)."""
        n = self.params["pose_iters"] + self.params["shape_iters"]
        e = np.empty(max(n, 1))
        acc = np.empty(max(self.params["pose_iters"], 1), np.int32)
        na = lib().orc_track_frame(self.h, np.ascontiguousarray(depth, np.float32).ravel(), e, _ptr(acc))
        return e[:n], acc[:self.params["pose_iters"]], na

    # a full association pass at (theta, phi), as the frame schedule runs it -------------------------
    def pass_at(self, theta, phi, depth, with_ties=False):
        v, Hs = self.skin(theta, phi)
        n, nvalid = self.normals(v)
        z, zt, amb = self.raster(v, with_amb=with_ties)
        vis, pix, marg = self.visibility(v, n, nvalid, z, amb, with_marg=with_ties)
        corr, acc, cnt, tie = self.associate(v, vis, pix, depth, marg, with_tie=with_ties)
        r, inA, E = self.residuals(theta, n, nvalid, acc, cnt)
        return dict(v=v, Hs=Hs, n=n, nvalid=nvalid, z=z, ztri=zt, zamb=amb, vis=vis, pix=pix, marg=marg, corr=corr,
                    acc=acc, cnt=cnt, tie=tie, r=r, inA=inA, E=E)
