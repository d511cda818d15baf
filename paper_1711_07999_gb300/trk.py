"""ctypes binding of the C ABI in include/trk.h (argument marshalling only; every step of the tracker runs
in the CUDA kernels of libtrk.so).  Loading fails loudly when the library has not been built or no CUDA
device is usable: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

TRK_OK, TRK_ERR_INVALID_ARG, TRK_ERR_OOM, TRK_ERR_CUDA, TRK_ERR_NO_CAPACITY, TRK_ERR_TIMEOUT, TRK_ERR_NUMERIC = range(7)
MAX_LINKS = 79
PRECISION_FP32, PRECISION_BF16X3, PRECISION_TF32X3 = 0, 1, 2
MODE_TRACK, MODE_SHAPE_MATCH, MODE_SMOOTH_BIND = 0, 1, 2
SERVER_DISPATCH_BATCHED, SERVER_DISPATCH_SESSION = 0, 1

FIELDS = dict(VERTS=0, NORMALS=1, ZBUF=2, VISPIX=3, CORR=4, ACC=5, NORMAL_EQ=6, THETA=7, PHI=8, LAMBDA=9, ENERGY=10,
              LM_TRIALS=11, SHAPE_RG=12, NEIGHBOURS=13, PRIOR=14, LM_SOLVER=15)

# symbols include/trk.h declares (checked by the tests against the library's exports)
EXPORTS = ["trk_create", "trk_create_evicted", "trk_session_evict", "trk_session_restore", "trk_session_is_resident",
           "trk_set_pose", "trk_track_frame", "trk_track_frame_device", "trk_read_result",
           "trk_render_depth", "trk_session_export", "trk_session_import", "trk_destroy", "trk_last_error",
           "trk_set_depth", "trk_step_skin", "trk_step_raster",
           "trk_step_visibility", "trk_step_associate", "trk_step_normal_equations", "trk_step_lm", "trk_step_shape",
           "trk_read", "trk_get_info", "trk_profile_iteration", "trk_jtj_rows", "trk_jtj_rows_noalloc",
           "trk_jtj_rows_tc", "trk_fk_joint_positions", "trk_subdivide_counts", "trk_subdivide",
           "trk_batch_create", "trk_batch_track_device", "trk_batch_profile",
           "trk_batch_destroy",
           "trk_schedule_create", "trk_schedule_track_device", "trk_schedule_get_config", "trk_schedule_autotune",
           "trk_schedule_destroy", "trk_schedule_signature", "trk_tuning_cache_lookup", "trk_tuning_cache_store",
           "trk_server_create", "trk_server_configure", "trk_server_attach", "trk_server_detach", "trk_server_submit", "trk_server_wait",
           "trk_server_get_stats", "trk_server_destroy"]

STAGES = ["skin", "raster", "visibility", "associate", "resid_jtj", "reduce", "lm_solve", "lm_eval", "shape"]


class TrkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"trk status {status}: {msg}")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("verts", C.c_void_p), ("tris", C.c_void_p),
                ("bone_idx", C.c_void_p), ("bone_w", C.c_void_p)]


class Skeleton(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("parent", C.c_void_p), ("type", C.c_void_p), ("axis", C.c_void_p),
                ("offset_dq", C.c_void_p), ("prior_mask", C.c_void_p)]


class Intrinsics(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float)]


class Params(C.Structure):
    _fields_ = [("pose_iters", C.c_int32), ("shape_iters", C.c_int32), ("shape_sweeps", C.c_int32),
                ("lambda_k0", C.c_float), ("lambda_s", C.c_float), ("lambda_phi", C.c_float), ("lambda_N", C.c_float),
                ("lambda_w", C.c_float), ("cutoff_m", C.c_float), ("eps_vis_m", C.c_float), ("z_near_m", C.c_float),
                ("window_half_px", C.c_int32), ("knn", C.c_int32), ("precision", C.c_int32),
                ("shape_solver", C.c_int32), ("mode", C.c_int32), ("association", C.c_int32),
                ("jtj_group", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("n_verts", C.c_int32), ("n_tris", C.c_int32), ("width", C.c_int32),
                ("height", C.c_int32), ("kernels_per_frame", C.c_int32), ("device_bytes", C.c_size_t),
                ("jtj_group", C.c_int32)]


class ScheduleConfig(C.Structure):
    _fields_ = [("groups", C.c_int32), ("assoc_blocks", C.c_int32), ("tail_blocks", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("frames_done", C.c_uint64), ("in_flight", C.c_int32), ("sessions", C.c_int32),
                ("hbm_used_bytes", C.c_size_t), ("latency_p50_us", C.c_double), ("latency_p99_us", C.c_double),
                ("latency_max_us", C.c_double), ("steps", C.c_uint64), ("mean_frames_per_step", C.c_double),
                ("device_bytes_reserved", C.c_size_t)]


class Result(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("offsets", C.c_void_p), ("energy", C.c_void_p), ("n_assoc_px", C.c_int32),
                ("n_assoc_verts", C.c_int32)]


_lib = None


def lib(build_if_missing: bool = True):
    """Loads libtrk.so (building it first if it is missing or stale and nvcc is available)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1711_07999_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
        sigs = {
            "trk_create": [vp, vp, vp, vp, C.POINTER(vp)], "trk_create_evicted": [vp, vp, vp, vp, C.POINTER(vp)],
            "trk_session_evict": [vp], "trk_session_restore": [vp], "trk_session_is_resident": [vp],
            "trk_set_pose": [vp, vp, vp],
            "trk_track_frame": [vp, vp, vp], "trk_track_frame_device": [vp, vp, vp], "trk_read_result": [vp, vp],
            "trk_render_depth": [vp, vp, vp, vp], "trk_session_export": [vp, vp, C.POINTER(sz)],
            "trk_session_import": [vp, vp, sz], "trk_set_depth": [vp, vp], "trk_step_skin": [vp],
            "trk_step_raster": [vp], "trk_step_visibility": [vp], "trk_step_associate": [vp],
            "trk_step_normal_equations": [vp], "trk_step_lm": [vp], "trk_step_shape": [vp],
            "trk_read": [vp, i32, vp, sz], "trk_get_info": [vp, vp], "trk_profile_iteration": [vp, i32, sz, vp],
            "trk_jtj_rows": [vp, i32, i32, i32, vp, vp], "trk_jtj_rows_noalloc": [vp, i32, i32, i32, vp, vp],
            "trk_jtj_rows_tc": [vp, i32, i32, i32, i32, vp, vp],
            "trk_fk_joint_positions": [vp, vp, vp],
            "trk_subdivide_counts": [vp, vp, i32, i32, i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
            "trk_subdivide": [vp, vp, vp, i32, i32, vp, vp, i32, i32, vp, vp, vp, vp],
            "trk_batch_create": [C.POINTER(vp), i32, C.POINTER(vp)], "trk_batch_track_device": [vp, C.POINTER(vp), vp],
            "trk_batch_profile": [vp, C.POINTER(vp), i32, sz, vp],
            "trk_schedule_create": [C.POINTER(vp), i32, vp, C.c_char_p, C.POINTER(vp)],
            "trk_schedule_track_device": [vp, C.POINTER(vp), vp], "trk_schedule_get_config": [vp, vp],
            "trk_schedule_autotune": [vp, C.POINTER(vp), i32, C.c_char_p, vp, C.POINTER(C.c_double)],
            "trk_schedule_signature": [C.POINTER(vp), i32, C.c_char_p, sz],
            "trk_tuning_cache_lookup": [C.c_char_p, C.c_char_p, vp, C.POINTER(C.c_double)],
            "trk_tuning_cache_store": [C.c_char_p, C.c_char_p, vp, C.c_double],
            "trk_server_create": [sz, i32, C.POINTER(vp)], "trk_server_configure": [vp, i32, i32, i32, C.c_int64],
            "trk_server_attach": [vp, vp], "trk_server_detach": [vp, vp],
            "trk_server_submit": [vp, vp, vp, C.POINTER(C.c_uint64)], "trk_server_wait": [vp, C.c_uint64, C.c_int64, vp],
            "trk_server_get_stats": [vp, vp],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.trk_destroy.argtypes = [vp]
        L.trk_destroy.restype = None
        L.trk_server_destroy.argtypes = [vp]
        L.trk_server_destroy.restype = None
        L.trk_batch_destroy.argtypes = [vp]
        L.trk_batch_destroy.restype = None
        L.trk_schedule_destroy.argtypes = [vp]
        L.trk_schedule_destroy.restype = None
        L.trk_last_error.argtypes = []
        L.trk_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != TRK_OK:
        raise TrkError(status, lib().trk_last_error().decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def jtj_rows(rows_ptr: int, n_rows: int, n_cols: int, ld: int, out_ptr: int, stream_ptr: int = 0):
    """[J r]^T [J r] of device FP32 rows [n_rows][ld] into device FP64 [n_cols][n_cols] (enqueued on the
    given CUDA stream handle; device pointers e.g. from ``tensor.data_ptr()``)."""
    _check(lib().trk_jtj_rows(C.c_void_p(rows_ptr), n_rows, n_cols, ld, C.c_void_p(out_ptr),
                              C.c_void_p(stream_ptr or None)))


def jtj_rows_noalloc(rows_ptr: int, n_rows: int, n_cols: int, ld: int, out_ptr: int, stream_ptr: int = 0):
    """trk_jtj_rows without any allocation (fixed scratch, n_cols <= 80; overlapping calls race)."""
    _check(lib().trk_jtj_rows_noalloc(C.c_void_p(rows_ptr), n_rows, n_cols, ld, C.c_void_p(out_ptr),
                                      C.c_void_p(stream_ptr or None)))


def jtj_rows_tc(rows_ptr: int, n_rows: int, n_cols: int, ld: int, precision: int, out_ptr: int,
                stream_ptr: int = 0):
    """trk_jtj_rows on the tensor cores: split-BF16x3 (PRECISION_BF16X3) or 3xTF32 (PRECISION_TF32X3)."""
    _check(lib().trk_jtj_rows_tc(C.c_void_p(rows_ptr), n_rows, n_cols, ld, precision, C.c_void_p(out_ptr),
                                 C.c_void_p(stream_ptr or None)))


def joint_positions(skeleton: dict, theta) -> np.ndarray:
    """[n_links, 3] camera-frame joint positions (each link's frame origin) for joint values theta
    (trk_fk_joint_positions: FP64 forward kinematics on the host)."""
    parent = np.ascontiguousarray(skeleton["parent"], np.int32)
    typ = np.ascontiguousarray(skeleton["type"], np.int32)
    axis = np.ascontiguousarray(skeleton["axis"], np.float32)
    off = np.ascontiguousarray(skeleton["offset_dq"], np.float32)
    mask = np.ascontiguousarray(skeleton["prior_mask"], np.float32)
    L = len(parent)
    sk = Skeleton(L, _p(parent), _p(typ), _p(axis), _p(off), _p(mask))
    th = np.ascontiguousarray(theta, np.float64)
    out = np.empty((L, 3))
    _check(lib().trk_fk_joint_positions(C.byref(sk), _p(th), _p(out)))
    return out


def subdivide_counts(face_off, face_vert, n_verts: int, levels: int = 2):
    """trk_subdivide_counts: (vertices, triangles) after `levels` Catmull-Clark levels of a polygon cage
    (host connectivity only; no device work)."""
    fo = np.ascontiguousarray(face_off, np.int32)
    fv = np.ascontiguousarray(face_vert, np.int32)
    nv, nt = C.c_int32(), C.c_int32()
    _check(lib().trk_subdivide_counts(_p(fo), _p(fv), n_verts, len(fo) - 1, levels, C.byref(nv), C.byref(nt)))
    return nv.value, nt.value


def subdivide(verts, face_off, face_vert, bone_idx, bone_w, n_bones: int, levels: int = 2):
    """Template authoring (trk_subdivide): Catmull-Clark subdivision of a polygon cage with its skin
    weights; returns (verts [V'][3] float32, tris [T'][3] int32, bone_idx [V'][4] uint8, bone_w [V'][4])."""
    v = np.ascontiguousarray(verts, np.float32)
    fo = np.ascontiguousarray(face_off, np.int32)
    fv = np.ascontiguousarray(face_vert, np.int32)
    bi = np.ascontiguousarray(bone_idx, np.uint8)
    bw = np.ascontiguousarray(bone_w, np.float32)
    nv, nt = C.c_int32(), C.c_int32()
    _check(lib().trk_subdivide_counts(_p(fo), _p(fv), len(v), len(fo) - 1, levels, C.byref(nv), C.byref(nt)))
    ov = np.empty((nv.value, 3), np.float32)
    ot = np.empty((nt.value, 3), np.int32)
    obi = np.empty((nv.value, 4), np.uint8)
    obw = np.empty((nv.value, 4), np.float32)
    _check(lib().trk_subdivide(_p(v), _p(fo), _p(fv), len(v), len(fo) - 1, _p(bi), _p(bw), n_bones, levels,
                               _p(ov), _p(ot), _p(obi), _p(obw)))
    return ov, ot, obi, obw


def params_struct(p: dict) -> Params:
    return Params(pose_iters=p["pose_iters"], shape_iters=p["shape_iters"], shape_sweeps=p["shape_sweeps"],
                  lambda_k0=p["lambda_k0"], lambda_s=p["lambda_s"], lambda_phi=p["lambda_phi"],
                  lambda_N=p["lambda_N"], lambda_w=p["lambda_w"], cutoff_m=p["cutoff"], eps_vis_m=p["eps_vis"],
                  z_near_m=p["z_near"], window_half_px=p["window_half"], knn=p["knn"],
                  precision=p.get("precision", PRECISION_FP32), shape_solver=p.get("shape_solver", 0),
                  mode=p.get("mode", MODE_TRACK), association=p.get("association", 0),
                  jtj_group=p.get("jtj_group", 0))


class Session:
    """One tracking session (trk_create ... trk_destroy) for a model dict of ``synth.make_model`` form."""

    def __init__(self, model: dict, evicted: bool = False):
        """trk_create (device state allocated), or trk_create_evicted with evicted=True (no device memory
        until restore() or a server's attach)."""
        sk, me, cam, pr = model["skeleton"], model["mesh"], model["camera"], model["params"]
        self._keep = k = dict(
            parent=np.ascontiguousarray(sk["parent"], np.int32), type=np.ascontiguousarray(sk["type"], np.int32),
            axis=np.ascontiguousarray(sk["axis"], np.float32), off=np.ascontiguousarray(sk["offset_dq"], np.float32),
            mask=np.ascontiguousarray(sk["prior_mask"], np.float32),
            verts=np.ascontiguousarray(me["verts"], np.float32), tris=np.ascontiguousarray(me["tris"], np.int32),
            bidx=np.ascontiguousarray(me["bone_idx"], np.uint8), bw=np.ascontiguousarray(me["bone_w"], np.float32))
        self.L, self.V, self.F = len(k["parent"]), len(k["verts"]), len(k["tris"])
        self.W, self.H = int(cam["width"]), int(cam["height"])
        self.params = dict(pr)
        mesh = Mesh(self.V, self.F, _p(k["verts"]), _p(k["tris"]), _p(k["bidx"]), _p(k["bw"]))
        skel = Skeleton(self.L, _p(k["parent"]), _p(k["type"]), _p(k["axis"]), _p(k["off"]), _p(k["mask"]))
        intr = Intrinsics(self.W, self.H, cam["fx"], cam["fy"], cam["cx"], cam["cy"])
        prm = params_struct(pr)
        h = C.c_void_p()
        create = lib().trk_create_evicted if evicted else lib().trk_create
        _check(create(C.byref(mesh), C.byref(skel), C.byref(intr), C.byref(prm), C.byref(h)))
        self.h = h
        self.n_energy = pr["pose_iters"] + pr["shape_iters"]

    def close(self):
        if getattr(self, "h", None):
            lib().trk_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- device residency -------------------------------------------------------------------------
    def evict(self):
        """trk_session_evict: tracking state to the host, device state freed."""
        _check(lib().trk_session_evict(self.h))

    def restore(self):
        """trk_session_restore: device state allocated again, tracking state restored."""
        _check(lib().trk_session_restore(self.h))

    @property
    def resident(self) -> bool:
        return bool(lib().trk_session_is_resident(self.h))

    # -- state / frames ---------------------------------------------------------------------------
    def set_pose(self, theta, offsets=None):
        th = np.ascontiguousarray(theta, np.float64)
        of = None if offsets is None else np.ascontiguousarray(offsets, np.float32).reshape(self.V, 3)
        _check(lib().trk_set_pose(self.h, _p(th), _p(of)))

    def export_state(self) -> bytes:
        """trk_session_export: the tracking state (Theta, Phi, lambda, frames since set_pose) as bytes."""
        n = C.c_size_t(0)
        _check(lib().trk_session_export(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().trk_session_export(self.h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def import_state(self, blob: bytes):
        """trk_session_import: resumes from a blob of export_state (same model and parameters)."""
        b = bytes(blob)
        _check(lib().trk_session_import(self.h, b, len(b)))

    def _result(self, want_offsets=True):
        th = np.empty(self.L, np.float64)
        of = np.empty((self.V, 3), np.float32) if want_offsets else None
        en = np.empty(max(self.n_energy, 1), np.float64)
        r = Result(_p(th), _p(of), _p(en), 0, 0)
        return r, th, of, en

    def track_frame(self, depth, want_offsets=True) -> dict:
        """Host depth [H, W] float32 metres; returns theta, offsets, energy and association counts."""
        dep = np.ascontiguousarray(depth, np.float32)
        assert dep.size == self.W * self.H
        r, th, of, en = self._result(want_offsets)
        _check(lib().trk_track_frame(self.h, _p(dep), C.byref(r)))
        return dict(theta=th, offsets=of, energy=en[:self.n_energy], n_assoc_px=r.n_assoc_px,
                    n_assoc_verts=r.n_assoc_verts)

    def track_frame_device(self, depth_ptr: int, stream_ptr: int = 0):
        """Enqueues a frame reading depth from a device pointer (e.g. ``tensor.data_ptr()``) on a CUDA
        stream handle (e.g. ``torch.cuda.Stream().cuda_stream``); returns without waiting."""
        _check(lib().trk_track_frame_device(self.h, C.c_void_p(depth_ptr), C.c_void_p(stream_ptr or None)))

    def read_result(self, want_offsets=True) -> dict:
        r, th, of, en = self._result(want_offsets)
        _check(lib().trk_read_result(self.h, C.byref(r)))
        return dict(theta=th, offsets=of, energy=en[:self.n_energy], n_assoc_px=r.n_assoc_px,
                    n_assoc_verts=r.n_assoc_verts)

    def render_depth(self, theta, offsets=None) -> np.ndarray:
        out = np.empty((self.H, self.W), np.float32)
        th = np.ascontiguousarray(theta, np.float64)
        of = None if offsets is None else np.ascontiguousarray(offsets, np.float32).reshape(self.V, 3)
        _check(lib().trk_render_depth(self.h, _p(th), _p(of), _p(out)))
        return out

    def info(self) -> dict:
        inf = Info()
        _check(lib().trk_get_info(self.h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def profile_iteration(self, reps: int = 10, flush_bytes: int = 0) -> dict:
        """Mean CUDA-event duration (ms) of each stage of an iteration, at the current state and depth."""
        ms = np.empty(len(STAGES), np.float32)
        _check(lib().trk_profile_iteration(self.h, reps, flush_bytes, _p(ms)))
        return dict(zip(STAGES, ms.tolist()))

    # -- step-level calls -------------------------------------------------------------------------
    def set_depth(self, depth):
        dep = np.ascontiguousarray(depth, np.float32)
        _check(lib().trk_set_depth(self.h, _p(dep)))

    def step(self, name: str):
        _check(getattr(lib(), "trk_step_" + name)(self.h))

    def read(self, field: str) -> np.ndarray:
        V, npx, L, NP = self.V, self.W * self.H, self.L, self.L + 1
        shapes = dict(VERTS=((V, 4), np.float32), NORMALS=((V, 4), np.float32), ZBUF=((npx,), np.uint64),
                      VISPIX=((V,), np.int32), CORR=((npx,), np.int32), ACC=((V, 4), np.int64),
                      NORMAL_EQ=((NP, NP), np.float64), THETA=((L,), np.float64), PHI=((V, 4), np.float32),
                      LAMBDA=((1,), np.float64), ENERGY=((self.n_energy,), np.float64), LM_TRIALS=((8,), np.float64),
                      SHAPE_RG=((V, 4), np.float32), NEIGHBOURS=((V, 4), np.int32), PRIOR=((L,), np.float64),
                      LM_SOLVER=((6,), np.int32))
        shp, dt = shapes[field]
        out = np.empty(shp, dt)
        _check(lib().trk_read(self.h, FIELDS[field], _p(out), out.nbytes))
        return out


class Batch:
    """Sessions stepped together (trk_batch_*): one launch per stage over all members' blocks."""

    def __init__(self, sessions):
        self.sessions = list(sessions)
        arr = (C.c_void_p * len(self.sessions))(*[x.h.value for x in self.sessions])
        h = C.c_void_p()
        _check(lib().trk_batch_create(arr, len(self.sessions), C.byref(h)))
        self.h = h

    def track_device(self, depth_ptrs, stream_ptr: int = 0):
        """One frame of every member; depth_ptrs[k] is a device pointer to member k's depth image."""
        arr = (C.c_void_p * len(self.sessions))(*depth_ptrs)
        _check(lib().trk_batch_track_device(self.h, arr, C.c_void_p(stream_ptr or None)))

    def profile(self, depth_ptrs, reps: int = 5, flush_bytes: int = 0) -> dict:
        """Mean CUDA-event duration (ms) of each stage as one batched launch (the members advance)."""
        arr = (C.c_void_p * len(self.sessions))(*depth_ptrs)
        ms = np.empty(len(STAGES), np.float32)
        _check(lib().trk_batch_profile(self.h, arr, reps, flush_bytes, _p(ms)))
        return dict(zip(STAGES, ms.tolist()))

    def close(self):
        if self.h:
            lib().trk_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cfg_dict(c: ScheduleConfig) -> dict:
    return {"groups": c.groups, "assoc_blocks": c.assoc_blocks, "tail_blocks": c.tail_blocks}


def tuning_cache_lookup(path: str, signature: str):
    """The cached schedule of a size class as (config dict, ms per frame), or None."""
    c, ms = ScheduleConfig(), C.c_double()
    st = lib().trk_tuning_cache_lookup(path.encode(), signature.encode(), C.byref(c), C.byref(ms))
    return None if st != TRK_OK else (_cfg_dict(c), ms.value)


def tuning_cache_store(path: str, signature: str, cfg: dict, ms: float):
    _check(lib().trk_tuning_cache_store(path.encode(), signature.encode(), C.byref(ScheduleConfig(**cfg)), ms))


class Schedule:
    """How a set of sessions is stepped per frame (trk_schedule_*): work-balanced groups on concurrent
    streams, each a fused batch or a session's own graph; autotune() picks the fastest and caches it."""

    def __init__(self, sessions, config: dict | None = None, cache_path: str | None = None):
        self.sessions = list(sessions)
        arr = (C.c_void_p * len(self.sessions))(*[x.h.value for x in self.sessions])
        cfg = C.byref(ScheduleConfig(**config)) if config else None
        h = C.c_void_p()
        _check(lib().trk_schedule_create(arr, len(self.sessions), cfg, cache_path.encode() if cache_path else None,
                                         C.byref(h)))
        self.h = h

    @staticmethod
    def signature(sessions) -> str:
        arr = (C.c_void_p * len(sessions))(*[x.h.value for x in sessions])
        buf = C.create_string_buffer(256)
        _check(lib().trk_schedule_signature(arr, len(sessions), buf, 256))
        return buf.value.decode()

    def track_device(self, depth_ptrs, stream_ptr: int = 0):
        arr = (C.c_void_p * len(self.sessions))(*depth_ptrs)
        _check(lib().trk_schedule_track_device(self.h, arr, C.c_void_p(stream_ptr or None)))

    def config(self) -> dict:
        c = ScheduleConfig()
        _check(lib().trk_schedule_get_config(self.h, C.byref(c)))
        return _cfg_dict(c)

    def autotune(self, depth_ptrs, reps: int = 3, cache_path: str | None = None):
        """Times candidate schedules on real frames (the sessions advance) and keeps the fastest;
        returns (config dict, ms per frame)."""
        arr = (C.c_void_p * len(self.sessions))(*depth_ptrs)
        c, ms = ScheduleConfig(), C.c_double()
        _check(lib().trk_schedule_autotune(self.h, arr, reps, cache_path.encode() if cache_path else None,
                                           C.byref(c), C.byref(ms)))
        return _cfg_dict(c), ms.value

    def close(self):
        if self.h:
            lib().trk_schedule_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching frame server (trk_server_*) over attached sessions."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 32, dispatch: int = SERVER_DISPATCH_BATCHED,
                 max_batch: int = 64, concurrent_steps: int = 2, max_wait_us: int = 2000):
        h = C.c_void_p()
        _check(lib().trk_server_create(hbm_budget_bytes, max_inflight, C.byref(h)))
        self.h = h
        self._sessions = {}
        _check(lib().trk_server_configure(self.h, dispatch, max_batch, concurrent_steps, max_wait_us))

    def attach(self, session: Session):
        _check(lib().trk_server_attach(self.h, session.h))
        self._sessions[session.h.value] = session

    def detach(self, session: Session):
        _check(lib().trk_server_detach(self.h, session.h))
        self._sessions.pop(session.h.value, None)

    def submit(self, session: Session, depth) -> int:
        dep = np.ascontiguousarray(depth, np.float32)
        t = C.c_uint64()
        _check(lib().trk_server_submit(self.h, session.h, _p(dep), C.byref(t)))
        return t.value

    def wait(self, session: Session, ticket: int, timeout_us: int = 10_000_000, want_offsets=True) -> dict:
        r, th, of, en = session._result(want_offsets)
        _check(lib().trk_server_wait(self.h, ticket, timeout_us, C.byref(r)))
        return dict(theta=th, offsets=of, energy=en[:session.n_energy], n_assoc_px=r.n_assoc_px,
                    n_assoc_verts=r.n_assoc_verts)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().trk_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().trk_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

