#!/usr/bin/env python3
"""Benchmark of the tracker on the 50k-vertex humanoid / 640x480 depth workload (one tracking session
per GPU, a seeded synthetic 30 fps sequence; one step = one frame = 10 pose LM iterations + 2 shape
iterations through the whole hot path).

Prints one JSON line (rank 0):
  value      frames/s over all ranks of the batched measurement: --sessions concurrent sessions per GPU
             (one stream and one CUDA graph each) each tracking one frame per step; device-timed (CUDA
             events) with the depth frames already resident in HBM; L2 is flushed (a 256 MiB write)
             before every step, outside the timed intervals.  "plain" holds the same figures for one
             session alone (--sessions 1 makes it the headline)
  latency    p50 / p99 per-frame latency (from the step's start to the session's completion)
  serving    (in "batched") --serve-streams streams with Poisson arrivals at 30 fps each through the frame
             server (trk_server_*): achieved frames/s and submit -> completion p50 / p99 latency
  e2e        frames/s through trk_track_frame with host (pinned) depth: H2D of the frame and D2H of
             Theta, Phi and the energies inside the timed region
  precision  per [J r]^T [J r] arithmetic (fp32, bf16x3, tf32x3; the last two on the tensor cores): batched
             frames/s, the contraction stage's time and each result's error against the oracle on the
             CPU-baseline frames (joint values, also where the energy determines them; offsets, also where
             the two final poses agree; energies)
  uneven     --uneven-sessions sessions of random-tree bodies (5k-200k vertices, 12-40 bones, 320x240 to
             1280x720): frames/s one by one, on one stream each, as one fused batch (trk_batch_*), and
             under the schedule the autotuner picks (trk_schedule_*); each stage's HBM roofline in the fused
             batch, profiled at the first frame's state (--uneven-jtj-group sets the sessions' [J r] grouping)
  admission_serving  --admission-streams streams of uneven sessions with Poisson starts under a 1 GiB HBM
             budget: admitted as capacity frees, 30 Poisson frames/s each, then leaving; served frames/s,
             latency, admission waits, peak admitted bytes
  experiments  the paper's conditions (full tracking, shape-match, smooth-bind) on the sequence with its
             ground truth: joint accuracy (AUC up to 10 cm) and reconstruction error
  roofline   the dominant kernel's achieved rate against the measured peak of MEASURED_PEAKS.json, with a
             note on what bounds it
  cpu_baseline  the FP64 oracle on the host, one core, a bounded sample of the same sequence
--impl reference times the oracle itself (on host cores) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s and p99 frame latency, 50k-vert/640x480, batched vs plain, same GPU"
PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 2}
WORKLOAD = "humanoid-22bone-55dof-50k-vert-640x480-30fps-sinusoidal"
L2_FLUSH_BYTES = 256 << 20


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values of x (the job takes as long as its slowest rank): an all-reduce of
    one float64 over the process group (NCCL on the GPUs; gloo when device is "cpu"); x itself at world 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, max_seconds):
    """Units per second of the whole job: every rank processes units_per_rank units (weak scaling, sessions
    sharded by rank, no data-path collective) and the job ends with its slowest rank."""
    return world * units_per_rank / max_seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]), src="measured")
    except (OSError, KeyError, ValueError):
        return dict(hbm_gbs=6800.0, bf16=1900.0, src="fallback")


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# algorithmic work per launch of each stage (bytes a minimal implementation must move / flops)
# ------------------------------------------------------------------------------------------------
# What bounds the dominant stage of one 50k-vertex session (its grids are one or two waves and its
# working set sits in L2; ncu summaries under profiles/); the streaming stages' HBM fractions at batch
# scale are the uneven batch's fused_stage_roofline.
ROOFLINE_NOTES = {
    "associate": "exact ring search per depth pixel: chains of dependent bucket loads (latency, not bytes)",
    "lm_solve": "six 55x55 damped solves on 6 SMs: FP32 blocked Cholesky steps and FP64 refinement, "
                "barrier- and dependency-latency bound",
}


def algorithmic(stage, V, F, npx, NP, nvis, nassoc_px, nA, n_valid_px, nblk):
    """Minimum bytes (or FP64 flops) a stage must move for one session: V vertices, F triangles, npx
    pixels, NP = links + 1, nvis visible vertices, nassoc_px associated pixels, nA vertices in A,
    n_valid_px valid depth pixels, nblk [J r] blocks (256 jtj_group vertices each) that hold rows."""
    if stage == "skin":  # v0, phi, bone idx, bone w in; v out; sums cleared; z-buffer, heads, corr cleared
        return "hbm", V * (16 + 16 + 4 + 16 + 16 + 32) + npx * (8 + 4 + 4)
    if stage == "raster":  # triangles, posed vertices, face normals out, covered z-buffer words
        return "hbm", F * (16 + 16) + V * 16 + n_valid_px * 8
    if stage == "visibility":  # CSR, face normals, v, normals out, z-buffer probes, bucket records
        return "hbm", V * (4 + 16 + 16 + 4) + 3 * F * 4 + F * 16 + nvis * (8 + 4 + 16)
    if stage == "associate":  # depth in and correspondences out over the image, the associated vertices' sums
        return "hbm", npx * (4 + 4) + nA * 28
    if stage == "resid_jtj":  # sums and normals of every vertex; streams of A; partials of blocks with rows;
        # the 64-byte record of every row for the candidate energies
        return "hbm", V * (32 + 16) + nA * (4 + 16 + 16 + 16 + 16) + nblk * NP * NP * 4 + nA * 64
    if stage == "reduce":
        return "hbm", nblk * NP * NP * 4 + NP * NP * 8
    if stage == "lm_eval":  # the rows' records and row counts (the first pass: candidates 0 and 1)
        return "hbm", nA * 64 + nblk * 4
    if stage == "shape":  # phi, neighbours, sums, normals in; phi, r/g, phi0 out; bones of A
        return "hbm", V * (16 + 16 + 32 + 16 + 16 + 16 + 16) + nA * (4 + 16)
    if stage == "lm_solve":  # 6 FP64 Cholesky factorisations + solves of the P x P system
        P = NP - 1
        return "fp64", 6 * (P ** 3 / 3.0 + 2 * P * P)
    return None, 0


def session_counts(sess, depth):
    """The per-session counts the byte model needs, read back at the session's current state."""
    info = sess.info()
    acc = sess.read("ACC")
    NP = info["n_links"] + 1
    nA = int((acc[:, 3] > 0).sum())
    blocks = (np.nonzero(acc[:, 3] > 0)[0] // (256 * info["jtj_group"]))
    return dict(V=info["n_verts"], F=info["n_tris"], npx=info["width"] * info["height"], NP=NP,
                nvis=int((sess.read("VISPIX") >= 0).sum()), nassoc_px=int(acc[:, 3].sum()), nA=nA,
                n_valid_px=int((np.asarray(depth) > 0).sum()), nblk=int(len(np.unique(blocks))))


def kernel_source_hash():
    """Hash of the device-kernel sources (the host runtime files do not change a kernel's traffic)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1711_07999_gb300", "csrc")
    for n in sorted(os.listdir(csrc)):
        if n.startswith("kernels_") and n.endswith(".cu") or n.endswith(".cuh"):
            with open(os.path.join(csrc, n), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if it was captured from the
    current kernel sources (an entry's own source hash, else the file's; otherwise None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get("kernels", {}).get(kernel)
    if e is None or e.get("kernel_source_hash", t.get("kernel_source_hash")) != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch_full_size")


# ------------------------------------------------------------------------------------------------
def render_sequence(model, session, n_frames, seed):
    from paper_1711_07999_gb300 import synth
    rng = np.random.default_rng(seed)
    frames = np.empty((n_frames, model["camera"]["height"], model["camera"]["width"]), np.float32)
    for f in range(n_frames):
        t = f / 30.0
        z = session.render_depth(synth.gt_theta(model, t), synth.gt_offsets(model, t))
        frames[f] = synth.add_noise(z, 2, rng)
    return frames


def oracle_frames(model, n_frames, seed):
    import oracle
    from paper_1711_07999_gb300 import synth
    o = oracle.Oracle(model)
    rng = np.random.default_rng(seed)
    frames = []
    for f in range(n_frames):
        t = f / 30.0
        frames.append(synth.add_noise(o.render(synth.gt_theta(model, t), synth.gt_offsets(model, t)), 2, rng))
    return o, frames


def cpu_baseline(model, n_frames):
    """The oracle as it stands, single-threaded FP64, on the first n_frames of the sequence.  Also returns
    the frames and the oracle's state after each (for the per-result error of the precision modes)."""
    from paper_1711_07999_gb300 import synth
    o, frames = oracle_frames(model, n_frames, seed=synth.seed_for(2, 900))
    o.set_state(synth.gt_theta(model, 0.0), None)
    states = []
    dt = 0.0
    start = (synth.gt_theta(model, 0.0), np.zeros((o.V, 3)), model["params"]["lambda_k0"])
    for d in frames:
        t0 = time.perf_counter()
        e, _, _ = o.track_frame(d)
        dt += time.perf_counter() - t0
        th, phi, lam = o.get_state()
        states.append((th, phi, e, determined_dofs(o, model, th, phi, d), start))
        start = (th, phi, lam)
    return dict(value=n_frames / dt, unit="frames/s", cores=1, kind="oracle",
                sample=f"first {n_frames} frames of the sequence, 10 pose + 2 shape iterations each, FP64, 1 thread",
                seconds=round(dt, 2)), frames, states, o


def determined_dofs(o, model, th, phi, depth, tol=1e-3):
    """DoFs the energy fixes to within tol at the oracle's state: moving DoF k by tol (the others
    re-optimised) raises E by more than 1e-5 relative, sqrt(1e-5 E [H^-1]_kk) < tol, H = J^T J + prior."""
    import oracle
    P = o.pass_at(th, phi, depth)
    J = o.jacobian(th, phi, P["n"], P["inA"])
    JTJ, _ = oracle.normal_eq(J, P["r"], P["inA"])
    _, S, _ = o.derived()
    H = JTJ + np.diag((model["params"]["lambda_s"] * S) ** 2)
    return np.sqrt(1e-5 * P["E"] * np.diag(np.linalg.inv(H))) < tol


def _oracle_worker(k, n_frames):
    """One independent oracle session (the all-cores baseline): its own model and frames; returns the
    frames tracked and the seconds the tracking took."""
    import oracle
    from paper_1711_07999_gb300 import synth
    model = synth.make_model(2, session=3000 + k)
    o, frames = oracle_frames(model, n_frames, seed=synth.seed_for(2, 3100 + k))
    o.set_state(synth.gt_theta(model, 0.0), None)
    t0 = time.perf_counter()
    for d in frames:
        o.track_frame(d)
    return n_frames, time.perf_counter() - t0


def cpu_baseline_all_cores(n_frames):
    """The oracle over all host cores: one independent session per core (spawned processes), each
    tracking n_frames frames; aggregate frames/s over the slowest worker's tracking time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(k, n_frames) for k in range(cores)])
    frames = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return {"value": frames / secs, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent sessions of the 50k-vertex workload, {n_frames} frames each, one per process"}


def lockstep_vs_oracle(model, prec, frames, states, o, n_frames=2):
    """Per-result error of one precision mode against the oracle, frame by frame from the oracle's own
    state (tests/sequence.py): both run the frame in lockstep, the oracle taking the GPU's choice only at
    pixels it flags as correspondence ties; then joint values on all DoFs, offsets on all vertices, the
    energy of every iteration at the same state, the LM decisions."""
    from paper_1711_07999_gb300 import synth, trk
    from tests import sequence as seq
    out = []
    with trk.Session(synth.make_model(2, precision=prec)) as s:
        for f, (d, st) in enumerate(zip(frames[:n_frames], states[:n_frames])):
            th, phi, lam = st[4]
            out.append(seq.summary(seq.follow_frame(o, s, d, th, np.asarray(phi, np.float32), lam, frames_done=f)))
    return {"frames": len(out), "theta_rad_max": max(x["theta_rad_max"] for x in out),
            "offsets_mm_max": max(x["offsets_mm_max"] for x in out),
            "energy_rel_max_matched": max(x["energy_rel_max_matched"] for x in out),
            "nontie_mismatches": sum(x["nontie_mismatches"] for x in out),
            "tie_flips": sum(x["tie_flips"] for x in out), "invalid_flips": sum(x["invalid_flips"] for x in out),
            "lm_decisions_equal": all(x["lm_decisions_equal"] for x in out)}


def errors_vs_oracle(model, prec, frames, states, o):
    """Per-result error of one precision mode against the oracle on the same frames, free-running from
    the same start (the two paths part at correspondence ties): joint values (all, and those the energy
    determines to 1e-3 rad), offsets (99th percentile and max over vertices; and the 99th percentile over
    the vertices the two final poses place within 0.05 mm of each other), energies."""
    from paper_1711_07999_gb300 import synth, trk
    dth, dthd, ndet, dphi99, dphimax, de, agree99, agree_frac = [], [], [], [], [], [], [], []
    zero = np.zeros((o.V, 3))
    with trk.Session(synth.make_model(2, precision=prec)) as s:
        s.set_pose(synth.gt_theta(model, 0.0))
        for d, (th, phi, e, det, _) in zip(frames, states):
            g = s.track_frame(d)
            dth.append(float(np.abs(g["theta"] - th).max()))
            dthd.append(float(np.abs(g["theta"] - th)[det].max()))
            ndet.append(int(det.sum()))
            dd = np.abs(g["offsets"] - phi).max(axis=1)
            dphi99.append(float(np.percentile(dd, 99)))
            dphimax.append(float(dd.max()))
            de.append(float(np.max(np.abs(g["energy"] - e) / e)))
            disp = np.linalg.norm(o.skin(g["theta"], zero)[0] - o.skin(th, zero)[0], axis=1)
            keep = disp < 5e-5
            agree_frac.append(float(keep.mean()))
            agree99.append(float(np.percentile(dd[keep], 99)) if keep.any() else float("nan"))
    return {"frames": len(frames), "theta_rad_max_determined": max(dthd), "determined_dofs": min(ndet),
            "theta_rad_max": max(dth), "offsets_mm_p99": 1e3 * max(dphi99),
            "offsets_mm_max": 1e3 * max(dphimax), "offsets_mm_p99_where_poses_agree": 1e3 * max(agree99),
            "vertices_where_poses_agree": min(agree_frac), "energy_rel_max": max(de)}


def run_precision_modes(args, model, rank, host_frames, nA, NP, sample):
    """The serving path in each [J r]^T [J r] arithmetic (FP32 cores, split-BF16x3 and 3xTF32 on the tensor
    cores): --precision-sessions streams through the frame server with batched dispatch, closed loop (host
    depth in, results out), beside the plain FP32 per-session dispatch of the same streams; one session's
    contraction-stage time; and (rank 0, one GPU) each mode's error against the oracle on the CPU-baseline
    frames, in lockstep and free-running."""
    from paper_1711_07999_gb300 import synth, trk
    out = {}
    B = args.precision_sessions
    runs = (("fp32_per_session", trk.PRECISION_FP32, trk.SERVER_DISPATCH_SESSION),
            ("fp32", trk.PRECISION_FP32, trk.SERVER_DISPATCH_BATCHED),
            ("bf16x3", trk.PRECISION_BF16X3, trk.SERVER_DISPATCH_BATCHED),
            ("tf32x3", trk.PRECISION_TF32X3, trk.SERVER_DISPATCH_BATCHED))
    for name, prec, disp in runs:
        # per-session dispatch: the grouping chosen for one session; batched: the batches' grouping
        G = 0 if disp == trk.SERVER_DISPATCH_SESSION else args.batch_jtj_group
        group = [trk.Session(synth.make_model(2, session=rank * 1000 + b, precision=prec, jtj_group=G))
                 for b in range(B)]
        for b, x in enumerate(group):
            x.set_pose(synth.gt_theta(model, (7 * b % len(host_frames)) / 30.0))
        srv = run_serving_closed_loop(group, host_frames, max(3, args.steps // 3), disp,
                                      concurrent_steps=args.server_steps)
        r = {"dispatch": "per-session" if disp == trk.SERVER_DISPATCH_SESSION else "batched",
             "serving_fps": srv["fps"], "latency_ms": srv["latency_ms"], "frames_per_launch": srv["frames_per_launch"]}
        if name != "fp32_per_session":
            group[0].set_depth(host_frames[0])
            prof = group[0].profile_iteration(reps=args.profile_reps, flush_bytes=L2_FLUSH_BYTES)
            r["resid_jtj_ms"] = prof["resid_jtj"]
            if prec != trk.PRECISION_FP32:
                # the method's contraction work: NP^2 multiply-adds per row of A, 3 split products each
                r["contraction_tflops_in_stage"] = 3 * 2 * NP * NP * nA / (prof["resid_jtj"] / 1000.0) / 1e12
            if sample is not None:
                r["lockstep_vs_oracle"] = lockstep_vs_oracle(model, prec, *sample)
                r["free_running_vs_oracle"] = errors_vs_oracle(model, prec, *sample)
        for x in group:
            x.close()
        out[name] = r
    return out


def run_reference(args, rank, world):
    from paper_1711_07999_gb300 import synth
    if rank != 0:
        return
    model = synth.make_model(2)
    o, frames = oracle_frames(model, args.warmup + args.steps, seed=synth.seed_for(2, 900))
    o.set_state(synth.gt_theta(model, 0.0), None)
    for f in range(args.warmup):
        o.track_frame(frames[f])
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        o.track_frame(frames[args.warmup + k])
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames": args.steps, "l2": "host"},
            "latency_ms": {"p50": 1000 * float(np.percentile(times, 50)), "p99": 1000 * float(np.percentile(times, 99))},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} frames of the sequence, one frame per step, FP64, 1 thread"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(sessions, dev_frames, n_seq, steps, warmup, flush):
    """B sessions, one stream and one CUDA graph each, all tracking a frame per step concurrently.
    Returns (total device ms over the timed steps, per-frame latencies in ms: from the step's start to
    the session's completion)."""
    import torch
    B = len(sessions)
    streams = [torch.cuda.Stream() for _ in range(B)]
    main = torch.cuda.current_stream()

    def step(k, record):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        ends = []
        for b, (sess, st) in enumerate(zip(sessions, streams)):
            st.wait_event(e0)
            sess.track_frame_device(dev_frames[(k + 7 * b) % n_seq].data_ptr(), st.cuda_stream)
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            ends.append(e)
        for e in ends:
            main.wait_event(e)
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(main)
        return (e0, ends, e1) if record else None

    for k in range(warmup):
        step(k, False)
    torch.cuda.synchronize()
    recs = [step(warmup + k, True) for k in range(steps)]
    torch.cuda.synchronize()
    total = sum(e0.elapsed_time(e1) for e0, _, e1 in recs)
    lat = [e0.elapsed_time(e) for e0, ends, _ in recs for e in ends]
    return total, lat


def run_schedule(sessions, dev_frames, n_seq, steps, warmup, flush):
    """The sessions under the schedule the autotuner picks (groups of fused batches on concurrent streams,
    tuned on the warm-up frames), each step one frame of every session; device-timed with CUDA events on
    the launching stream, L2 flushed before every step.  A frame's latency is its step's time (every
    group starts at the step's start)."""
    import torch
    from paper_1711_07999_gb300 import trk
    B = len(sessions)
    st = torch.cuda.Stream()

    def ptrs(k):
        return [dev_frames[(k + 7 * b) % n_seq].data_ptr() for b in range(B)]

    with trk.Schedule(sessions) as sc:
        cfg, _ = sc.autotune(ptrs(0), reps=2)
        for k in range(warmup):
            sc.track_device(ptrs(k), st.cuda_stream)
        torch.cuda.synchronize()
        ev = []
        for k in range(steps):
            with torch.cuda.stream(st):  # the flush is done before the step starts (same stream)
                flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sc.track_device(ptrs(warmup + k), st.cuda_stream)
            e1.record(st)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        t = np.array([a.elapsed_time(b) for a, b in ev])
    return {"config": cfg, "total_ms": float(t.sum()),
            "latency_ms": {"p50": float(np.percentile(t, 50)), "p99": float(np.percentile(t, 99))}}


def run_batched_e2e(sessions, host_frames, n_seq, steps, flush):
    """The same through the public host-buffer call, one host thread per session (the calls release the
    interpreter lock); returns (wall seconds, per-call latencies in ms)."""
    import threading
    import torch
    B = len(sessions)
    lat = [[] for _ in range(B)]
    barrier = threading.Barrier(B + 1)

    def worker(b):
        barrier.wait()
        for k in range(steps):
            t0 = time.perf_counter()
            sessions[b].track_frame(host_frames[(k + 7 * b) % n_seq], want_offsets=True)
            lat[b].append(1000 * (time.perf_counter() - t0))
        barrier.wait()

    flush.fill_(3)
    torch.cuda.synchronize()
    th = [threading.Thread(target=worker, args=(b,)) for b in range(B)]
    for t in th:
        t.start()
    barrier.wait()
    t0 = time.perf_counter()
    barrier.wait()
    wall = time.perf_counter() - t0
    for t in th:
        t.join()
    return wall, [x for l in lat for x in l]


def run_serving(sessions, host_frames, n_seq, duration_s, fps, seed):
    """Poisson arrivals (rate fps per stream, random phase) submitted through the frame server at their
    arrival times; one collector thread per stream.  Returns frames/s and submit -> completion latency."""
    import threading
    from paper_1711_07999_gb300 import trk
    rng = np.random.default_rng(seed)
    N = len(sessions)
    arrivals = []
    for b in range(N):
        t = rng.uniform(0, 1.0 / fps)
        while t < duration_s:
            arrivals.append((t, b))
            t += rng.exponential(1.0 / fps)
    arrivals.sort()
    budget = sum(x.info()["device_bytes"] for x in sessions) + (1 << 30)  # not binding here (admission: below)
    tickets = [[] for _ in range(N)]
    done = [0] * N
    with trk.Server(budget, max_inflight=N) as sv:
        for x in sessions:
            sv.attach(x)
        cond = threading.Condition()

        def collector(b):
            k = 0
            while True:
                with cond:
                    while k >= len(tickets[b]) and not finished[0]:
                        cond.wait(0.01)
                    if k >= len(tickets[b]):
                        return
                    t = tickets[b][k]
                sv.wait(sessions[b], t, timeout_us=30_000_000, want_offsets=True)
                done[b] += 1
                k += 1

        finished = [False]
        th = [threading.Thread(target=collector, args=(b,)) for b in range(N)]
        for t in th:
            t.start()
        nxt = [0] * N
        lag = []
        t0 = time.perf_counter()
        for ta, b in arrivals:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            lag.append(time.perf_counter() - t0 - ta)
            tk = sv.submit(sessions[b], host_frames[(nxt[b] + 7 * b) % n_seq])
            nxt[b] += 1
            with cond:
                tickets[b].append(tk)
                cond.notify_all()
        with cond:
            finished[0] = True
            cond.notify_all()
        t_sub = time.perf_counter() - t0
        for t in th:
            t.join()
        wall = time.perf_counter() - t0
        st = sv.stats()
        for x in sessions:
            sv.detach(x)
    n = sum(done)
    # served frames over the span from the first arrival to the last completion (the drain included)
    return {"streams": N, "offered_fps": N * fps, "arrivals": "poisson", "frames": n, "seconds": round(wall, 3),
            "achieved_fps": n / wall, "drain_ms": (wall - t_sub) * 1e3,
            "submit_lag_ms": {"p50": float(np.percentile(lag, 50)) * 1e3, "max": float(np.max(lag)) * 1e3},
            "latency_ms": {"p50": st["latency_p50_us"] / 1000,
                                                      "p99": st["latency_p99_us"] / 1000,
                                                      "max": st["latency_max_us"] / 1000}}


def run_serving_closed_loop(sessions, host_frames, frames_per_stream, dispatch, max_batch=64, concurrent_steps=4):
    """Saturated serving: every stream submits its next frame as soon as its previous one is collected
    (closed loop, one thread per stream), through the frame server in the given dispatch mode.  Returns
    frames/s over the wall time and the server's submit -> completion latency."""
    import threading
    from paper_1711_07999_gb300 import trk
    N = len(sessions)
    budget = sum(x.info()["device_bytes"] for x in sessions) + (1 << 30)
    with trk.Server(budget, max_inflight=N, dispatch=dispatch, max_batch=max_batch,
                    concurrent_steps=concurrent_steps) as sv:
        for x in sessions:
            sv.attach(x)
        for b, x in enumerate(sessions):  # warm-up frame (frame graphs, step buffers, staging)
            sv.wait(x, sv.submit(x, host_frames[b % len(host_frames)]), timeout_us=60_000_000, want_offsets=False)
        barrier = threading.Barrier(N + 1)
        lat = [[] for _ in range(N)]

        def stream(b):
            barrier.wait()
            for k in range(frames_per_stream):
                t0 = time.perf_counter()
                t = sv.submit(sessions[b], host_frames[(k + 7 * b) % len(host_frames)])
                sv.wait(sessions[b], t, timeout_us=60_000_000, want_offsets=True)
                lat[b].append(1e3 * (time.perf_counter() - t0))
            barrier.wait()

        th = [threading.Thread(target=stream, args=(b,)) for b in range(N)]
        for t in th:
            t.start()
        st0 = sv.stats()
        barrier.wait()
        t0 = time.perf_counter()
        barrier.wait()
        wall = time.perf_counter() - t0
        for t in th:
            t.join()
        st = sv.stats()
        for x in sessions:
            sv.detach(x)
    n = N * frames_per_stream
    steps = st["steps"] - st0["steps"]
    la = np.concatenate([np.array(x) for x in lat])
    return {"streams": N, "frames": n, "seconds": round(wall, 3), "fps": n / wall,
            "frames_per_launch": n / max(steps, 1),
            "latency_ms": {"p50": float(np.percentile(la, 50)), "p99": float(np.percentile(la, 99)),
                           "max": float(la.max())},
            "h2d_bytes_per_frame": int(sessions[0].W * sessions[0].H * 4)}


def run_admission_serving(args, rank):
    """Streams of uneven sessions arriving over time under an HBM budget that binds: --admission-streams
    sessions of the random-tree bodies; stream starts form a Poisson process (rate: all streams within
    about a second); each stream, once admitted (attach succeeds within the budget, otherwise it waits in
    arrival order until a departing stream frees enough), submits --admission-frames frames at Poisson
    arrivals of 30 frames/s, collects them and leaves (detach).  Reports served frames/s, submit ->
    completion latency, admission waits and the peak of the admitted device bytes."""
    import threading
    import torch
    from paper_1711_07999_gb300 import synth, trk
    N, K, fps = args.admission_streams, args.admission_frames, 30.0
    budget = int(args.admission_budget_gib * (1 << 30))
    rng = np.random.default_rng(synth.seed_for(5, rank))
    models = [synth.make_model(4, session=20000 + rank * 1000 + k) for k in range(N)]
    frames = []
    for i, m in enumerate(models):
        r = np.random.default_rng(synth.seed_for(5, 100 + i))
        with trk.Session(m) as s:
            frames.append([synth.add_noise(s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)),
                                           4, r) for f in range(4)])
    torch.cuda.synchronize()
    base_free = torch.cuda.mem_get_info()[0]
    # the sessions are created evicted: no device memory until the server admits them
    sess = [trk.Session(m, evicted=True) for m in models]
    for m, s in zip(models, sess):
        s.set_pose(synth.gt_theta(m, 0.0))
    need = [s.info()["device_bytes"] for s in sess]
    starts = np.cumsum(rng.exponential(1.0 / N, N))
    gaps = [rng.exponential(1.0 / fps, K) for _ in range(N)]
    torch.cuda.synchronize()
    lock = threading.Condition()
    queue = []  # streams waiting for admission, in arrival order
    used = [0]
    peak = [0]
    waits, served = [0.0] * N, [0] * N
    with trk.Server(budget, max_inflight=N) as sv:
        def admit(b, t0):
            with lock:
                queue.append(b)
                while True:
                    if queue[0] == b:
                        try:
                            sv.attach(sess[b])
                            used[0] += need[b]
                            peak[0] = max(peak[0], used[0])
                            queue.pop(0)
                            lock.notify_all()
                            return time.perf_counter()
                        except trk.TrkError as e:
                            if e.status != trk.TRK_ERR_NO_CAPACITY:
                                raise
                    lock.wait(0.005)

        def stream(b, t0):
            if need[b] > budget:  # never admissible
                waits[b] = float("nan")
                return
            dt = t0 + starts[b] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            t_arrive = time.perf_counter()
            t_adm = admit(b, t0)
            waits[b] = t_adm - t_arrive
            tickets, t = [], t_adm
            for k in range(K):
                t += gaps[b][k]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets.append(sv.submit(sess[b], frames[b][k % 4]))
            for tk in tickets:
                sv.wait(sess[b], tk, timeout_us=60_000_000, want_offsets=True)
                served[b] += 1
            with lock:
                sv.detach(sess[b])
                used[0] -= need[b]
                lock.notify_all()

        dev_peak = [0]
        sampling = [True]

        def sample_memory():  # device memory in use beyond what it was before the sessions existed
            while sampling[0]:
                dev_peak[0] = max(dev_peak[0], base_free - torch.cuda.mem_get_info()[0])
                time.sleep(0.002)

        mon = threading.Thread(target=sample_memory, daemon=True)
        mon.start()
        t0 = time.perf_counter()
        th = [threading.Thread(target=stream, args=(b, t0)) for b in range(N)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        wall = time.perf_counter() - t0
        sampling[0] = False
        mon.join()
        st = sv.stats()
    for s in sess:
        s.close()
    w = np.array([x for x in waits if x == x]) * 1e3
    return {"streams": N, "frames_per_stream": K, "fps_per_stream": fps, "budget_bytes": budget,
            "sum_of_session_bytes": int(sum(need)), "peak_admitted_bytes": int(peak[0]),
            "peak_device_bytes_in_use": int(dev_peak[0]),
            "device_memory_note": "cudaMemGetInfo sampled every 2 ms against its value before the sessions existed "
                                  "(sessions created evicted; the server's step buffers included)",
            "frames_per_launch": st["mean_frames_per_step"],
            "streams_that_waited": int((w > 1.0).sum()), "streams_over_budget": int(N - len(w)),
            "admission_wait_ms": {"p50": float(np.percentile(w, 50)), "p99": float(np.percentile(w, 99)),
                                  "max": float(w.max())},
            "frames": int(sum(served)), "seconds": round(wall, 3), "achieved_fps": sum(served) / wall,
            "latency_ms": {"p50": st["latency_p50_us"] / 1000, "p99": st["latency_p99_us"] / 1000,
                           "max": st["latency_max_us"] / 1000}}


def run_uneven(args, rank, flush):
    """The uneven batch: --uneven-sessions sessions of the random-tree bodies (5k-200k vertices, 12-40
    bones, three image sizes), the same frames stepped one by one, on one stream each, as one fused
    batch, and under the schedule the autotuner picks (tuned on warm-up frames).  Device-timed steps,
    L2 flushed before each."""
    import torch
    from paper_1711_07999_gb300 import synth, trk
    B = args.uneven_sessions
    models = [synth.make_model(4, session=rank * 10000 + k, jtj_group=args.uneven_jtj_group) for k in range(B)]
    sess = [trk.Session(m) for m in models]
    nf = 4
    frames = []
    for i, (m, s) in enumerate(zip(models, sess)):
        rng = np.random.default_rng(synth.seed_for(4, 7000 + rank * 10000 + i))
        frames.append([torch.from_numpy(synth.add_noise(
            s.render_depth(synth.gt_theta(m, f / 30.0), synth.gt_offsets(m, f / 30.0)), 4, rng)).cuda()
            for f in range(nf)])
        s.set_pose(synth.gt_theta(m, 0.0))
    st = torch.cuda.Stream()
    steps = max(3, args.steps // 3)

    def timed(fn, n):
        for k in range(3):
            fn(k)
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(n):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(3 + k)
            e1.record(st)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / n

    def ptrs(k):
        return [frames[i][k % nf].data_ptr() for i in range(B)]

    def one_by_one(k):
        for i, s in enumerate(sess):
            s.track_frame_device(frames[i][k % nf].data_ptr(), st.cuda_stream)

    modes = set(args.uneven_modes.split(","))
    out = {"sessions": B, "total_verts": int(sum(s.V for s in sess)),
           "total_pixels": int(sum(s.W * s.H for s in sess)), "steps": steps}
    if "one_by_one" in modes:
        out["one_by_one_fps"] = B * 1000.0 / timed(one_by_one, 2)
    strs = [torch.cuda.Stream() for _ in sess]

    def streams(k):
        e = torch.cuda.Event()
        e.record(st)
        ends = []
        for i, (s, x) in enumerate(zip(sess, strs)):
            x.wait_event(e)
            s.track_frame_device(frames[i][k % nf].data_ptr(), x.cuda_stream)
            ee = torch.cuda.Event()
            ee.record(x)
            ends.append(ee)
        for ee in ends:
            st.wait_event(ee)
    if "streams" in modes:
        out["streams_fps"] = B * 1000.0 / timed(streams, steps)
    if "fused" in modes:
        with trk.Batch(sess) as b:
            out["fused_batch_fps"] = B * 1000.0 / timed(lambda k: b.track_device(ptrs(k), st.cuda_stream), steps)
            for m, s in zip(models, sess):  # profiled at the first frame's state (pose at its ground truth)
                s.set_pose(synth.gt_theta(m, 0.0))
            prof = b.profile(ptrs(0), reps=3, flush_bytes=L2_FLUSH_BYTES)
        out["fused_stage_roofline"] = fused_rooflines(sess, frames, prof)
    if "schedule" in modes:
        with trk.Schedule(sess) as sc:
            cfg, _ = sc.autotune(ptrs(0), reps=2)
            out["schedule"] = cfg
            out["schedule_fps"] = B * 1000.0 / timed(lambda k: sc.track_device(ptrs(k), st.cuda_stream), steps)
    for s in sess:
        s.close()
    return out


def fused_rooflines(sess, frames, prof):
    counts = [session_counts(s, frames[i][0].cpu().numpy()) for i, s in enumerate(sess)]
    pk = peaks()
    roof = {}
    for stage in ("skin", "raster", "visibility", "associate", "resid_jtj", "reduce", "lm_eval", "shape"):
        amount = sum(algorithmic(stage, **c)[1] for c in counts)
        gbs = amount / (prof[stage] / 1000.0) / 1e9
        roof[stage] = {"ms": round(prof[stage], 4), "algorithmic_bytes": int(amount), "achieved_gbs": round(gbs, 1),
                       "frac": round(gbs / pk["hbm_gbs"], 4)}
    return {"peak_gbs": pk["hbm_gbs"], "peak_source": pk["src"] + " (burst copy)",
            "l2": "flushed before each stage", "stages": roof}


def run_experiments(args, rank):
    """The paper's experiment conditions (Sec. 5) on the synthetic sequence with its ground truth: full
    tracking, shape-match and smooth-bind, each tracking the same frames from the true first pose, and full
    tracking with the raster-ID association (accuracy against cost).  Reported per condition: pose accuracy
    (area under the joint-accuracy curve up to 10 cm, mean joint error), reconstruction error (visible
    vertex to the nearest observed point) and the association stage's time (CUDA events, cold L2)."""
    from paper_1711_07999_gb300 import metrics, synth, trk
    n = args.experiment_frames
    out = {"frames": n, "auc_up_to_m": 0.1, "modes": {}}
    for name, mode, assoc in (("track", trk.MODE_TRACK, 0), ("shape_match", trk.MODE_SHAPE_MATCH, 0),
                              ("smooth_bind", trk.MODE_SMOOTH_BIND, 0), ("track_raster_id", trk.MODE_TRACK, 1)):
        model = synth.make_model(2, session=rank, mode=mode, association=assoc)
        cam = model["camera"]
        joints = metrics.joint_links(model["skeleton"])
        errs, recon = [], []
        with trk.Session(model) as s:
            frames = render_sequence(model, s, n, seed=synth.seed_for(2, 800 + rank))
            s.set_pose(synth.gt_theta(model, 0.0))
            for f in range(n):
                g = s.track_frame(frames[f], want_offsets=False)
                gt = trk.joint_positions(model["skeleton"], synth.gt_theta(model, f / 30.0))[joints]
                est = trk.joint_positions(model["skeleton"], g["theta"])[joints]
                errs.append(metrics.joint_errors(est, gt))
                verts = s.read("VERTS")[:, :3]
                vis = s.read("VISPIX") >= 0
                recon.append(metrics.reconstruction_error(verts, vis, frames[f], cam["fx"], cam["fy"], cam["cx"],
                                                          cam["cy"]))
            s.set_depth(frames[0])
            prof = s.profile_iteration(reps=5, flush_bytes=L2_FLUSH_BYTES)
        e = np.concatenate(errs)
        r = np.concatenate(recon)
        out["modes"][name] = {"joint_auc": round(metrics.auc(e, 0.1), 4), "joint_err_mean_mm": round(1e3 * e.mean(), 3),
                              "joint_err_max_mm": round(1e3 * e.max(), 3),
                              "recon_err_mean_mm": round(1e3 * r.mean(), 4),
                              "recon_err_median_mm": round(1e3 * float(np.median(r)), 4),
                              "associate_ms": round(prof["associate"], 5)}
    return out


def summary_of(line):
    """The figures a reader wants first: throughput plain / batched / end to end, the serving comparison
    per arithmetic, parity in lockstep with the oracle, the admission run's device memory against its
    budget, the roofline fraction."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    out = {"plain_fps": g(line, "plain", "value"), "batched_fps": line["value"], "e2e_fps": g(line, "e2e", "value"),
           "latency_p99_ms": g(line, "latency_ms", "p99"), "roofline_frac": g(line, "roofline", "frac"),
           "roofline_kernel": g(line, "roofline", "kernel")}
    prec = line.get("precision") or {}
    out["serving_fps"] = {k: round(v["serving_fps"], 1) for k, v in prec.items() if "serving_fps" in v}
    out["serving_p99_ms"] = {k: round(v["latency_ms"]["p99"], 2) for k, v in prec.items() if "latency_ms" in v}
    out["lockstep_vs_oracle"] = {
        k: {q: v["lockstep_vs_oracle"][q] for q in ("theta_rad_max", "offsets_mm_max", "energy_rel_max_matched",
                                                    "nontie_mismatches", "lm_decisions_equal")}
        for k, v in prec.items() if "lockstep_vs_oracle" in v}
    adm = line.get("admission_serving") or {}
    if adm:
        out["admission"] = {q: adm.get(q) for q in ("budget_bytes", "peak_device_bytes_in_use", "achieved_fps")}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1711_07999_gb300 import synth, trk

    torch.cuda.set_device(local_rank)
    if args.only == "uneven":  # the uneven batch alone (a diagnostic line, not the benchmark line)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        return {"uneven": run_uneven(args, rank, flush)} if rank == 0 else None
    if args.only == "schedule":  # the headline's batched step alone, for profilers (a diagnostic line)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        m0 = synth.make_model(2, session=rank)
        group = [trk.Session(synth.make_model(2, session=rank * 1000 + b, jtj_group=args.batch_jtj_group))
                 for b in range(args.sessions)]
        fr = render_sequence(m0, group[0], max(args.frames, 1), seed=synth.seed_for(2, 500 + rank))
        dev = torch.from_numpy(fr).cuda()
        for b, x in enumerate(group):
            x.set_pose(synth.gt_theta(m0, (7 * b % len(fr)) / 30.0))
        sched = run_schedule(group, dev, len(fr), args.steps, args.warmup, flush)
        for x in group:
            x.close()
        return {"schedule": sched["config"], "sessions": args.sessions,
                "fps": args.sessions * args.steps / (sched["total_ms"] / 1000.0)} if rank == 0 else None
    prec = PRECISIONS[args.precision]
    model = synth.make_model(2, session=rank, precision=prec)
    sess = trk.Session(model)
    info = sess.info()
    n_seq = max(args.frames, 1)
    frames = render_sequence(model, sess, n_seq, seed=synth.seed_for(2, 500 + rank))
    H, W = frames.shape[1:]
    host = torch.from_numpy(frames).pin_memory()
    dev = host.cuda()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    sess.set_pose(synth.gt_theta(model, 0.0))

    def frame_dev(k):
        sess.track_frame_device(dev[k % n_seq].data_ptr(), stream.cuda_stream)

    # warm-up (also builds the CUDA graph)
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            frame_dev(k)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                frame_dev(args.warmup + k)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times = np.array([a.elapsed_time(b) for a, b in ev])  # ms
    total_ms = float(times.sum())
    res = sess.read_result(want_offsets=False)
    max_ms = max_over_ranks(total_ms, world)
    value = whole_job_rate(world, args.steps, max_ms / 1000.0)

    # end to end through the public call: host pinned depth in, Theta / Phi / energies out
    e2e_t = []
    for k in range(args.steps):
        flush.fill_((k + 7) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sess.track_frame(host[(args.warmup + args.steps + k) % n_seq].numpy(), want_offsets=True)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = whole_job_rate(world, args.steps, max_over_ranks(sum(e2e_t), world))

    # per-stage kernel times (CUDA events on the launching stream, cold L2), dominant kernel, roofline
    sess.set_depth(frames[(args.warmup + 2 * args.steps) % n_seq])
    prof = sess.profile_iteration(reps=args.profile_reps, flush_bytes=L2_FLUSH_BYTES)
    P, S = model["params"]["pose_iters"], model["params"]["shape_iters"]
    per_frame = {}
    for st, ms in prof.items():
        n = P + S if st in ("skin", "raster", "visibility", "associate") else (S if st == "shape" else P)
        per_frame[st] = ms * n
    dom = max(per_frame, key=per_frame.get)
    cnt = session_counts(sess, frames[(args.warmup + 2 * args.steps) % n_seq])
    nA, NP = cnt["nA"], cnt["NP"]
    kind, amount = algorithmic(dom, **cnt)
    pk = peaks()
    dur_s = prof[dom] / 1000.0
    if kind == "hbm":
        achieved = amount / dur_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": ncu_traffic(dom), "kernel": dom,
                "algorithmic_bytes": amount, "peak_source": pk["src"] + " (burst copy)"}
    else:
        achieved = amount / dur_s / 1e12
        fp64_peak = 1.25  # TFLOP/s, nominal dense FP64 of GB300 (no measured figure in MEASURED_PEAKS.json)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": ncu_traffic(dom), "kernel": dom,
                "algorithmic_flops": amount, "peak_source": "nominal FP64 rate"}
    roof["note"] = ROOFLINE_NOTES.get(dom, "")
    h2d = W * H * 4
    d2h = info["n_links"] * 8 + (P + S) * 8 + info["n_verts"] * 12 + 8  # trk_track_frame's copies
    d2h_srv = info["n_links"] * 8 + (P + S) * 8 + info["n_verts"] * 16 + 16  # the server's mapped staging
    # batched: B sessions of the same workload on this GPU, three ways (device-timed, depth resident):
    # one stream and graph per session; one fused batch per group of the autotuned schedule (the headline);
    # and end to end through the frame server (host depth in, results out, batched dispatch)
    batched = None
    B = args.sessions
    if B > 1:
        group = [trk.Session(synth.make_model(2, session=rank * 1000 + b, precision=prec,
                                              jtj_group=args.batch_jtj_group)) for b in range(B)]
        for b, x in enumerate(group):
            x.set_pose(synth.gt_theta(model, (7 * b % n_seq) / 30.0))
        tb, lat_b = run_batched(group, dev, n_seq, args.steps, args.warmup, flush)
        streams_fps = whole_job_rate(world, B * args.steps, max_over_ranks(tb, world) / 1000.0)
        for b, x in enumerate(group):
            x.set_pose(synth.gt_theta(model, (7 * b % n_seq) / 30.0))
        with ClockSampler(local_rank) as clk_b:
            sched = run_schedule(group, dev, n_seq, args.steps, args.warmup, flush)
        ts_max = max_over_ranks(sched["total_ms"], world)
        # the batched step's stages, one launch each over all B sessions (a fused batch profiled at the
        # sequence's first frame, cold L2): the dominant stage and its roofline
        for x in group:
            x.set_pose(synth.gt_theta(model, 0.0))
        with trk.Batch(group) as fb:
            bprof = fb.profile([dev[0].data_ptr()] * B, reps=3, flush_bytes=L2_FLUSH_BYTES)
        bcounts = [session_counts(x, frames[0]) for x in group]
        host_frames = [host[i].numpy() for i in range(n_seq)]
        for b, x in enumerate(group):
            x.set_pose(synth.gt_theta(model, (7 * b % n_seq) / 30.0))
        e2e_srv = run_serving_closed_loop(group, host_frames, max(3, args.steps // 2), trk.SERVER_DISPATCH_BATCHED,
                                          concurrent_steps=args.server_steps)
        e2e_fps = whole_job_rate(world, e2e_srv["frames"] / world, max_over_ranks(e2e_srv["seconds"], world))
        batched = {"sessions": B, "jtj_group": args.batch_jtj_group, "clocks": clk_b.summary(),
                   "stage_ms": {k: round(v, 5) for k, v in bprof.items()},
                   "value": whole_job_rate(world, B * args.steps, ts_max / 1000.0),
                   "ms_per_step": ts_max / args.steps, "schedule": sched["config"],
                   "latency_ms": sched["latency_ms"],
                   "streams_fps": streams_fps,
                   "streams_latency_ms": {"p50": float(np.percentile(lat_b, 50)), "p99": float(np.percentile(lat_b, 99))},
                   "e2e": {"value": e2e_fps, "p50_ms": e2e_srv["latency_ms"]["p50"],
                           "p99_ms": e2e_srv["latency_ms"]["p99"], "server": e2e_srv}}
        serving = None
        if args.serve_streams > 0:
            streams = group[:args.serve_streams]
            for b, x in enumerate(streams):
                x.set_pose(synth.gt_theta(model, (7 * b % n_seq) / 30.0))
            serving = run_serving(streams, host_frames, n_seq, args.serve_seconds, 30.0, synth.seed_for(5, rank))
        batched["serving"] = serving
        for x in group:
            if x is not sess:
                x.close()
    line = None
    cpu, sample = None, None
    if rank == 0 and world == 1 and args.cpu_frames > 0:
        cpu, frames_o, states_o, o_ref = cpu_baseline(model, args.cpu_frames)
        sample = (frames_o, states_o, o_ref)
        if args.cpu_all_cores_frames > 0:
            cpu["all_cores"] = cpu_baseline_all_cores(args.cpu_all_cores_frames)
    precision = None
    if args.precision_modes and B > 1:
        precision = run_precision_modes(args, model, rank, [host[i].numpy() for i in range(n_seq)], nA, NP, sample)
    uneven = run_uneven(args, rank, flush) if args.uneven_sessions > 0 else None
    admission = run_admission_serving(args, rank) if args.admission_streams > 0 else None
    experiments = run_experiments(args, rank) if (args.experiment_frames > 0 and rank == 0) else None
    if batched is not None:  # the headline is the batched step: its dominant stage's roofline
        pf = {st: ms * ((P + S) if st in ("skin", "raster", "visibility", "associate") else (S if st == "shape" else P))
              for st, ms in batched["stage_ms"].items()}
        dom_b = max(pf, key=pf.get)
        kind_b, amount_b = "hbm", 0
        for c in bcounts:
            kind_b, a_b = algorithmic(dom_b, **c)
            amount_b += a_b
        if kind_b == "hbm":
            ach = amount_b / (batched["stage_ms"][dom_b] / 1000.0) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                    "traffic": ncu_traffic(dom_b + "_batch"), "kernel": dom_b,
                    "launch": f"one launch over {B} sessions (fused batch)", "algorithmic_bytes": amount_b,
                    "peak_source": pk["src"] + " (burst copy)", "note": ROOFLINE_NOTES.get(dom_b, "")}
        batched["stage_share"] = {k: round(v / sum(pf.values()), 4) for k, v in pf.items()}
    if rank == 0:
        plain = {"value": value, "ms_per_step": max_ms / args.steps,
                 "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                 "e2e": {"value": e2e_value, "p50_ms": 1000 * float(np.percentile(e2e_t, 50)),
                         "p99_ms": 1000 * float(np.percentile(e2e_t, 99))}}
        head = batched if batched is not None else plain
        line = {
            "metric": METRIC, "value": head["value"], "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_verts": info["n_verts"], "n_tris": info["n_tris"],
                       "dof": info["n_links"], "image": f"{W}x{H}", "pose_iters": P, "shape_iters": S,
                       "sessions_per_gpu": B if batched is not None else 1,
                       "batching": (f"autotuned schedule: {batched['schedule']['groups']} groups of fused batches "
                                    "(one launch per stage over a group's sessions, one CUDA graph per group) on "
                                    "concurrent streams; e2e through the frame server (batched dispatch)")
                       if batched else "none",
                       "jtj_group": args.batch_jtj_group if batched else info["jtj_group"],
                       "l2": "flushed (256 MiB write) before every step",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": head["latency_ms"],
            "e2e": {"value": head["e2e"]["value"], "unit": "frames/s", "h2d_bytes_per_step": h2d * B,
                    "d2h_bytes_per_step": (d2h_srv if batched is not None else d2h) * B,
                    "p50_ms": head["e2e"]["p50_ms"], "p99_ms": head["e2e"]["p99_ms"],
                    "path": "trk_server_submit / trk_server_wait, host depth in, results out" if batched is not None
                    else "trk_track_frame, host depth in, results out"},
            "plain": plain,
            "batched": batched,
            "precision": precision,
            "uneven": uneven,
            "admission_serving": admission,
            "experiments": experiments,
            "gpu_launches": (batched["schedule"]["groups"] * (info["kernels_per_frame"] + P + S) * args.steps
                             if batched is not None else info["kernels_per_frame"] * args.steps),
            "roofline": roof,
            "stage_ms": {k: round(v, 5) for k, v in prof.items()},
            "stage_share": {k: round(v / sum(per_frame.values()), 4) for k, v in per_frame.items()},
            "clocks": batched["clocks"] if batched is not None else clk.summary(),
            "plain_clocks": clk.summary(),
            "cpu_baseline": cpu,
            "check": {"last_energy": float(res["energy"][P - 1]), "assoc_px": res["n_assoc_px"]},
        }
        line["summary"] = summary_of(line)  # last, so that a truncated tail of the line still shows it
    sess.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=150, help="length of the pre-rendered sequence")
    ap.add_argument("--cpu-frames", type=int, default=4, help="oracle frames of the CPU baseline sample")
    ap.add_argument("--cpu-all-cores-frames", type=int, default=2,
                    help="frames per core of the all-cores oracle baseline (0: skip)")
    ap.add_argument("--profile-reps", type=int, default=20)
    ap.add_argument("--sessions", type=int, default=64, help="sessions of the batched measurement")
    ap.add_argument("--batch-jtj-group", type=int, default=4, choices=[0, 1, 2, 4],
                    help="[J r] grouping of the batched sessions (4: fewer block partials; 0: by mesh size)")
    ap.add_argument("--server-steps", type=int, default=4, help="concurrent batched steps of the frame server")
    ap.add_argument("--precision-sessions", type=int, default=64,
                    help="streams of the serving run in each precision mode")
    ap.add_argument("--serve-streams", type=int, default=32, help="Poisson streams (30 fps each) of the serving run")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32",
                    help="arithmetic of [J r]^T [J r] in the plain and batched sessions")
    ap.add_argument("--only", choices=["all", "plain", "uneven", "schedule"], default="all",
                    help="plain: the one-session and batched measurements only; uneven: the uneven batch only; "
                         "schedule: the batched step alone (for profilers)")
    ap.add_argument("--uneven-modes", default="one_by_one,streams,fused,schedule")
    ap.add_argument("--admission-streams", type=int, default=32,
                    help="streams of uneven sessions arriving under an HBM budget (0: skip)")
    ap.add_argument("--admission-frames", type=int, default=30)
    ap.add_argument("--admission-budget-gib", type=float, default=1.0)
    ap.add_argument("--experiment-frames", type=int, default=30,
                    help="frames of the sequence tracked in each of the paper's experiment conditions")
    ap.add_argument("--uneven-jtj-group", type=int, default=0, choices=[0, 1, 2, 4],
                    help="vertex blocks per [J r] block of the uneven sessions (0: chosen from each mesh's size)")
    ap.add_argument("--uneven-sessions", type=int, default=64,
                    help="sessions of the uneven batch (one by one / streams / fused batch / tuned schedule)")
    ap.add_argument("--precision-modes", type=int, default=1,
                    help="also time the tensor-core [J r]^T [J r] modes and their error against the oracle")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only == "plain":
        args.uneven_sessions, args.precision_modes, args.experiment_frames, args.admission_streams = 0, 0, 0, 0
    rank, world, local_rank = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
