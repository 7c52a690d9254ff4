"""Benchmark: bundle-adjustment solves per second on the sliding-window workload.

Workload (one "step"): one batched solve of B problems of the sliding-window
shape -- 22 buffered frames, 96 patches per frame (2112 patches), every patch
connected to the frames within +-13 of its source frame (39,552 edges), the
last 10 poses free, 2 Gauss-Newton iterations -- through the C ABI on device
buffers.  B = two problems per SM by default (296 on a B300: one work item per
problem fills exactly one wave), so one step's inputs (~290 MB) exceed the
126 MB L2 and every iteration re-reads them from HBM.  Inputs are seeded synthetic
scenes (paper_2208_04726_b300/scenes.py).

Also measured and reported on the same JSON line:
  plain     the same problems solved one per call, back to back (latency p50/p99)
  e2e       the batched solve through the host-buffer entry point, host<->device
            copies of every step's inputs and results inside the timed region
  roofline  the linearise/Schur kernel against the FP32-ALU or HBM roofline
  parity    sampled problems of the first timed-configuration solve vs the FP64 oracle
  cpu_baseline  the FP64 oracle timed on this host's cores on a bounded sample
  serving   256 VO sessions (uneven shapes) with device-resident state, Poisson
            requests at 2000/s: p50/p99 latency and solves/s, continuous
            batching vs one launch per solve, plus a saturated closed loop;
            and the Default/Fast mix as 256 served sliding windows (a request
            appends a frame and solves), the same measurements
  stress    64 large-window sessions (64 frames, 32 free poses, 4 iterations)
  grad      16 eight-frame problems: forward, the pose supervision loss of
            Sec. 3.4 on the device, and the backward to targets and weights
  window    256 sliding windows kept on the device: append a frame to each,
            then one batched solve
  vo_mix    the paper's Default and Fast configurations as one mix of 256
            sliding-window sessions: initialisation (8 frames, 12 solves),
            then frames
  corr      the correlation features (Sec. 3.2) of every edge of the window
            graph on the tensor cores

``--impl reference`` times the FP64 oracle (the reference arm) instead.
Launch: ``python bench.py --gpus N --steps K --warmup W`` (torchrun for N > 1,
one replica per GPU, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BA solves/s (2 GN iters) + p50/p99 latency, batched vs plain, at ≤1e-4 vs FP64"
WORKLOAD = ("sliding window: N=22 frames, 96 patches/frame (2112 patches), radius 13 (39552 edges), "
            "last 10 poses free, 2 GN iterations")
PEAK_ALU_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=0, help="problems per step (0: two per SM)")
    ap.add_argument("--distinct", type=int, default=64, help="distinct seeded scenes, tiled to --batch")
    ap.add_argument("--plain", type=int, default=200, help="one-problem solves timed for the plain form")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--parity-samples", type=int, default=2)
    ap.add_argument("--serving", type=int, default=1, help="run the serving measurement (Poisson sessions)")
    ap.add_argument("--tf32", type=int, default=1, help="also time the other Schur modes (tensor cores on the fused path, FP32 assembly on the wide windows)")
    ap.add_argument("--grad", type=int, default=16, help="problems of the differentiation workload; 0 skips")
    ap.add_argument("--window", type=int, default=256, help="sliding windows maintained on the device; 0 skips")
    ap.add_argument("--vo-mix", type=int, default=1, help="the Default/Fast serving mix with initialisation; 0 skips")
    ap.add_argument("--corr", type=int, default=1, help="the correlation features of the window graph; 0 skips")
    ap.add_argument("--stress", type=int, default=64,
                    help="large-window sessions timed (64 frames, 256 patches each, radius 24, 32 free poses, 4 "
                         "iterations); 0 skips")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------- work accounting

def algorithmic_work(scene):
    """Algorithmic FP32 flops and HBM bytes of one linearise/Schur pass over a
    problem: 200 flops and 24 bytes per edge (projection, residual, Jacobians,
    weighted products; kk, jj, target, weight), 20 bytes per patch, and per
    patch 36 f (f + 1) + 12 f flops for its upper-triangle Schur blocks and
    right-hand side, f = free poses the patch touches."""
    i = scene.anchor[scene.kk]
    nonself = i != scene.jj
    E = int(nonself.sum())
    t0 = scene.t0
    f = np.zeros(scene.n_patches, np.int64)
    m = nonself & (scene.jj >= t0)
    np.add.at(f, scene.kk[m], 1)
    f += ((scene.anchor >= t0) & np.isin(np.arange(scene.n_patches), scene.kk[nonself])).astype(np.int64)
    flops = 200.0 * E + float(np.sum(36 * f * (f + 1) + 12 * f))
    bytes_ = 24.0 * scene.n_edges + 20.0 * scene.n_patches
    return flops, bytes_


def stress_bench(n_sessions, steps, stream, hbm_peak, mode=0):
    """Large-window workload: n_sessions problems of 64 frames x 256 patches
    (16,384), radius 24 (649,216 edges), the last 32 poses free (192 x 192), 4
    Gauss-Newton iterations, 20 % outliers; 8 distinct seeded scenes tiled.
    Per-kernel times from the library's launch events.  mode: the Schur mode
    (0, the default: the assembly as three TF32 products on the tensor cores;
    2: compensated FP32 on the CUDA cores)."""
    import torch
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import scenes as S
    distinct = [S.make_scene(S.STRESS_N64, 500 + s) for s in range(min(8, n_sessions))]
    batch = ba.PackedBatch([distinct[b % len(distinct)] for b in range(n_sessions)], "cuda")
    solver = ba.Solver(schur_tf32=mode)
    for _ in range(2):
        solver.solve_arrays(batch.dims, batch.probs, n_sessions, stream)
    torch.cuda.synchronize()
    statuses = batch.status.cpu().numpy()
    solver.set_timing(True)
    solver.timing()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        solver.solve_arrays(batch.dims, batch.probs, n_sessions, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = solver.timing(cap=64 * steps + 64)
    solver.set_timing(False)
    solver.close()
    kinds = {}
    for k, v in launches:
        kinds.setdefault(int(k), []).append(v)
    names = {0: "plan", 1: "linearize", 2: "reduced_solve", 3: "schur_assembly", 4: "final_backsub"}
    kern = {names[k] + "_ms": float(np.mean(v)) for k, v in kinds.items() if k in names}
    kern.update({names[k] + "_launches_per_step": len(v) // steps for k, v in kinds.items() if k in names})
    sc = distinct[0]
    bytes_lin = n_sessions * (24.0 * sc.n_edges + 20.0 * sc.n_patches)
    t_lin = float(np.mean(kinds.get(1, [0.0])))   # the launches that linearise (kind 4 back-substitutes)
    kern["linearize_linearising_ms"] = t_lin
    gbs = bytes_lin / (t_lin / 1e3) / 1e9 if t_lin > 0 else None
    return {"workload": "64 frames x 256 patches (16,384), radius 24 (649,216 edges), last 32 poses free "
                        "(192 x 192 reduced system), 4 GN iterations, 20 % outliers, weights U[0,1]",
            "sessions": n_sessions, "solves_per_s": n_sessions / (ms / 1e3), "ms_per_step": ms,
            "schur_assembly": ("compensated FP32 on the CUDA cores" if mode == 2 else
                               "three TF32 products on the tensor cores (tcgen05, TMEM), FP32 accumulation "
                               "over at most 2048 patches, ranges added in FP64"),
            "statuses_nonzero": int((statuses != 0).sum()), "kernels": kern,
            "linearize_hbm": {"algorithmic_bytes_per_launch": bytes_lin, "achieved_gbs": gbs,
                              "peak_gbs": hbm_peak, "frac": (gbs / hbm_peak) if gbs else None},
            "parity": "tests/test_gpu_large.py: one instance against the dense FP64 oracle"}


def grad_bench(n_problems=16, steps=20, warmup=3, parity=True):
    """The differentiation workload: n_problems eight-frame problems (64
    patches per frame, every frame connected, 2 fixed poses, 2 iterations).
    A step = forward solve from the initial state, the pose supervision loss
    of Sec. 3.4 (Eq. 7) and its pose gradient on the device, and the backward
    to the targets and weights -- all through the C ABI, CUDA events around
    each part.  Parity: problem 0's target/weight gradients vs autograd of the
    FP64 twin with the same loss."""
    import torch
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import scenes as S
    scenes = [S.make_scene(S.PLAIN_N8, 300 + b) for b in range(n_problems)]
    start = [ba.problem_from_scene(sc) for sc in scenes]
    work = [ba.problem_from_scene(sc) for sc in scenes]
    gt = [torch.tensor(sc.poses_gt, dtype=torch.float32, device="cuda") for sc in scenes]
    zero_d = [torch.zeros_like(p.patches[:, 2]) for p in start]
    solver = ba.Solver()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_fwd, t_loss, t_bwd = [], [], []
    out = None
    for it in range(warmup + steps):
        for w, s0 in zip(work, start):
            w.poses.copy_(s0.poses)
            w.patches.copy_(s0.patches)
        ev[0].record()
        solver.solve(work)
        ev[1].record()
        loss, gp = ba.pose_loss([w.poses for w in work], gt)
        ev[2].record()
        gts, gws = solver.backward(start, gp, zero_d)
        ev[3].record()
        torch.cuda.synchronize()
        if it >= warmup:
            t_fwd.append(ev[0].elapsed_time(ev[1]))
            t_loss.append(ev[1].elapsed_time(ev[2]))
            t_bwd.append(ev[2].elapsed_time(ev[3]))
        out = (gts[0].cpu().numpy(), gws[0].cpu().numpy())
    solver.close()
    step = float(np.median(np.array(t_fwd) + np.array(t_loss) + np.array(t_bwd)))
    res = {"workload": f"{n_problems} problems of 8 frames x 64 patches (512), all frames connected (4096 edges), "
                       "t0 = 2, 2 GN iterations; loss = pose supervision of Eq. 7 (ordered frame pairs)",
           "ms_per_step": step, "problems_per_s": n_problems / step * 1e3,
           "forward_ms": float(np.median(t_fwd)), "pose_loss_ms": float(np.median(t_loss)),
           "backward_ms": float(np.median(t_bwd)), "steps": steps}
    if parity:
        from oracle import pose_loss as PL
        from oracle import unrolled_grad as ug
        sc = scenes[0]
        target = torch.tensor(np.asarray(sc.target, np.float64), requires_grad=True)
        weight = torch.tensor(np.asarray(sc.weight, np.float64), requires_grad=True)
        R, t, _ = ug.unrolled(sc, target, weight)
        rt, rw = torch.autograd.grad(PL.loss_torch(R, t, sc.poses_gt), [target, weight])
        res["parity"] = {"problem": 0, "tolerance": 1e-3,
                         "dL_dtarget_rel_err": float(np.linalg.norm(out[0] - rt.numpy()) / np.linalg.norm(rt.numpy())),
                         "dL_dweight_rel_err": float(np.linalg.norm(out[1] - rw.numpy()) / np.linalg.norm(rw.numpy()))}
    return res


def window_bench(n_windows=256, steps=10, warmup=3, seed=0):
    """Sliding windows kept on the device (Sec. 3.3): n_windows windows of 22
    frames (96 patches per new frame, radius 13, the last 10 poses free).  A
    step appends one frame to every window (constant-velocity pose, median
    depth, the oldest frame dropped, the edges regenerated; one batched call,
    two launches per 128 windows) and then runs one batched 2-iteration solve over all windows with
    the regenerated targets revised by N(0, 0.5 px^2) noise."""
    import torch
    from paper_2208_04726_b300 import ba
    rng = np.random.default_rng(seed)
    intr = (320.0, 320.0, 320.0, 240.0)
    wins = [ba.Window(22, 96, 13, 10, intr) for _ in range(n_windows)]
    xy = [torch.tensor(rng.uniform([16, 16], [624, 464], (96, 2)).astype(np.float32), device="cuda")
          for _ in range(8)]
    for f in range(22):                               # fill the windows
        ba.append_windows(wins, [xy[f % 8]] * n_windows)
    solver = ba.Solver()
    solver.reserve(22, 2112, 39552, 2, n_windows)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_app, t_solve = [], []
    statuses = 0
    for it in range(warmup + steps):
        ev[0].record()
        ba.append_windows(wins, [xy[it % 8]] * n_windows)
        ev[1].record()
        probs = [w.problem() for w in wins]           # views of the windows' arrays
        for p in probs:                               # the update operator's revision, simulated
            p.target.add_(torch.randn_like(p.target), alpha=0.7071)
        n, dims, cp = solver._arrays(probs)
        ev[2].record()
        solver.solve_arrays(dims, cp, n)
        ev[3].record()
        torch.cuda.synchronize()
        if it >= warmup:
            t_app.append(ev[0].elapsed_time(ev[1]))
            t_solve.append(ev[2].elapsed_time(ev[3]))
            statuses += sum(int(p.status.item()) != 0 for p in probs)
    solver.close()
    for w in wins:
        w.close()
    a, sv = float(np.median(t_app)), float(np.median(t_solve))
    return {"workload": f"{n_windows} windows of 22 frames x 96 patches per frame, radius 13, last 10 poses free; "
                        "per step one appended frame per window, then one batched 2-iteration solve",
            "append_all_ms": a, "append_us_per_window": a * 1e3 / n_windows,
            "solve_ms": sv, "frames_per_s": n_windows / (a + sv) * 1e3, "statuses_nonzero": statuses,
            "note": "device time of the batched append call and of the batched solve (CUDA events); the target "
                    "revision and the host marshalling between them are not counted"}


def vo_mix_bench(n_default=128, n_fast=128, steps=10, warmup=3, seed=1):
    """The paper's two configurations as one serving mix on device-maintained
    windows (Sec. 4: Default 96 patches/frame and 10 free poses, Fast 48 and 7;
    radius 13, 22-frame buffers).  Initialisation (Sec. 3.3): every session
    accumulates 8 frames and runs 12 update iterations, each a 2-iteration
    solve on revised targets, batched over all sessions.  Steady state: per
    step one appended frame per session and one mixed batched solve.  Device
    time by CUDA events (target revision and host marshalling not counted)."""
    import torch
    from paper_2208_04726_b300 import ba
    rng = np.random.default_rng(seed)
    intr = (320.0, 320.0, 320.0, 240.0)
    kinds = [(96, 10)] * n_default + [(48, 7)] * n_fast
    wins = [ba.Window(22, m, 13, f, intr) for m, f in kinds]
    xy = {m: [torch.tensor(rng.uniform([16, 16], [624, 464], (m, 2)).astype(np.float32), device="cuda")
              for _ in range(8)] for m in (96, 48)}
    solver = ba.Solver()
    solver.reserve(22, 2112, 39552, 2, len(wins))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def solve_all():
        probs = [w.problem() for w in wins]
        for p in probs:
            p.target.add_(torch.randn_like(p.target), alpha=0.7071)
        n, dims, cp = solver._arrays(probs)
        ev[2].record()
        solver.solve_arrays(dims, cp, n)
        ev[3].record()
        torch.cuda.synchronize()
        return ev[2].elapsed_time(ev[3]), sum(int(p.status.item()) != 0 for p in probs)

    # initialisation: 8 frames, then 12 update iterations
    t_init, bad = 0.0, 0
    for f in range(8):
        ev[0].record()
        ba.append_windows(wins, [xy[m][f] for m, _ in kinds])
        ev[1].record()
        torch.cuda.synchronize()
        t_init += ev[0].elapsed_time(ev[1])
    for _ in range(12):
        t, b = solve_all()
        t_init += t
        bad += b
    # steady state
    t_app, t_solve = [], []
    for it in range(warmup + steps):
        ev[0].record()
        ba.append_windows(wins, [xy[m][it % 8] for m, _ in kinds])
        ev[1].record()
        torch.cuda.synchronize()
        t, b = solve_all()
        if it >= warmup:
            t_app.append(ev[0].elapsed_time(ev[1]))
            t_solve.append(t)
            bad += b
    solver.close()
    for w in wins:
        w.close()
    a, sv = float(np.median(t_app)), float(np.median(t_solve))
    return {"workload": f"{n_default} Default (96 patches/frame, 10 free poses) + {n_fast} Fast (48, 7) sessions, "
                       "radius 13, 22-frame windows, 2 GN iterations per solve",
            "init_ms": t_init, "init_note": "8 appended frames, then 12 batched 2-iteration solves, all sessions",
            "append_all_ms": a, "solve_ms": sv, "frames_per_s": len(wins) / (a + sv) * 1e3,
            "statuses_nonzero": bad}


def corr_bench(steps=20, warmup=3, seed=7, hbm_peak=6400.0, parity=True):
    """Correlation features (Sec. 3.2, Eq. 4) of the sliding-window graph: 22
    frames of 120 x 160 x 128 bfloat16 matching features (a quarter of a 640 x
    480 image), level 1 pooled by 4, 2112 patches of 3 x 3 pixels, radius 13
    (39,552 edges), 7 x 7 grids at both levels.  One call = every edge.  Device
    time by CUDA events; flops as executed by the tensor cores (footprint x 16
    patch-pixel GEMMs) and as defined (49 bilinear samples per pixel and
    level); bytes = the inputs read once and the outputs written."""
    import torch
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import corr_inputs as CI
    inp = CI.make_corr_inputs(22, 96, 13, 120, 160, 4, seed)
    bf = lambda a: torch.from_numpy(a.view(np.int16)).view(torch.bfloat16).cuda()
    args = (bf(inp.fmap0), bf(inp.fmap1), bf(inp.gpatch), torch.from_numpy(inp.kk).cuda(),
            torch.from_numpy(inp.jj).cuda(), torch.from_numpy(inp.coords).cuda())
    out = torch.empty((inp.n_edges, 2, 9, 7, 7), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        ba.correlation(*args, inp.scale, out=out, status=st)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        ba.correlation(*args, inp.scale, out=out, status=st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    E = inp.n_edges
    # footprint chunks per edge and level, from the coordinates (as the kernel forms them)
    fl_exec = 0.0
    for s_ in (1.0, float(inp.scale)):
        xy = np.floor(inp.coords.astype(np.float32) / np.float32(s_))
        w = xy[:, :, 0].max(1) - xy[:, :, 0].min(1) + 8
        h = xy[:, :, 1].max(1) - xy[:, :, 1].min(1) + 8
        fl_exec += float(np.sum(np.ceil(w * h / 128.0))) * 128 * 16 * 128 * 2
    fl_def = E * 2 * 9 * 49 * (128 * 2 + 4 * 128 * 2)
    byts = (inp.fmap0.nbytes + inp.fmap1.nbytes + inp.gpatch.nbytes + inp.kk.nbytes + inp.jj.nbytes
            + inp.coords.nbytes + out.numel() * 4)
    res = {"workload": "22 frames x 120 x 160 x 128 bf16 features (level 1 pooled by 4), 2112 patches of 3 x 3, "
                       "radius 13 (39,552 edges), 7 x 7 grids at 2 levels",
           "ms_per_call": ms, "edges_per_s": E / ms * 1e3,
           "tensor_tflops_executed": fl_exec / ms / 1e9, "tflops_by_definition": fl_def / ms / 1e9,
           "hbm": {"bytes_per_call": byts, "achieved_gbs": byts / ms / 1e6, "peak_gbs": hbm_peak,
                   "frac": byts / ms / 1e6 / hbm_peak},
           "status": int(st.item())}
    if parity:
        from oracle import corr as C
        edges = np.random.default_rng(0).choice(E, 32, replace=False)
        ref = C.correlation(inp, edges)
        got = out.cpu().numpy()[edges].astype(np.float64)
        res["parity"] = {"edges_checked": 32, "max_abs_err": float(np.abs(got - ref).max()),
                         "rel_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                         "tolerance": "1e-3 abs, 1e-5 rel"}
    return res


def traffic_from_profiles(kernel_source_sha):
    """DRAM bytes per launch per problem from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "linearize_window_n22.md")
    if not os.path.exists(path):
        return None
    sha, val = None, None
    for line in open(path):
        if line.startswith("kernel_source_sha1:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch_per_problem:"):
            val = float(line.split(":", 1)[1].strip())
    return val if (sha == kernel_source_sha and val is not None) else None


# the sources the linearise kernel and its launch are built from
KERNEL_SOURCES = ("ba_common.cuh", "dpvo_ba.cu", "kernels.cuh", "se3.cuh", "tc.cuh")


def kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2208_04726_b300", "csrc", f), "rb").read())
    return h.hexdigest()


# --------------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2208_04726_b300 import scenes as S
    from oracle import dense_gn as dg
    scenes = [S.make_scene(S.WINDOW_N22, 1000 + s) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        dg.solve_scene(scenes[s])
    t = time.perf_counter()
    for s in range(args.steps):
        dg.solve_scene(scenes[args.warmup + s])
    el = time.perf_counter() - t
    value = args.steps / el
    cores = oracle_threads()
    sample = "one sliding-window problem per step (dense FP64 oracle, 2 GN iterations)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------- serving

def serving_bench(n_sessions=256, distinct=32, rate=2000.0, duration=2.0, saturate=1.0, seed=0):
    """Poisson open loop (rate requests/s over n_sessions) and a saturated
    closed loop, for continuous batching and for one launch per solve.
    Latency is the library's (submit to completion on the device)."""
    import time as _t
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import scenes as S
    import torch
    mix = S.make_serving_mix(distinct, base_seed=seed)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.copy_(torch.from_numpy(np.ascontiguousarray(a, np.float32)))
        return t

    # each request's targets and weights sit in page-locked memory (read in place)
    reqs = [[(pinned(f.target), pinned(f.weight)) for f in (S.refresh_factors(sc, 10_000 + 10 * i + r)
                                                            for r in range(3))] for i, sc in enumerate(mix)]
    sess_of = [b % distinct for b in range(n_sessions)]
    max_n = max(sc.n_frames for sc in mix)
    max_p = max(sc.n_patches for sc in mix)
    max_e = max(sc.n_edges for sc in mix)
    out = {"sessions": n_sessions, "distinct_shapes": distinct, "poisson_rate": rate,
           "workload": "N~U{8..32} frames, {48,64,96} patches/frame, radius U{8..13}, last min(10, N-2) poses free, "
                       "2 GN iterations, fresh targets and weights per request (page-locked, read in place)"}
    for mode, (mb, mif) in (("batched", (n_sessions, 2)), ("plain", (1, 1))):
        srv = ba.Solver()
        srv.serve_start(max_n, max_p, max_e, 2, max_batch=mb, max_in_flight=mif)
        sids = [srv.session_open(mix[sess_of[b]]) for b in range(n_sessions)]

        def request(b, k):
            t, w = reqs[sess_of[b]][k % 3]
            return srv.submit(sids[b], t, w)

        for b in range(n_sessions):                     # warm-up: one request per session
            srv.wait(request(b, 0), 60000)
        rng = np.random.default_rng(1)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 10))
        arrivals = arrivals[arrivals < duration]
        who = rng.integers(0, n_sessions, size=arrivals.shape[0])
        busy = {}                                       # session -> ticket
        queued = {b: [] for b in range(n_sessions)}     # arrivals waiting for their session
        lat, k, done = [], 0, 0
        t0 = _t.perf_counter()
        while done < arrivals.shape[0]:
            now = _t.perf_counter() - t0
            while k < arrivals.shape[0] and arrivals[k] <= now:
                b = int(who[k])
                if b in busy:
                    queued[b].append(k)
                else:
                    busy[b] = request(b, k)
                k += 1
            for b, tk in list(busy.items()):
                ok, st, ms = srv.poll(tk)
                if ok:
                    lat.append(ms)
                    done += 1
                    del busy[b]
                    if queued[b]:
                        busy[b] = request(b, queued[b].pop(0))
        elapsed = _t.perf_counter() - t0
        res = {"latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
               "completed": done, "solves_per_s": done / elapsed}
        # saturated closed loop: every session resubmits as soon as its request finishes
        busy = {b: request(b, 1) for b in range(n_sessions)}
        cnt = 0
        t0 = _t.perf_counter()
        while _t.perf_counter() - t0 < saturate:
            for b, tk in list(busy.items()):
                ok, st, ms = srv.poll(tk)
                if ok:
                    cnt += 1
                    busy[b] = request(b, cnt)
        el = _t.perf_counter() - t0
        for tk in busy.values():
            srv.wait(tk, 60000)
        res["saturated_solves_per_s"] = cnt / el
        out[mode] = res
        srv.serve_stop()
        srv.close()
    out["full_batch_linearize_hbm"] = serving_batch_hbm([mix[sess_of[b]] for b in range(n_sessions)])
    return out


def serving_batch_hbm(scenes):
    """The linearise launch on one full batch of the serving mix (every
    session's problem in one batched solve): its device time from the library's
    launch events and its HBM fraction by the algorithmic bytes (24 per edge,
    20 per patch), for comparison with the window batch's roofline."""
    import torch
    from paper_2208_04726_b300 import ba
    batch = ba.PackedBatch(scenes, "cuda")
    solver = ba.Solver()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        batch.reset()
        solver.solve_arrays(batch.dims, batch.probs, len(scenes), stream)
    solver.set_timing(True)
    solver.timing()
    for _ in range(10):
        batch.reset()
        solver.solve_arrays(batch.dims, batch.probs, len(scenes), stream)
    torch.cuda.synchronize()
    lin = [ms for k, ms in solver.timing(cap=4096) if k == 1]
    solver.set_timing(False)
    solver.close()
    t = float(np.median(lin))
    bytes_ = float(sum(24.0 * sc.n_edges + 20.0 * sc.n_patches for sc in scenes))
    peak, src = load_peaks()
    gbs = bytes_ / (t / 1e3) / 1e9
    return {"problems": len(scenes), "linearize_ms": t, "algorithmic_bytes": bytes_, "achieved_gbs": gbs,
            "peak_gbs": peak, "frac": gbs / peak, "peak_source": src}


def serving_slid_bench(n_default=128, n_fast=128, rate=2000.0, duration=2.0, saturate=1.0, seed=2):
    """The paper's Default (96 patches/frame, 10 free poses) and Fast (48, 7)
    configurations (Sec. 4) as served sliding-window sessions (radius 13,
    22-frame windows, 2 GN iterations): every request appends a frame and
    solves the window (Sec. 3.3).  The windows are first filled (22 frames
    each); then a Poisson open loop (rate requests/s over all sessions) and a
    saturated closed loop, for continuous batching and for one launch per
    solve.  Each request's patch centres, edge revisions N(0, 0.5 px^2) and
    weights U[0, 1] sit in page-locked memory and are read in place.  Latency
    is the library's (submit to completion on the device)."""
    import time as _t
    import torch
    from paper_2208_04726_b300 import ba
    rng = np.random.default_rng(seed)
    intr = (320.0, 320.0, 320.0, 240.0)
    kinds = [(96, 10)] * n_default + [(48, 7)] * n_fast
    n = len(kinds)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.copy_(torch.from_numpy(a))
        return t

    xy = {m: [pinned(rng.uniform([16, 16], [624, 464], (m, 2)).astype(np.float32)) for _ in range(4)]
          for m in (96, 48)}
    out = {"sessions": n, "poisson_rate": rate,
           "workload": f"{n_default} Default (96 patches/frame, 10 free poses) + {n_fast} Fast (48, 7) sliding "
                       "windows, radius 13, 22 frames, 2 GN iterations; a request appends a frame and solves"}
    for mode, (mb, mif) in (("batched", (n, 2)), ("plain", (1, 1))):
        srv = ba.Solver()
        srv.serve_start(22, 22 * 96, 22 * 96 * 22, 2, max_batch=mb, max_in_flight=mif)   # window capacities
        sids = [srv.session_open_window(ba.WindowParams(22, m, 13, f, 2, *intr)) for m, f in kinds]
        for f in range(22):                              # fill the windows (no revisions)
            tks = [srv.submit_frame(sid, xy[m][f % 4]) for sid, (m, _) in zip(sids, kinds)]
            for tk in tks:
                srv.wait(tk, 60000)
        E = {m: srv.session_frame_edges(sids[kinds.index((m, f))], m) for m, f in set(kinds)}
        fac = {m: [(pinned(rng.normal(scale=np.sqrt(0.5), size=(E[m], 2)).astype(np.float32)),
                    pinned(rng.uniform(0.0, 1.0, size=(E[m], 2)).astype(np.float32))) for _ in range(3)]
               for m in E}

        def request(b, k):
            m = kinds[b][0]
            d, w = fac[m][k % 3]
            return srv.submit_frame(sids[b], xy[m][k % 4], d, w)

        rng2 = np.random.default_rng(1)
        arrivals = np.cumsum(rng2.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 10))
        arrivals = arrivals[arrivals < duration]
        who = rng2.integers(0, n, size=arrivals.shape[0])
        busy, queued = {}, {b: [] for b in range(n)}
        lat, k, done, bad = [], 0, 0, 0
        t0 = _t.perf_counter()
        while done < arrivals.shape[0]:
            now = _t.perf_counter() - t0
            while k < arrivals.shape[0] and arrivals[k] <= now:
                b = int(who[k])
                if b in busy:
                    queued[b].append(k)
                else:
                    busy[b] = request(b, k)
                k += 1
            for b, tk in list(busy.items()):
                ok, st, ms = srv.poll(tk)
                if ok:
                    lat.append(ms)
                    bad += int(st != 0)
                    done += 1
                    del busy[b]
                    if queued[b]:
                        busy[b] = request(b, queued[b].pop(0))
        elapsed = _t.perf_counter() - t0
        res = {"latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
               "completed": done, "solves_per_s": done / elapsed, "statuses_nonzero": bad}
        busy = {b: request(b, 1) for b in range(n)}
        cnt = 0
        t0 = _t.perf_counter()
        while _t.perf_counter() - t0 < saturate:
            for b, tk in list(busy.items()):
                ok, st, ms = srv.poll(tk)
                if ok:
                    cnt += 1
                    busy[b] = request(b, cnt)
        el = _t.perf_counter() - t0
        for tk in busy.values():
            srv.wait(tk, 60000)
        res["saturated_solves_per_s"] = cnt / el
        out[mode] = res
        for sid in sids:
            srv.session_close(sid)
        srv.serve_stop()
        srv.close()
    return out


# --------------------------------------------------------------------- our arm

def parity_of(batch, scenes, refs):
    """Errors of sampled problems' whole-solve updates (final - initial state)
    against the FP64 oracle: relative 2-norm over the free poses / inverse
    depths, and per element (the largest error of one free pose's 7 stored
    entries, or of one inverse depth, over the largest reference entry)."""
    out = {"problems_checked": sorted(refs), "tolerance": 1e-4}
    ep, ed, mp, md, ap, ad = [], [], [], [], [], []
    for b, ref in refs.items():
        sc = scenes[b]
        poses = batch.view("poses", b).view(-1, 7).cpu().numpy().astype(np.float64)
        poses[:, 3:] *= np.sign((poses[:, 3:] * ref["poses"][:, 3:]).sum(1))[:, None]
        p0 = sc.poses.astype(np.float64).copy()
        p0[:, 3:] *= np.sign((p0[:, 3:] * ref["poses"][:, 3:]).sum(1))[:, None]
        t0 = sc.t0
        du, dr = poses[t0:] - p0[t0:], ref["poses"][t0:] - p0[t0:]
        ep.append(float(np.linalg.norm(du - dr) / np.linalg.norm(dr)))
        mp.append(float(np.linalg.norm(du - dr, axis=1).max() / np.linalg.norm(dr, axis=1).max()))
        ap.append(float(np.abs(du - dr).max()))
        d = batch.view("patches", b).view(-1, 3)[:, 2].cpu().numpy().astype(np.float64)
        d0 = sc.patches[:, 2].astype(np.float64)
        gu, gr = d - d0, ref["depths"] - d0
        ed.append(float(np.linalg.norm(gu - gr) / np.linalg.norm(gr)))
        md.append(float(np.abs(gu - gr).max() / np.abs(gr).max()))
        ad.append(float(np.abs(gu - gr).max()))
    out.update({"pose_update_rel_err_max": max(ep), "depth_update_rel_err_max": max(ed),
                "pose_update_per_pose_err_max": max(mp), "depth_update_per_patch_err_max": max(md),
                "pose_update_max_abs": max(ap), "depth_update_max_abs": max(ad)})
    return out


def plain_n8_bench(stream, n=200, warmup=10, seed=20_000):
    """The 8-frame problem (8 frames x 64 patches, every patch connected to every
    frame: 4,096 edges, poses 0-1 fixed, 2 GN iterations) solved one per call,
    back to back: per-solve latency from CUDA events around each call on the
    launching stream, and the split over the kernels of one call."""
    import torch
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import scenes as S
    scenes = [S.make_scene(S.PLAIN_N8, seed + s) for s in range(8)]
    batch = ba.PackedBatch(scenes, "cuda")
    solver = ba.Solver()
    solver.reserve(8, 512, 4096, 2, 1)
    subsets = [batch.subset(b % len(scenes)) for b in range(n)]
    for d_, p_ in subsets[:warmup]:
        batch.reset()
        solver.solve_arrays(d_, p_, 1, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for (a, b_), (d_, p_) in zip(ev, subsets):
        a.record(stream)
        solver.solve_arrays(d_, p_, 1, stream)
        b_.record(stream)
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b_) for a, b_ in ev])
    split = kernel_split(solver, subsets[:20], stream)
    solver.close()
    return {"workload": "8 frames x 64 patches (512), all frames connected (4,096 edges), poses 0-1 fixed, "
                        "2 GN iterations; one problem per call",
            "solves": n, "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)), **split}


def kernel_split(solver, subsets, stream):
    """Median device time of each kernel kind over one-problem solves of
    `subsets`, each launch bracketed by CUDA events on `stream`."""
    import torch
    solver.set_timing(True)
    solver.timing()
    for d_, p_ in subsets:
        solver.solve_arrays(d_, p_, 1, stream)
    torch.cuda.synchronize()
    launches = solver.timing(cap=64 * len(subsets))
    solver.set_timing(False)
    names = {0: "plan", 1: "linearize", 2: "reduced_solve", 3: "schur_assembly", 4: "final_backsub"}
    kinds = {}
    for k, v in launches:
        kinds.setdefault(names.get(int(k), str(k)), []).append(v)
    return {"kernel_ms_per_launch": {k: float(np.median(v)) for k, v in kinds.items()},
            "kernel_launches_per_solve": {k: len(v) // len(subsets) for k, v in kinds.items()}}


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist
    from paper_2208_04726_b300 import ba
    from paper_2208_04726_b300 import scenes as S

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # ---- workload: distinct seeded scenes tiled to the batch size
    base = 10_000 * (rank + 1)
    n_batch = args.batch if args.batch > 0 else 2 * torch.cuda.get_device_properties(dev).multi_processor_count
    distinct = [S.make_scene(S.WINDOW_N22, base + s) for s in range(min(args.distinct, n_batch))]
    scenes = [distinct[b % len(distinct)] for b in range(n_batch)]
    B = len(scenes)
    batch = ba.PackedBatch(scenes, "cuda")
    solver = ba.Solver()
    solver.reserve(22, 2112, 39552, 2, B)

    # ---- first solve from the initial state: full-size parity on sampled problems
    solver.solve_arrays(batch.dims, batch.probs, B, stream)
    torch.cuda.synchronize()
    statuses = batch.status.cpu().numpy()
    parity = None
    cpu_baseline = None
    refs = {}
    if rank == 0 and args.parity_samples > 0:
        from oracle import dense_gn as dg
        idx = sorted(set([0, B - 1] + list(range(1, B - 1, max(1, B // max(1, args.parity_samples))))))[
            :args.parity_samples]
        t_or = 0.0
        refs = {}
        for b in idx:
            t = time.perf_counter()
            refs[b] = dg.solve_scene(scenes[b])
            t_or += time.perf_counter() - t
        parity = parity_of(batch, scenes, refs)
        parity["statuses_nonzero"] = int((statuses != 0).sum())
        cpu_baseline = {"value": len(idx) / t_or, "unit": "solves/s", "cores": oracle_threads(), "kind": "oracle",
                        "sample": f"{len(idx)} sliding-window problems of this batch, dense FP64 oracle, "
                                  f"2 GN iterations each ({t_or:.1f} s)"}

    # ---- warm-up
    for _ in range(max(3, args.warmup)):
        batch.reset()
        solver.solve_arrays(batch.dims, batch.probs, B, stream)
    torch.cuda.synchronize()

    # ---- timed region: K batched solves, per-launch events on the launching stream
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    solver.set_timing(True)
    solver.timing()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            batch.reset()                       # every step solves from the initial state
            solver.solve_arrays(batch.dims, batch.probs, B, stream)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = solver.timing(cap=16 * args.steps + 64)
    if parity is not None:                      # the last timed step, checked like the first solve
        post = parity_of(batch, scenes, refs)
        parity["after_timed_steps"] = {k: post[k] for k in post if k != "problems_checked"}
    solver.set_timing(False)
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    # one timing record per kernel launch: the launches of a step, and the
    # kernels' device times by kind (0 plan, 1 linearise/Schur, 2 reduced
    # solve, 4 last back-substitution)
    n_launch_per_solve = len(launches) // args.steps
    value = world * B * args.steps / (elapsed_ms / 1e3)
    by_kind = {}
    for k, ms in launches:
        by_kind.setdefault(k, []).append(ms)
    kern = {"plan_ms": float(np.mean(by_kind[0])), "linearize_schur_ms": float(np.mean(by_kind[1])),
            "backsub_final_ms": float(np.mean(by_kind[4])),
            "reduce_cholesky_ms": float(np.mean(by_kind[2])),
            "launches_per_step": n_launch_per_solve}
    step_ms = elapsed_ms / args.steps
    kern["share_linearize_schur"] = 2 * kern["linearize_schur_ms"] / step_ms
    kern["share_reduce_cholesky"] = 2 * kern["reduce_cholesky_ms"] / step_ms

    hbm_peak, hbm_src = load_peaks()
    flops_p, bytes_p = zip(*[algorithmic_work(sc) for sc in distinct])
    flops = float(np.mean(flops_p)) * B
    bytes_ = float(np.mean(bytes_p)) * B
    t_lin = kern["linearize_schur_ms"] / 1e3
    traffic_pp = traffic_from_profiles(kernel_sha())
    # The linearising pass's algorithmic FP32 work (edges and the Schur
    # products) and bytes (24 per edge, 20 per patch): its roofline is the
    # larger of the two times -- the FP32-ALU one on this workload; the HBM
    # fraction of the same launch is reported beside it.
    alu_time, hbm_time = flops / (PEAK_ALU_TFLOPS * 1e12), bytes_ / (hbm_peak * 1e9)
    if alu_time >= hbm_time:
        achieved = flops / t_lin / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": PEAK_ALU_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / PEAK_ALU_TFLOPS,
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 x 2032 MHz"}
    else:
        achieved = bytes_ / t_lin / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": hbm_src}
    roof["kernel"] = "linearize_kernel (back-substitution + linearisation + Schur, one launch per GN iteration)"
    roof["traffic"] = traffic_pp * B if traffic_pp is not None else None
    roof["algorithmic_per_launch"] = {"flops": flops, "bytes": bytes_}
    roof["launch_ms"] = kern["linearize_schur_ms"]
    roof["hbm_gbs_achieved"] = bytes_ / t_lin / 1e9
    roof["hbm_frac_of_measured"] = roof["hbm_gbs_achieved"] / hbm_peak

    # batched per-solve latency: every solve of a step completes with the step
    step_times = []
    for s in range(len(launches) // n_launch_per_solve):
        step_times.append(sum(x[1] for x in launches[s * n_launch_per_solve:(s + 1) * n_launch_per_solve]))

    # ---- plain form: one problem per call, back to back
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.plain)]
    subsets = [batch.subset(b % B) for b in range(args.plain)]
    for d_, p_ in subsets[:5]:
        solver.solve_arrays(d_, p_, 1, stream)
    torch.cuda.synchronize()
    tp0 = torch.cuda.Event(enable_timing=True); tp1 = torch.cuda.Event(enable_timing=True)
    tp0.record(stream)
    for (a, b_), (d_, p_) in zip(ev, subsets):
        a.record(stream)
        solver.solve_arrays(d_, p_, 1, stream)
        b_.record(stream)
    tp1.record(stream)
    torch.cuda.synchronize()
    plain_lat = np.array([a.elapsed_time(b_) for a, b_ in ev])
    plain_value = args.plain / (tp0.elapsed_time(tp1) / 1e3) if args.plain > 0 else None
    plain_split = kernel_split(solver, subsets[:20], stream) if args.plain > 0 else {}

    # ---- end to end through the host-buffer entry point
    hbatch = ba.PackedBatch(scenes, "pinned")
    h2d = hbatch.bytes_of([k for k, _ in ba.PackedBatch.KINDS])
    d2h = hbatch.bytes_of(["poses", "patches"]) + 4 * B
    hstream = torch.cuda.current_stream()
    lib = solver.lib
    for _ in range(2):
        rc = lib.dpvo_ba_solve_host(solver.h, hbatch.dims, hbatch.probs, B, hstream.cuda_stream)
        assert rc == 0, rc
    if world > 1:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        rc = lib.dpvo_ba_solve_host(solver.h, hbatch.dims, hbatch.probs, B, hstream.cuda_stream)
        assert rc == 0, rc
    e2e_s = time.perf_counter() - t
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e_value = world * B * args.e2e_steps / e2e_s

    # ---- opt-in tensor-core Schur mode on the same batch: throughput, parity
    tf32 = None
    if args.tf32:
        tsolver = ba.Solver(schur_tf32=True)
        tsolver.reserve(22, 2112, 39552, 2, B)
        for _ in range(3):
            batch.reset()
            tsolver.solve_arrays(batch.dims, batch.probs, B, stream)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            batch.reset()
            tsolver.solve_arrays(batch.dims, batch.probs, B, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        tf32 = {"solves_per_s": world * B * args.steps / (a0.elapsed_time(a1) / 1e3),
                "note": "sum_k E_k C_k^-1 E_k^T as three TF32 products on the tensor cores (tcgen05, TMEM)"}
        if refs:
            sub = ba.PackedBatch([scenes[b] for b in refs], "cuda")
            tsolver.solve_arrays(sub.dims, sub.probs, len(refs), stream)
            torch.cuda.synchronize()
            par = parity_of(sub, [scenes[b] for b in refs], {i: refs[b] for i, b in enumerate(refs)})
            tf32.update({k: par[k] for k in par if k != "problems_checked"})
        tsolver.close()

    plain_n8 = plain_n8_bench(stream) if (rank == 0 and args.plain > 0) else None
    serving = serving_bench() if (rank == 0 and args.serving) else None
    if serving is not None:
        serving["slid_default_fast_mix"] = serving_slid_bench()
    stress = stress_bench(args.stress, 5, stream, load_peaks()[0]) if (rank == 0 and args.stress > 0) else None
    if stress is not None and args.tf32:
        st = stress_bench(args.stress, 5, stream, load_peaks()[0], mode=2)
        stress["fp32_assembly"] = {k: st[k] for k in ("solves_per_s", "ms_per_step", "statuses_nonzero", "kernels",
                                                      "schur_assembly")}
        stress["fp32_assembly"]["note"] = ("Schur mode 2: S - E C^-1 E^T assembled in compensated FP32 on the "
                                           "CUDA cores; parity: tests/test_gpu_large.py, both assemblies")
    grad = grad_bench(args.grad, parity=args.parity_samples > 0) if (rank == 0 and args.grad > 0) else None
    window = window_bench(args.window) if (rank == 0 and args.window > 0) else None
    vo_mix = vo_mix_bench() if (rank == 0 and args.vo_mix) else None
    corr = corr_bench(hbm_peak=load_peaks()[0], parity=args.parity_samples > 0) if (rank == 0 and args.corr) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f32 (edges, reductions, Schur sums compensated, partials f64); reduced solve: f32 "
                      "LDL^T factor (approximate pivot reciprocals) + f64 residuals and iterative refinement "
                      "(f64 elimination when an f32 pivot fails or refinement stalls); retraction: f32, "
                      "as an increment added once to the stored pose"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_step": B, "distinct_scenes": len(distinct),
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush)",
                       "input_bytes_per_step": int(batch.bytes_of([k for k, _ in ba.PackedBatch.KINDS])),
                       "state": ("every step solves from the initial state: poses and patches restored by a "
                                 "device-to-device copy inside the timed region")},
            "batched": {"solves_per_s": value, "latency_ms_p50": float(np.percentile(step_times, 50)),
                        "latency_ms_p99": float(np.percentile(step_times, 99))},
            "plain": ({"solves_per_s": plain_value, "latency_ms_p50": float(np.percentile(plain_lat, 50)),
                       "latency_ms_p99": float(np.percentile(plain_lat, 99)), "solves": args.plain,
                       **plain_split}
                      if args.plain > 0 else None),
            "plain_n8": plain_n8,
            "kernels": kern,
            "roofline": roof,
            "parity": parity,
            "cpu_baseline": cpu_baseline,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": args.e2e_steps, "api": "dpvo_ba_solve_host (pinned host buffers)"},
            "serving": serving,
            "tf32_schur": tf32,
            "stress": stress,
            "grad": grad,
            "window": window,
            "vo_mix": vo_mix,
            "corr": corr,
            "gpu_launches": world * n_launch_per_solve * args.steps,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
