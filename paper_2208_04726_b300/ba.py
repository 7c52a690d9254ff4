"""Python binding of the C ABI in ``include/dpvo_ba.h`` (ctypes; argument
marshalling only -- every step of the solve runs in the CUDA library).

The library must be built (``paper_2208_04726_b300.build``); there is no
fallback: importing a missing or stale library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

# ---- C structs ---------------------------------------------------------------


class Dims(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("n_patches", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("t0", ctypes.c_int32), ("n_iters", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class Config(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_float), ("z_min", ctypes.c_float), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_sessions", ctypes.c_int32), ("schur_tf32", ctypes.c_int32),
                ("reduced_solve_f64", ctypes.c_int32)]


class Grads(ctypes.Structure):
    _fields_ = [("dL_dposes", ctypes.c_void_p), ("dL_ddepth", ctypes.c_void_p), ("dL_dtarget", ctypes.c_void_p),
                ("dL_dweight", ctypes.c_void_p)]


class PoseLossProblem(ctypes.Structure):
    _fields_ = [("poses", ctypes.c_void_p), ("gt_poses", ctypes.c_void_p), ("loss", ctypes.c_void_p),
                ("dL_dposes", ctypes.c_void_p), ("n_frames", ctypes.c_int32), ("scale", ctypes.c_float)]


class WindowParams(ctypes.Structure):
    _fields_ = [("max_frames", ctypes.c_int32), ("max_new_patches", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("free_poses", ctypes.c_int32), ("n_iters", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class CorrDims(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("n_patches", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32), ("level1_scale", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("poses", ctypes.c_void_p), ("patches", ctypes.c_void_p), ("anchor", ctypes.c_void_p),
                ("kk", ctypes.c_void_p), ("jj", ctypes.c_void_p), ("target", ctypes.c_void_p),
                ("weight", ctypes.c_void_p), ("status", ctypes.c_void_p)]


OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
STATUS_OK, STATUS_NOT_SPD, STATUS_BAD_INPUT, STATUS_NONFINITE, STATUS_TIMEOUT = 0, 1, 2, 4, 8
MAX_FRAMES, MAX_FREE, MAX_ITERS = 128, 32, 16

# Every symbol the header declares (checked by the CPU tests).
EXPORTS = ["dpvo_ba_create", "dpvo_ba_destroy", "dpvo_ba_reserve", "dpvo_ba_solve", "dpvo_ba_solve_host",
           "dpvo_ba_reduced_system", "dpvo_ba_iterate", "dpvo_ba_set_timing", "dpvo_ba_timing",
           "dpvo_ba_solve_noalloc", "dpvo_ba_backward", "dpvo_ba_serve_start",
           "dpvo_ba_serve_stop", "dpvo_ba_session_open", "dpvo_ba_session_close", "dpvo_ba_session_read",
           "dpvo_ba_submit", "dpvo_ba_poll", "dpvo_ba_wait", "dpvo_ba_strerror", "dpvo_ba_pose_loss",
           "dpvo_ba_window_create", "dpvo_ba_window_destroy", "dpvo_ba_window_append", "dpvo_ba_window_problem",
           "dpvo_ba_window_append_batch", "dpvo_ba_correlation", "dpvo_ba_selftest_bounded_wait",
           "dpvo_ba_session_open_window", "dpvo_ba_session_frame_edges", "dpvo_ba_session_dims",
           "dpvo_ba_submit_frame"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    lib.dpvo_ba_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.dpvo_ba_destroy.argtypes = [vp]
    lib.dpvo_ba_reserve.argtypes = [vp, ctypes.POINTER(Dims), i32]
    lib.dpvo_ba_solve.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem), i32, vp]
    lib.dpvo_ba_solve_host.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem), i32, vp]
    lib.dpvo_ba_reduced_system.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem), vp, vp, vp]
    lib.dpvo_ba_iterate.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.dpvo_ba_set_timing.argtypes = [vp, i32]
    lib.dpvo_ba_timing.argtypes = [vp, vp, vp, i32]
    lib.dpvo_ba_solve_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Dims), ctypes.POINTER(Problem), vp]
    lib.dpvo_ba_backward.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem), ctypes.POINTER(Grads), i32, vp]
    i64, u64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)
    lib.dpvo_ba_serve_start.argtypes = [vp, ctypes.POINTER(Dims), i32, i32]
    lib.dpvo_ba_serve_stop.argtypes = [vp]
    lib.dpvo_ba_session_open.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem), ctypes.POINTER(i64)]
    lib.dpvo_ba_session_close.argtypes = [vp, i64]
    lib.dpvo_ba_session_read.argtypes = [vp, i64, vp, vp]
    lib.dpvo_ba_submit.argtypes = [vp, i64, vp, vp, u64p]
    lib.dpvo_ba_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    lib.dpvo_ba_wait.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_double)]
    lib.dpvo_ba_pose_loss.argtypes = [ctypes.POINTER(PoseLossProblem), i32, vp]
    lib.dpvo_ba_window_create.argtypes = [ctypes.POINTER(WindowParams), ctypes.POINTER(vp)]
    lib.dpvo_ba_window_destroy.argtypes = [vp]
    lib.dpvo_ba_window_append.argtypes = [vp, vp, i32, vp]
    lib.dpvo_ba_window_problem.argtypes = [vp, ctypes.POINTER(Dims), ctypes.POINTER(Problem)]
    lib.dpvo_ba_correlation.argtypes = [ctypes.POINTER(CorrDims), vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.dpvo_ba_window_append_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32), i32, vp]
    lib.dpvo_ba_selftest_bounded_wait.argtypes = [vp, i32, i32, vp]
    lib.dpvo_ba_session_open_window.argtypes = [vp, ctypes.POINTER(WindowParams), ctypes.POINTER(i64)]
    lib.dpvo_ba_session_frame_edges.argtypes = [vp, i64, i32, ctypes.POINTER(ctypes.c_int32)]
    lib.dpvo_ba_session_dims.argtypes = [vp, i64, ctypes.POINTER(Dims)]
    lib.dpvo_ba_submit_frame.argtypes = [vp, i64, vp, i32, vp, vp, u64p]
    lib.dpvo_ba_strerror.argtypes = [i32]
    lib.dpvo_ba_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "dpvo_ba_strerror":
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def selftest_bounded_wait(arrive: bool, polls: int = 1000, stream=None) -> int:
    """The kernels' bounded mbarrier wait on a phase that completes only if
    `arrive`; returns the status it reports (STATUS_TIMEOUT when it gave up)."""
    import torch
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    _check(load().dpvo_ba_selftest_bounded_wait(st.data_ptr(), int(bool(arrive)), int(polls), _stream_ptr(stream)),
           "dpvo_ba_selftest_bounded_wait")
    return int(st.item())


class BAError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = load().dpvo_ba_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise BAError(code, what)


# ---- problems -----------------------------------------------------------------


@dataclass
class BAProblem:
    """Device tensors of one problem (layouts as in include/dpvo_ba.h)."""
    poses: torch.Tensor      # [N, 7] float32, updated in place
    patches: torch.Tensor    # [P, 3] float32, column 2 updated in place
    anchor: torch.Tensor     # [P] int32
    kk: torch.Tensor         # [E] int32
    jj: torch.Tensor         # [E] int32
    target: torch.Tensor     # [E, 2] float32
    weight: torch.Tensor     # [E, 2] float32
    intrinsics: Sequence[float]
    t0: int
    n_iters: int = 2
    status: Optional[torch.Tensor] = None   # [1] int32

    def dims(self) -> Dims:
        fx, fy, cx, cy = (float(v) for v in self.intrinsics)
        return Dims(self.poses.shape[0], self.patches.shape[0], self.kk.shape[0], int(self.t0),
                    int(self.n_iters), fx, fy, cx, cy)

    def cstruct(self) -> Problem:
        for name in ("poses", "patches", "anchor", "kk", "jj", "target", "weight"):
            t = getattr(self, name)
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        if self.status is None:
            self.status = torch.zeros(1, dtype=torch.int32, device=self.poses.device)
        return Problem(self.poses.data_ptr(), self.patches.data_ptr(), self.anchor.data_ptr(),
                       self.kk.data_ptr(), self.jj.data_ptr(), self.target.data_ptr(),
                       self.weight.data_ptr(), self.status.data_ptr())


def problem_from_scene(scene, device="cuda", n_iters=None) -> BAProblem:
    """Copy a ``scenes.Scene`` (float32 / int32 arrays) to the device."""
    f = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
    return BAProblem(
        poses=f(scene.poses, torch.float32), patches=f(scene.patches, torch.float32),
        anchor=f(scene.anchor, torch.int32), kk=f(scene.kk, torch.int32), jj=f(scene.jj, torch.int32),
        target=f(scene.target, torch.float32), weight=f(scene.weight, torch.float32),
        intrinsics=[float(v) for v in scene.intrinsics], t0=scene.t0,
        n_iters=scene.n_iters if n_iters is None else n_iters)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Solver:
    """A library handle (workspace + staging) on the current CUDA device."""

    def __init__(self, damping: float = 1e-4, z_min: float = 0.1, mem_budget_bytes: int = 0,
                 max_sessions: int = 0, schur_tf32=False, reduced_solve_f64: bool = False):
        """schur_tf32: the Schur mode of dpvo_ba_config (False / 0: the default,
        True / 1: tensor cores on the fused path too, 2: FP32 CUDA cores
        everywhere)."""
        self.lib = load()
        self.schur_mode = int(schur_tf32)
        if self.schur_mode not in (0, 1, 2):
            raise ValueError("schur_tf32 must be 0, 1 or 2")
        self.schur_tf32 = self.schur_mode == 1
        cfg = Config(damping, z_min, mem_budget_bytes, max_sessions, self.schur_mode, 1 if reduced_solve_f64 else 0)
        h = ctypes.c_void_p()
        _check(self.lib.dpvo_ba_create(ctypes.byref(cfg), ctypes.byref(h)), "dpvo_ba_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.dpvo_ba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, max_frames: int, max_patches: int, max_edges: int, max_iters: int, n_problems: int):
        d = Dims(max_frames, max_patches, max_edges, 0, max_iters, 1.0, 1.0, 0.0, 0.0)
        _check(self.lib.dpvo_ba_reserve(self.h, ctypes.byref(d), n_problems), "dpvo_ba_reserve")

    @staticmethod
    def _arrays(problems: List[BAProblem]):
        n = len(problems)
        dims = (Dims * n)(*[p.dims() for p in problems])
        probs = (Problem * n)(*[p.cstruct() for p in problems])
        return n, dims, probs

    def solve(self, problems: List[BAProblem], stream=None):
        """Batched solve on device tensors (asynchronous on ``stream``)."""
        n, dims, probs = self._arrays(problems)
        _check(self.lib.dpvo_ba_solve(self.h, dims, probs, n, _stream_ptr(stream)), "dpvo_ba_solve")

    def solve_arrays(self, dims, probs, n, stream=None):
        """Solve with prebuilt ctypes arrays (no per-call marshalling)."""
        _check(self.lib.dpvo_ba_solve(self.h, dims, probs, n, _stream_ptr(stream)), "dpvo_ba_solve")

    def solve_host(self, scenes_np: List[dict], stream=None):
        """Solve problems held in host numpy arrays (copied in and out by the library)."""
        n = len(scenes_np)
        dims = (Dims * n)()
        probs = (Problem * n)()
        keep = []
        for b, s in enumerate(scenes_np):
            fx, fy, cx, cy = (float(v) for v in s["intrinsics"])
            dims[b] = Dims(s["poses"].shape[0], s["patches"].shape[0], s["kk"].shape[0], int(s["t0"]),
                           int(s["n_iters"]), fx, fy, cx, cy)
            arrs = [s[k] for k in ("poses", "patches", "anchor", "kk", "jj", "target", "weight", "status")]
            for a in arrs:
                assert a.flags["C_CONTIGUOUS"]
            keep.append(arrs)
            probs[b] = Problem(*[a.ctypes.data for a in arrs])
        _check(self.lib.dpvo_ba_solve_host(self.h, dims, probs, n, _stream_ptr(stream)), "dpvo_ba_solve_host")

    def reduced_system(self, problem: BAProblem, stream=None):
        """(S, v') of one linearisation at the problem's current state, FP64 on the device."""
        n6 = 6 * (problem.poses.shape[0] - problem.t0)
        S = torch.empty((n6, n6), dtype=torch.float64, device=problem.poses.device)
        v = torch.empty((n6,), dtype=torch.float64, device=problem.poses.device)
        d = problem.dims()
        p = problem.cstruct()
        _check(self.lib.dpvo_ba_reduced_system(self.h, ctypes.byref(d), ctypes.byref(p), S.data_ptr(),
                                               v.data_ptr(), _stream_ptr(stream)), "dpvo_ba_reduced_system")
        return S, v

    def iterate(self, index: int, it: int, n_frames: int, n_patches: int, t0: int):
        """(poses [N,7] f32, depths [P] f32, dxi [N-t0,6] f64 or None) of problem ``index``
        after iteration ``it`` of the last solve (host numpy arrays)."""
        poses = np.empty((n_frames, 7), np.float32)
        depth = np.empty((n_patches,), np.float32)
        dxi = np.empty((n_frames - t0, 6), np.float64)
        _check(self.lib.dpvo_ba_iterate(self.h, index, it, poses.ctypes.data, depth.ctypes.data,
                                        dxi.ctypes.data), "dpvo_ba_iterate")
        return poses, depth, dxi

    def set_timing(self, enable: bool):
        _check(self.lib.dpvo_ba_set_timing(self.h, int(bool(enable))), "dpvo_ba_set_timing")

    def timing(self, cap: int = 4096):
        """[(kind, ms)] of every launch since the last read (kind 0 plan,
        1 linearise/Schur, 2 reduce/Cholesky/retract, 3 Schur assembly, 4 last
        back-substitution)."""
        ms = np.zeros(cap, np.float32)
        kinds = np.zeros(cap, np.int32)
        n = self.lib.dpvo_ba_timing(self.h, ms.ctypes.data, kinds.ctypes.data, cap)
        if n < 0:
            raise BAError(n, "dpvo_ba_timing")
        return [(int(kinds[i]), float(ms[i])) for i in range(n)]

    def backward(self, problems: List[BAProblem], dL_dposes: List[torch.Tensor], dL_ddepth: List[torch.Tensor],
                 stream=None):
        """dL/dtarget and dL/dweight of every problem, given the gradients of a loss
        w.r.t. the final poses [N, 7] and final inverse depths [P].  ``problems``
        hold the state at the START of the forward solve (not modified)."""
        n, dims, probs = self._arrays(problems)
        gts = [torch.empty_like(p.target) for p in problems]
        gws = [torch.empty_like(p.weight) for p in problems]
        keep = [t.contiguous() for t in dL_dposes] + [t.contiguous() for t in dL_ddepth]
        gr = (Grads * n)(*[Grads(keep[b].data_ptr(), keep[n + b].data_ptr(), gts[b].data_ptr(), gws[b].data_ptr())
                           for b in range(n)])
        _check(self.lib.dpvo_ba_backward(self.h, dims, probs, gr, n, _stream_ptr(stream)), "dpvo_ba_backward")
        return gts, gws

    # ---- serving --------------------------------------------------------------
    def serve_start(self, max_frames: int, max_patches: int, max_edges: int, max_iters: int = 2,
                    max_batch: int = 64, max_in_flight: int = 2):
        d = Dims(max_frames, max_patches, max_edges, 0, max_iters, 1.0, 1.0, 0.0, 0.0)
        _check(self.lib.dpvo_ba_serve_start(self.h, ctypes.byref(d), max_batch, max_in_flight), "dpvo_ba_serve_start")

    def serve_stop(self):
        _check(self.lib.dpvo_ba_serve_stop(self.h), "dpvo_ba_serve_stop")

    def session_open(self, scene, n_iters=None) -> int:
        """Open a session from a scenes.Scene (host arrays copied to the device)."""
        fx, fy, cx, cy = (float(v) for v in scene.intrinsics)
        it = scene.n_iters if n_iters is None else n_iters
        d = Dims(scene.n_frames, scene.n_patches, scene.n_edges, scene.t0, it, fx, fy, cx, cy)
        arrs = [np.ascontiguousarray(a) for a in (scene.poses, scene.patches, scene.anchor, scene.kk, scene.jj,
                                                   scene.target, scene.weight)]
        p = Problem(*[a.ctypes.data for a in arrs], None)
        sid = ctypes.c_int64()
        rc = self.lib.dpvo_ba_session_open(self.h, ctypes.byref(d), ctypes.byref(p), ctypes.byref(sid))
        _check(rc, "dpvo_ba_session_open")
        return sid.value

    def session_close(self, sid: int):
        _check(self.lib.dpvo_ba_session_close(self.h, sid), "dpvo_ba_session_close")

    def session_read(self, sid: int, n_frames: int, n_patches: int):
        poses = np.empty((n_frames, 7), np.float32)
        patches = np.empty((n_patches, 3), np.float32)
        _check(self.lib.dpvo_ba_session_read(self.h, sid, poses.ctypes.data, patches.ctypes.data),
               "dpvo_ba_session_read")
        return poses, patches

    @staticmethod
    def _host_ptr(a):
        """(pointer, keep-alive) of a host float32 array: a page-locked torch tensor
        is passed as is (the library reads it in place until the request
        completes), anything else as a contiguous float32 numpy array."""
        if isinstance(a, torch.Tensor):
            a = a.detach()
            if a.is_pinned() and a.dtype == torch.float32 and a.is_contiguous():
                return a.data_ptr(), a
            a = a.cpu().numpy()
        a = np.ascontiguousarray(a, np.float32)
        return a.ctypes.data, a

    def submit(self, sid: int, target, weight) -> int:
        """New factors for a fixed-graph session; ``target``, ``weight`` [E, 2]."""
        pt, kt = self._host_ptr(target)
        pw, kw = self._host_ptr(weight)
        tk = ctypes.c_uint64()
        _check(self.lib.dpvo_ba_submit(self.h, sid, pt, pw, ctypes.byref(tk)), "dpvo_ba_submit")
        self._keep_alive(tk.value, (kt, kw))
        return tk.value

    def _keep_alive(self, ticket, objs):
        if not hasattr(self, "_inflight"):
            self._inflight = {}
        self._inflight[ticket] = objs

    def session_open_window(self, params: "WindowParams") -> int:
        """Open a sliding-window session (empty window)."""
        sid = ctypes.c_int64()
        _check(self.lib.dpvo_ba_session_open_window(self.h, ctypes.byref(params), ctypes.byref(sid)),
               "dpvo_ba_session_open_window")
        return sid.value

    def session_frame_edges(self, sid: int, n_new: int) -> int:
        e = ctypes.c_int32()
        _check(self.lib.dpvo_ba_session_frame_edges(self.h, sid, n_new, ctypes.byref(e)), "dpvo_ba_session_frame_edges")
        return e.value

    def session_dims(self, sid: int) -> "Dims":
        d = Dims()
        _check(self.lib.dpvo_ba_session_dims(self.h, sid, ctypes.byref(d)), "dpvo_ba_session_dims")
        return d

    def submit_frame(self, sid: int, new_xy, delta=None, weight=None) -> int:
        """Append a frame (patch centres ``new_xy`` [n, 2]) to a window session and
        solve it; ``delta``/``weight`` [E, 2] revise the regenerated targets and set
        the weights (E from ``session_frame_edges``), or both None."""
        n_new = int(new_xy.shape[0])
        px, kx = self._host_ptr(new_xy)
        pd, kd = self._host_ptr(delta) if delta is not None else (None, None)
        pw, kw = self._host_ptr(weight) if weight is not None else (None, None)
        tk = ctypes.c_uint64()
        _check(self.lib.dpvo_ba_submit_frame(self.h, sid, px, n_new, pd, pw, ctypes.byref(tk)), "dpvo_ba_submit_frame")
        self._keep_alive(tk.value, (kx, kd, kw))
        return tk.value

    def poll(self, ticket: int):
        """(done, status, latency_ms)."""
        st, lat = ctypes.c_int32(), ctypes.c_double()
        rc = self.lib.dpvo_ba_poll(self.h, ticket, ctypes.byref(st), ctypes.byref(lat))
        if rc == EBUSY:
            return False, None, None
        _check(rc, "dpvo_ba_poll")
        getattr(self, "_inflight", {}).pop(ticket, None)
        return True, st.value, lat.value

    def wait(self, ticket: int, timeout_ms: int = 10000):
        """(status, latency_ms); raises BAError(ETIMEOUT) when the bound runs out."""
        st, lat = ctypes.c_int32(), ctypes.c_double()
        _check(self.lib.dpvo_ba_wait(self.h, ticket, timeout_ms, ctypes.byref(st), ctypes.byref(lat)), "dpvo_ba_wait")
        getattr(self, "_inflight", {}).pop(ticket, None)
        return st.value, lat.value



class PackedBatch:
    """Many problems packed back to back in one tensor per array kind, with the
    ctypes descriptor arrays built once.  ``where`` is "cuda" (device tensors),
    "pinned" (page-locked host tensors, for the host-buffer entry point) or
    "cpu".  ``initial_*`` keep copies of the starting poses and patches."""

    KINDS = [("poses", torch.float32), ("patches", torch.float32), ("anchor", torch.int32), ("kk", torch.int32),
             ("jj", torch.int32), ("target", torch.float32), ("weight", torch.float32)]

    def __init__(self, scenes, where: str = "cuda", n_iters=None):
        self.n = len(scenes)
        self.where = where
        dev = "cuda" if where == "cuda" else "cpu"
        pin = where == "pinned"
        self.flat = {}
        self.offsets = {}
        for name, dt in self.KINDS:
            arrs = [np.ascontiguousarray(getattr(s, name)).reshape(-1) for s in scenes]
            lens = np.array([a.shape[0] for a in arrs], np.int64)
            self.offsets[name] = np.concatenate([[0], np.cumsum(lens)])
            host = torch.from_numpy(np.concatenate(arrs)).to(dt)
            if pin:
                t = torch.empty(host.shape, dtype=dt, pin_memory=True)
                t.copy_(host)
            else:
                t = host.to(dev)
            self.flat[name] = t
        if pin:
            self.status = torch.zeros(self.n, dtype=torch.int32, pin_memory=True)
        else:
            self.status = torch.zeros(self.n, dtype=torch.int32, device=dev)
        self.initial_poses = self.flat["poses"].clone()
        self.initial_patches = self.flat["patches"].clone()
        self.dims = (Dims * self.n)()
        self.probs = (Problem * self.n)()
        for b, s in enumerate(scenes):
            fx, fy, cx, cy = (float(v) for v in s.intrinsics)
            it = s.n_iters if n_iters is None else n_iters
            self.dims[b] = Dims(s.n_frames, s.n_patches, s.n_edges, s.t0, it, fx, fy, cx, cy)
            ptr = []
            for name, dt in self.KINDS:
                t = self.flat[name]
                ptr.append(t.data_ptr() + int(self.offsets[name][b]) * t.element_size())
            ptr.append(self.status.data_ptr() + 4 * b)
            self.probs[b] = Problem(*ptr)
        self.scenes = scenes

    def view(self, name: str, b: int):
        o = self.offsets[name]
        return self.flat[name][o[b]:o[b + 1]]

    def reset(self):
        self.flat["poses"].copy_(self.initial_poses)
        self.flat["patches"].copy_(self.initial_patches)

    def subset(self, b: int):
        """ctypes (dims, probs) arrays holding problem b alone."""
        return (Dims * 1)(self.dims[b]), (Problem * 1)(self.probs[b])

    def bytes_of(self, names) -> int:
        return int(sum(self.flat[n].numel() * self.flat[n].element_size() for n in names))

_default_solver = None


def pose_loss(poses, gt_poses, scale=1.0, stream=None):
    """Pose supervision loss (Sec. 3.4, Eq. 7) of each problem and its gradient
    w.r.t. the predicted poses, on the device (dpvo_ba_pose_loss).

    poses, gt_poses: lists of [N, 7] float32 CUDA tensors (t, q xyzw);
    scale: a float or one per problem (applied to the predicted translations,
    held constant).  Returns (loss [B] tensor, [dL/dposes [N, 7]] list)."""
    lib = load()
    B = len(poses)
    scales = [float(scale)] * B if not isinstance(scale, (list, tuple)) else [float(x) for x in scale]
    if len(gt_poses) != B or len(scales) != B:
        raise ValueError("poses, gt_poses and scale must have one entry per problem")
    dev = poses[0].device if B else torch.device("cuda")
    loss = torch.zeros(B, dtype=torch.float32, device=dev)
    grads, keep, descs = [], [], (PoseLossProblem * max(B, 1))()
    for b in range(B):
        T = poses[b].detach().to(torch.float32).contiguous()
        G = gt_poses[b].detach().to(torch.float32).contiguous()
        if T.shape != G.shape or T.dim() != 2 or T.shape[1] != 7:
            raise ValueError("poses and gt_poses must be matching [N, 7] tensors")
        g = torch.empty_like(T)
        keep += [T, G]
        grads.append(g)
        descs[b] = PoseLossProblem(T.data_ptr(), G.data_ptr(), loss.data_ptr() + 4 * b, g.data_ptr(),
                                   T.shape[0], scales[b])
    _check(lib.dpvo_ba_pose_loss(descs, B, ctypes.c_void_p(_stream_ptr(stream))), "dpvo_ba_pose_loss")
    return loss, grads


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Window:
    """Sliding optimisation window kept on the device (Sec. 3.3; dpvo_ba_window_*).

    append(new_xy) adds a frame with patches at the given pixel centres (a
    [n, 2] float32 CUDA tensor): constant-velocity pose, median inverse depth
    of the previous 3 frames' patches, the oldest frame dropped when full, the
    edges regenerated.  problem() returns the current BAProblem whose tensors
    view the library's arrays (valid until the next append)."""

    def __init__(self, max_frames, max_new_patches, radius, free_poses, intrinsics, n_iters=2):
        self.lib = load()
        fx, fy, cx, cy = (float(v) for v in intrinsics)
        self.params = WindowParams(max_frames, max_new_patches, radius, free_poses, n_iters, fx, fy, cx, cy)
        h = ctypes.c_void_p()
        _check(self.lib.dpvo_ba_window_create(ctypes.byref(self.params), ctypes.byref(h)), "dpvo_ba_window_create")
        self.h = h

    def append(self, new_xy, stream=None):
        xy = new_xy.detach().to(torch.float32).contiguous() if new_xy is not None else None
        n = 0 if xy is None else int(xy.shape[0])
        ptr = ctypes.c_void_p(xy.data_ptr() if n > 0 else 0)
        self._keep = xy
        _check(self.lib.dpvo_ba_window_append(self.h, ptr, n, ctypes.c_void_p(_stream_ptr(stream))),
               "dpvo_ba_window_append")

    def problem(self) -> BAProblem:
        d, p = Dims(), Problem()
        _check(self.lib.dpvo_ba_window_problem(self.h, ctypes.byref(d), ctypes.byref(p)), "dpvo_ba_window_problem")
        N, P, E = d.n_frames, d.n_patches, d.n_edges

        def view(ptr, shape, ts):
            return torch.as_tensor(_DeviceArray(ptr, shape, ts), device="cuda")
        return BAProblem(view(p.poses, (N, 7), "<f4"), view(p.patches, (P, 3), "<f4"), view(p.anchor, (P,), "<i4"),
                         view(p.kk, (E,), "<i4"), view(p.jj, (E,), "<i4"), view(p.target, (E, 2), "<f4"),
                         view(p.weight, (E, 2), "<f4"), (d.fx, d.fy, d.cx, d.cy), d.t0, d.n_iters,
                         status=view(p.status, (1,), "<i4"))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dpvo_ba_window_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def append_windows(windows, new_xy, stream=None):
    """Append one frame to each window in one batched call
    (dpvo_ba_window_append_batch); new_xy: one [n_b, 2] CUDA tensor per window."""
    lib = load()
    n = len(windows)
    xs = [x.detach().to(torch.float32).contiguous() for x in new_xy]
    hs = (ctypes.c_void_p * max(n, 1))(*[w.h for w in windows])
    ps = (ctypes.c_void_p * max(n, 1))(*[x.data_ptr() if x.shape[0] else 0 for x in xs])
    ns = (ctypes.c_int32 * max(n, 1))(*[int(x.shape[0]) for x in xs])
    for w, x in zip(windows, xs):
        w._keep = x
    _check(lib.dpvo_ba_window_append_batch(hs, ps, ns, n, ctypes.c_void_p(_stream_ptr(stream))),
           "dpvo_ba_window_append_batch")


def correlation(fmap0, fmap1, gpatch, kk, jj, coords, level1_scale, out=None, status=None, stream=None):
    """Correlation features of every edge (Sec. 3.2, Eq. 4; dpvo_ba_correlation).

    fmap0 [N, H0, W0, 128] and fmap1 [N, H1, W1, 128] bfloat16 CUDA tensors,
    gpatch [P, 9, 128] bfloat16, kk/jj [E] int32, coords [E, 9, 2] float32
    (level-0 pixels).  Returns (corr [E, 2, 9, 7, 7] float32, status [1] int32)."""
    lib = load()
    N, H, W, D = fmap0.shape
    E = int(kk.shape[0])
    if D != 128 or fmap0.dtype != torch.bfloat16 or fmap1.dtype != torch.bfloat16 or gpatch.dtype != torch.bfloat16:
        raise ValueError("feature maps and patch features must be bfloat16 with 128 channels")
    for t in (fmap0, fmap1, gpatch, kk, jj, coords):
        if not t.is_contiguous():
            raise ValueError("inputs must be contiguous")
    out = torch.empty((E, 2, 9, 7, 7), dtype=torch.float32, device=fmap0.device) if out is None else out
    status = torch.zeros(1, dtype=torch.int32, device=fmap0.device) if status is None else status
    d = CorrDims(N, int(gpatch.shape[0]), E, H, W, int(level1_scale))
    _check(lib.dpvo_ba_correlation(ctypes.byref(d), fmap0.data_ptr(), fmap1.data_ptr(), gpatch.data_ptr(),
                                   kk.data_ptr(), jj.data_ptr(), coords.data_ptr(), out.data_ptr(),
                                   status.data_ptr(), ctypes.c_void_p(_stream_ptr(stream))), "dpvo_ba_correlation")
    return out, status


def default_solver() -> Solver:
    global _default_solver
    if _default_solver is None:
        _default_solver = Solver()
    return _default_solver


class DPVOBAFunction(torch.autograd.Function):
    """Differentiable bundle-adjustment layer: (poses, patches, target, weight)
    -> (final poses, final patches), differentiable w.r.t. the targets and the
    weights (the flow revisions and confidences of the update operator).

    apply(poses [N,7], patches [P,3], target [E,2], weight [E,2], anchor, kk, jj,
          intrinsics (fx, fy, cx, cy), t0, n_iters=2, solver=None)
    """

    @staticmethod
    def forward(ctx, poses, patches, target, weight, anchor, kk, jj, intrinsics, t0, n_iters=2, solver=None):
        solver = solver or default_solver()
        out_poses = poses.detach().clone().contiguous()
        out_patches = patches.detach().clone().contiguous()
        prob = BAProblem(out_poses, out_patches, anchor.contiguous(), kk.contiguous(), jj.contiguous(),
                         target.detach().contiguous(), weight.detach().contiguous(), intrinsics, t0, n_iters)
        solver.solve([prob])
        ctx.save_for_backward(poses.detach().contiguous(), patches.detach().contiguous(),
                              target.detach().contiguous(), weight.detach().contiguous(), anchor, kk, jj)
        ctx.meta = (intrinsics, t0, n_iters, solver)
        return out_poses, out_patches

    @staticmethod
    def backward(ctx, g_poses, g_patches):
        poses, patches, target, weight, anchor, kk, jj = ctx.saved_tensors
        intrinsics, t0, n_iters, solver = ctx.meta
        prob = BAProblem(poses, patches, anchor, kk, jj, target, weight, intrinsics, t0, n_iters)
        if g_poses is None:
            g_poses = torch.zeros_like(poses)
        g_depth = g_patches[:, 2].contiguous() if g_patches is not None else torch.zeros_like(patches[:, 2])
        gts, gws = solver.backward([prob], [g_poses.contiguous()], [g_depth])
        return None, None, gts[0], gws[0], None, None, None, None, None, None, None
