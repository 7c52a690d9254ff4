"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same seeded inputs.

Tolerances (relative 2-norm over a problem's free poses or inverse depths):
pose increments and inverse-depth increments 1e-4, gradients 1e-3.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from paper_2208_04726_b300 import ba
from oracle import dense_gn as dg

TOL_POSE = 1e-4
TOL_DEPTH = 1e-4
TOL_GRAD = 1e-3


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / max(nb, 1e-300)


def align_quats(poses, ref):
    out = np.asarray(poses, np.float64).copy()
    s = np.sign((out[:, 3:] * ref[:, 3:]).sum(1))
    s[s == 0] = 1
    out[:, 3:] *= s[:, None]
    return out


def scene_at(scene, poses, depths):
    """The scene with its state replaced (poses [N,7], inverse depths [P])."""
    patches = np.concatenate([scene.patches[:, :2], np.asarray(depths, np.float32)[:, None]], 1)
    return dataclasses.replace(scene, poses=np.asarray(poses, np.float32), patches=patches.astype(np.float32))


def solve_gpu(solver, scenes, n_iters=None):
    probs = [ba.problem_from_scene(s, n_iters=n_iters) for s in scenes]
    solver.solve(probs)
    torch.cuda.synchronize()
    return probs


def iteration_errors(solver, scene, index, n_iters):
    """Teacher-forced per-iteration errors: for every iteration t, the oracle
    takes one Gauss-Newton step from the CUDA path's own iterate t, and the two
    increments are compared."""
    N, P, t0 = scene.n_frames, scene.n_patches, scene.t0
    out = []
    for t in range(n_iters):
        poses_t, depth_t, dxi_t = solver.iterate(index, t, N, P, t0)
        _, depth_t1, _ = solver.iterate(index, t + 1, N, P, t0)
        ref = dg.solve_scene(scene_at(scene, poses_t, depth_t), n_iters=1)
        dd = depth_t1.astype(np.float64) - depth_t.astype(np.float64)
        out.append((rel(dxi_t, ref["dxi"][0]) if N > t0 else 0.0, rel(dd, ref["dd"][0])))
    return out


def iteration_abs_errors(solver, scene, index, n_iters):
    """Like iteration_errors, but each error is divided by the norm of the
    FIRST iteration's oracle increment: once the iterations converge the
    increments shrink to the FP32 rounding floor, where a relative error says
    nothing; measured against the solve's own update scale it still does."""
    N, P, t0 = scene.n_frames, scene.n_patches, scene.t0
    out, scale = [], None
    for t in range(n_iters):
        poses_t, depth_t, dxi_t = solver.iterate(index, t, N, P, t0)
        _, depth_t1, _ = solver.iterate(index, t + 1, N, P, t0)
        ref = dg.solve_scene(scene_at(scene, poses_t, depth_t), n_iters=1)
        dd = depth_t1.astype(np.float64) - depth_t.astype(np.float64)
        if scale is None:
            scale = (np.linalg.norm(ref["dxi"][0]), np.linalg.norm(ref["dd"][0]))
        out.append((np.linalg.norm(dxi_t - ref["dxi"][0]) / scale[0], np.linalg.norm(dd - ref["dd"][0]) / scale[1]))
    return out


def end_to_end_errors(scene, prob, ref=None):
    """Errors of the whole solve's update (final - initial state) against the
    oracle's, for poses and inverse depths."""
    if ref is None:
        ref = dg.solve_scene(scene)
    poses = align_quats(prob.poses.cpu().numpy(), ref["poses"])
    depths = prob.patches[:, 2].cpu().numpy().astype(np.float64)
    p0 = align_quats(scene.poses, ref["poses"])
    t0 = scene.t0
    e_pose = rel(poses[t0:] - p0[t0:], ref["poses"][t0:] - p0[t0:]) if scene.n_frames > t0 else 0.0
    e_depth = rel(depths - scene.patches[:, 2], ref["depths"] - scene.patches[:, 2].astype(np.float64))
    return e_pose, e_depth, ref
