"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same seeded inputs.

Tolerances: pose increments and inverse-depth increments 1e-4, gradients 1e-3.
Each output is held to its tolerance in two ways at once (``err``): the
relative 2-norm over a problem's free poses or inverse depths, and a
per-element bound -- the largest error of any one free pose (2-norm of its
6 twist entries, or 7 stored entries) or any one inverse depth, divided by the
largest reference entry of that output -- so that one patch or pose that is
off cannot hide under an aggregate norm.
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


def max_rel(a, b):
    """Per-element error: max_k |a_k - b_k| / max_k |b_k|, where for a 2-D array
    an element is a row (a pose) measured by its 2-norm."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim >= 2:
        da = np.linalg.norm((a - b).reshape(a.shape[0], -1), axis=1)
        nb = np.linalg.norm(b.reshape(b.shape[0], -1), axis=1)
    else:
        da, nb = np.abs(a - b), np.abs(b)
    if da.size == 0:
        return 0.0
    return float(da.max() / max(nb.max(), 1e-300))


def err(a, b):
    """The larger of the relative 2-norm and the per-element error."""
    return max(rel(a, b), max_rel(a, b))


def err_update(x, ref, x0, tol=TOL_POSE):
    """err() of the update x - x0 against ref - x0, where x and ref are FP32
    states stored from the same start x0.  The reference scale of both measures
    is at least 2 FP32 ulps of the state divided by ``tol``: a converged solve's
    update can be smaller than the state's own storage resolution allows to
    compare at ``tol`` (one ulp of a pose coordinate near 2.6 is 2.4e-7), and
    two FP32 results that differ by an ulp are then the same result."""
    x, ref, x0 = (np.asarray(a, np.float64) for a in (x, ref, x0))
    du, dr = x - x0, ref - x0
    floor = 2.0 * 2.0 ** -23 * np.abs(x0).max() / tol
    n_ref = max(np.linalg.norm(dr), floor)
    if du.ndim >= 2:
        e_el = np.linalg.norm((du - dr).reshape(du.shape[0], -1), axis=1).max()
        r_el = max(np.linalg.norm(dr.reshape(dr.shape[0], -1), axis=1).max(), floor)
    else:
        e_el, r_el = np.abs(du - dr).max(), max(np.abs(dr).max(), floor)
    return float(max(np.linalg.norm(du - dr) / n_ref, e_el / r_el))


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
        out.append((err(dxi_t, ref["dxi"][0]) if N > t0 else 0.0, err(dd, ref["dd"][0])))
    return out


def iteration_abs_errors(solver, scene, index, n_iters):
    """Like iteration_errors, but each error is divided by the norm of the
    FIRST iteration's oracle increment: once the iterations converge the
    increments shrink to the FP32 rounding floor, where a relative error says
    nothing; measured against the solve's own update scale it still does."""
    N, P, t0 = scene.n_frames, scene.n_patches, scene.t0
    out, first = [], None
    for t in range(n_iters):
        poses_t, depth_t, dxi_t = solver.iterate(index, t, N, P, t0)
        _, depth_t1, _ = solver.iterate(index, t + 1, N, P, t0)
        ref = dg.solve_scene(scene_at(scene, poses_t, depth_t), n_iters=1)
        dd = depth_t1.astype(np.float64) - depth_t.astype(np.float64)
        if first is None:
            first = (np.asarray(ref["dxi"][0], np.float64), np.asarray(ref["dd"][0], np.float64))
        # both measures of err(), with the first increment as the reference scale
        exi = np.asarray(dxi_t, np.float64) - ref["dxi"][0]
        edd = dd - ref["dd"][0]
        ex = max(np.linalg.norm(exi) / np.linalg.norm(first[0]),
                 np.linalg.norm(exi, axis=1).max() / np.linalg.norm(first[0], axis=1).max())
        ed = max(np.linalg.norm(edd) / np.linalg.norm(first[1]), np.abs(edd).max() / np.abs(first[1]).max())
        out.append((ex, ed))
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
    e_pose = err(poses[t0:] - p0[t0:], ref["poses"][t0:] - p0[t0:]) if scene.n_frames > t0 else 0.0
    e_depth = err(depths - scene.patches[:, 2], ref["depths"] - scene.patches[:, 2].astype(np.float64))
    return e_pose, e_depth, ref


def loss_grads(scene, poses, depths):
    """dL/dposes [N,7] and dL/ddepth [P] of the ground-truth loss at the given final state."""
    gt = scene.poses_gt.astype(np.float64)
    gp = np.zeros((scene.n_frames, 7))
    for a in range(scene.t0, scene.n_frames):
        q = poses[a, 3:].astype(np.float64)
        s = 1.0 if np.dot(q, gt[a, 3:]) >= 0 else -1.0
        gp[a, :3] = 2 * (poses[a, :3] - gt[a, :3])
        gp[a, 3:] = 2 * (q - s * gt[a, 3:])
    gd = 2 * (depths.astype(np.float64) - scene.depth_gt)
    return gp, gd


def oracle_loss(sc, target, weight):
    """The ground-truth loss of the oracle's solve with the given targets and
    weights (for central differences of the layer)."""
    sc2 = dataclasses.replace(sc, target=target, weight=weight)
    out = dg.solve_scene(sc2)
    L = float(np.sum((out["depths"] - sc.depth_gt.astype(np.float64)) ** 2))
    gt = sc.poses_gt.astype(np.float64)
    for a in range(sc.t0, sc.n_frames):
        q = out["poses"][a, 3:]
        s = 1.0 if np.dot(q, gt[a, 3:]) >= 0 else -1.0
        L += np.sum((out["poses"][a, :3] - gt[a, :3]) ** 2) + np.sum((q - s * gt[a, 3:]) ** 2)
    return L
