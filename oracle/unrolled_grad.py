"""FP64 torch-autograd twin of the unrolled Gauss-Newton iterations.
TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Sec. 3.1: the layer back-propagates through its Gauss-Newton iterations; the
Appendix "Bundle Adjustment Layer" keeps DROID-SLAM's analytic gradients, which
are not reproduced in the paper.  This module obtains the exact derivative of a
loss on the final state with respect to the targets and weights by automatic
differentiation of the same computation, written independently of
``dense_gn`` (different pose algebra: rotation/translation pairs, the pose-i
Jacobian in its direct form rather than through the adjoint, torch's matrix
exponential and Cholesky).  The derivative includes every path: the solve, the
assembly, the residuals and the dependence of the second iteration's Jacobians
on the first iteration's result.  The active-edge mask is treated as constant
(the scenes keep every reprojected depth far from the threshold).

The loss used by the differentiation workload is the squared distance of the
final free poses and all inverse depths from ground truth:

    L = sum_{a >= t0} |t_a - t_a^gt|^2 + |q_a - s_a q_a^gt|^2 + sum_k (d_k - d_k^gt)^2

with s_a = +-1 the sign that aligns the two quaternions.
"""
from __future__ import annotations

import numpy as np
import torch

DAMPING = 1e-4
Z_MIN = 0.1
f64 = torch.float64


def _rot_from_quat(q):
    q = q / q.norm()
    x, y, z, w = q[0], q[1], q[2], q[3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)]),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)]),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]),
    ])


def quat_from_rot(R):
    """Differentiable rotation -> quaternion (x, y, z, w) on the branch of the
    largest of (trace, R00, R11, R22)."""
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    diag = torch.stack([R[0, 0], R[1, 1], R[2, 2]])
    if tr >= diag.max():
        s = 2.0 * torch.sqrt(1.0 + tr)
        q = torch.stack([(R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s,
                         (R[1, 0] - R[0, 1]) / s, 0.25 * s])
    else:
        a = int(torch.argmax(diag))
        b, c = (a + 1) % 3, (a + 2) % 3
        s = 2.0 * torch.sqrt(1.0 + R[a, a] - R[b, b] - R[c, c])
        comp = [None] * 4
        comp[a] = 0.25 * s
        comp[b] = (R[b, a] + R[a, b]) / s
        comp[c] = (R[c, a] + R[a, c]) / s
        comp[3] = (R[c, b] - R[b, c]) / s
        q = torch.stack(comp)
    q = q / q.norm()
    return q


def _cross_mat(a):
    z = torch.zeros_like(a[..., 0])
    return torch.stack([
        torch.stack([z, -a[..., 2], a[..., 1]], -1),
        torch.stack([a[..., 2], z, -a[..., 0]], -1),
        torch.stack([-a[..., 1], a[..., 0], z], -1),
    ], -2)


def _twist(xi):
    M = torch.zeros(xi.shape[0], 4, 4, dtype=f64)
    M = M.clone()
    M[:, :3, :3] = _cross_mat(xi[:, 3:6])
    M[:, :3, 3] = xi[:, 0:3]
    return M


def unrolled(scene, target, weight, n_iters=2, damping=DAMPING, z_min=Z_MIN):
    """Differentiable forward pass; returns final (R (N,3,3), t (N,3), d (P,))."""
    poses = torch.tensor(np.asarray(scene.poses, np.float64))
    N = poses.shape[0]
    R = torch.stack([_rot_from_quat(poses[n, 3:7]) for n in range(N)])
    t = poses[:, :3].clone()
    patches = torch.tensor(np.asarray(scene.patches, np.float64))
    d = patches[:, 2].clone()
    fx, fy, cx, cy = (float(v) for v in scene.intrinsics)
    anchor = torch.tensor(np.asarray(scene.anchor, np.int64))
    kk = torch.tensor(np.asarray(scene.kk, np.int64))
    jj = torch.tensor(np.asarray(scene.jj, np.int64))
    ii = anchor[kk]
    P = d.shape[0]
    t0 = int(scene.t0)
    nf = N - t0
    pbar = torch.stack([(patches[:, 0] - cx) / fx, (patches[:, 1] - cy) / fy,
                        torch.ones(P, dtype=f64)], 1)[kk]                  # (E, 3)
    E = kk.shape[0]
    for _ in range(n_iters):
        Rij = R[jj] @ R[ii].transpose(1, 2)
        tij = t[jj] - (Rij @ t[ii][:, :, None])[:, :, 0]
        dk = d[kk]
        X = (Rij @ pbar[:, :, None])[:, :, 0] + tij * dk[:, None]
        act = (X[:, 2] > z_min).detach()
        Z = torch.where(act, X[:, 2], torch.ones_like(X[:, 2]))
        uv = torch.stack([fx * X[:, 0] / Z + cx, fy * X[:, 1] / Z + cy], 1)
        a = act.to(f64)[:, None]
        r = (target - uv) * a
        zero = torch.zeros(E, dtype=f64)
        Jpi = torch.stack([
            torch.stack([fx / Z, zero, -fx * X[:, 0] / (Z * Z)], 1),
            torch.stack([zero, fy / Z, -fy * X[:, 1] / (Z * Z)], 1)], 1) * a[:, :, None]
        eye = torch.eye(3, dtype=f64).expand(E, 3, 3)
        # perturbing T_j on the left moves X by [W I, -[X]x] xi_j  (W = d_k)
        Jj = Jpi @ torch.cat([dk[:, None, None] * eye, -_cross_mat(X)], 2)
        # perturbing T_i on the left moves X by -R_ij [d I, -[pbar]x] xi_i
        Ji = -(Jpi @ Rij) @ torch.cat([dk[:, None, None] * eye, -_cross_mat(pbar)], 2)
        Jd = (Jpi @ tij[:, :, None])[:, :, 0]
        # dense normal equations over (poses t0..N-1, all inverse depths)
        J = torch.cat([Ji, Jj, Jd[:, :, None]], 2)                          # (E,2,13)
        col = torch.cat([6 * (ii[:, None] - t0) + torch.arange(6), 6 * (jj[:, None] - t0) + torch.arange(6),
                         (6 * nf + kk)[:, None]], 1)                         # (E,13)
        keep = torch.cat([(ii >= t0)[:, None].expand(E, 6), (jj >= t0)[:, None].expand(E, 6),
                          torch.ones(E, 1, dtype=torch.bool)], 1)
        col = torch.where(keep, col, torch.zeros_like(col))
        J = J * keep.to(f64)[:, None, :]
        WJ = weight[:, :, None] * J
        Hloc = torch.einsum('eca,ecb->eab', J, WJ)
        gloc = torch.einsum('eca,ec->ea', WJ, r)
        n = 6 * nf + P
        rows = col[:, :, None].expand(E, 13, 13).reshape(-1)
        cols = col[:, None, :].expand(E, 13, 13).reshape(-1)
        H = torch.zeros(n, n, dtype=f64).index_put((rows, cols), Hloc.reshape(-1), accumulate=True)
        g = torch.zeros(n, dtype=f64).index_put((col.reshape(-1),), gloc.reshape(-1), accumulate=True)
        H = H + torch.diag(torch.cat([torch.zeros(6 * nf, dtype=f64), torch.full((P,), damping, dtype=f64)]))
        L = torch.linalg.cholesky(H)
        dx = torch.cholesky_solve(g[:, None], L)[:, 0]
        dxi = dx[:6 * nf].reshape(nf, 6)
        dd = dx[6 * nf:]
        Ex = torch.linalg.matrix_exp(_twist(dxi))
        Rf = Ex[:, :3, :3] @ R[t0:]
        tf = (Ex[:, :3, :3] @ t[t0:][:, :, None])[:, :, 0] + Ex[:, :3, 3]
        R = torch.cat([R[:t0], Rf], 0)
        t = torch.cat([t[:t0], tf], 0)
        d = d + dd
    return R, t, d


def gt_loss(scene, R, t, d):
    """Squared distance of final free poses and all inverse depths from ground truth."""
    gt = torch.tensor(np.asarray(scene.poses_gt, np.float64))
    dgt = torch.tensor(np.asarray(scene.depth_gt, np.float64))
    L = ((d - dgt) ** 2).sum()
    for a in range(int(scene.t0), R.shape[0]):
        q = quat_from_rot(R[a])
        qg = gt[a, 3:7]
        s = 1.0 if float(torch.dot(q.detach(), qg)) >= 0 else -1.0
        L = L + ((t[a] - gt[a, :3]) ** 2).sum() + ((q - s * qg) ** 2).sum()
    return L


def gradient(scene, n_iters=2, damping=DAMPING, z_min=Z_MIN):
    """dL/dtarget (E,2) and dL/dweight (E,2) of the ground-truth loss through
    n_iters unrolled iterations, and the loss value."""
    target = torch.tensor(np.asarray(scene.target, np.float64), requires_grad=True)
    weight = torch.tensor(np.asarray(scene.weight, np.float64), requires_grad=True)
    R, t, d = unrolled(scene, target, weight, n_iters, damping, z_min)
    L = gt_loss(scene, R, t, d)
    gt_, gw_ = torch.autograd.grad(L, [target, weight])
    return gt_.numpy(), gw_.numpy(), float(L.detach())


def final_state(scene, n_iters=2, damping=DAMPING, z_min=Z_MIN):
    """Final (poses (N,7) with qw >= 0, depths) of the twin, for cross-checking."""
    with torch.no_grad():
        target = torch.tensor(np.asarray(scene.target, np.float64))
        weight = torch.tensor(np.asarray(scene.weight, np.float64))
        R, t, d = unrolled(scene, target, weight, n_iters, damping, z_min)
        out = []
        for a in range(R.shape[0]):
            q = quat_from_rot(R[a])
            if q[3] < 0:
                q = -q
            out.append(torch.cat([t[a], q]))
        return torch.stack(out).numpy(), d.numpy()
