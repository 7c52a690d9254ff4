"""FP64 oracle of the pose supervision loss (Sec. 3.4, Eq. 7).
TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

    L = sum over ordered frame pairs (i, j), i != j, of
        || Log_SE(3)[ (G_i^-1 G_j)^-1 (T_i^-1 T_j) ] ||

T the predicted, G the ground-truth poses (world -> camera, (t, q xyzw)); the
twist is (rho, phi), translation first, with Exp((rho, phi)) = expm([[phi^, rho],
[0, 0]]), and the norm is the Euclidean norm of that 6-vector (the paper writes
the norm, not its square).  The predicted translations are first multiplied by
the alignment scale s (Umeyama in the paper), which is held constant.

Two independent forms:

* ``loss``/``grad_fd``: 4x4 matrices, ``scipy.linalg.logm`` for Log, and the
  gradient with respect to the raw 7 parameters of every pose by central
  differences of L(t, q / |q|) (so the quaternion part is orthogonal to q).
* ``loss_torch``: a differentiable torch form on rotation matrices and
  translations (rotation log from the matrix by atan2, V^-1 in closed form),
  for the gradient through the unrolled Gauss-Newton twin.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
from scipy.spatial.transform import Rotation

import torch

f64 = torch.float64


def _mat(p, s=1.0):
    p = np.asarray(p, np.float64)
    M = np.eye(4)
    M[:3, :3] = Rotation.from_quat(p[3:7] / np.linalg.norm(p[3:7])).as_matrix()
    M[:3, 3] = s * p[:3]
    return M


def log_se3(E):
    """Twist (rho, phi) of a rigid transform by the matrix logarithm."""
    L = scipy.linalg.logm(E)
    L = np.real(L)
    return np.array([L[0, 3], L[1, 3], L[2, 3], L[2, 1], L[0, 2], L[1, 0]])


def exp_se3(xi):
    M = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return scipy.linalg.expm(M)


def pair_twists(T, G, s=1.0):
    """{(i, j): Log((G_i^-1 G_j)^-1 (T_i^-1 T_j))} over ordered pairs i != j."""
    N = len(T)
    TM = [_mat(T[a], s) for a in range(N)]
    GM = [_mat(G[a]) for a in range(N)]
    out = {}
    for i in range(N):
        for j in range(N):
            if i != j:
                P = np.linalg.inv(TM[i]) @ TM[j]
                Q = np.linalg.inv(GM[i]) @ GM[j]
                out[(i, j)] = log_se3(np.linalg.inv(Q) @ P)
    return out


def loss(T, G, s=1.0):
    return float(sum(np.linalg.norm(x) for x in pair_twists(T, G, s).values()))


def grad_fd(T, G, s=1.0, h=1e-6):
    """dL/d(t, q) of every pose by central differences (quaternion renormalised
    inside L, so its component along q is zero)."""
    T = np.asarray(T, np.float64)
    g = np.zeros_like(T)
    for a in range(T.shape[0]):
        for c in range(7):
            Tp, Tm = T.copy(), T.copy()
            Tp[a, c] += h
            Tm[a, c] -= h
            g[a, c] = (loss(Tp, G, s) - loss(Tm, G, s)) / (2 * h)
    return g


# ---- differentiable torch form ----------------------------------------------------


def _vee(W):
    return torch.stack([W[2, 1], W[0, 2], W[1, 0]])


def _hat(v):
    z = torch.zeros((), dtype=v.dtype)
    return torch.stack([torch.stack([z, -v[2], v[1]]), torch.stack([v[2], z, -v[0]]),
                        torch.stack([-v[1], v[0], z])])


def so3_log(R):
    """Rotation vector of R: angle from atan2(|sin|, cos) of the matrix, axis from
    its antisymmetric part (series below 1e-4 rad)."""
    a = 0.5 * _vee(R - R.T)                        # sin(theta) * axis
    c = 0.5 * (R[0, 0] + R[1, 1] + R[2, 2] - 1.0)  # cos(theta)
    sn = torch.sqrt((a * a).sum())
    th = torch.atan2(sn, c)
    if float(th.detach()) < 1e-4:
        return a * (1.0 + th * th / 6.0)
    return a * (th / sn)


def se3_log(R, t):
    """(rho, phi) of (R, t): phi = log R, rho = V(phi)^-1 t."""
    phi = so3_log(R)
    th2 = (phi * phi).sum()
    th = torch.sqrt(th2)
    P = _hat(phi)
    if float(th.detach()) < 1e-3:
        beta = 1.0 / 12.0 + th2 / 720.0
    else:
        beta = (1.0 - th * torch.sin(th) / (2.0 * (1.0 - torch.cos(th)))) / th2
    Vinv = torch.eye(3, dtype=R.dtype) - 0.5 * P + beta * (P @ P)
    return torch.cat([Vinv @ t, phi])


def loss_torch(R, t, G, s=1.0):
    """L of predicted rotations R [N, 3, 3] and translations t [N, 3] (torch, any
    autograd graph) against ground-truth poses G [N, 7] (numpy)."""
    G = np.asarray(G, np.float64)
    RG = [torch.tensor(Rotation.from_quat(G[a, 3:7] / np.linalg.norm(G[a, 3:7])).as_matrix()) for a in range(len(G))]
    tG = [torch.tensor(G[a, :3]) for a in range(len(G))]
    N = R.shape[0]
    L = torch.zeros((), dtype=f64)
    ts = s * t
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            RP = R[i].T @ R[j]
            tP = R[i].T @ (ts[j] - ts[i])
            RQ = RG[i].T @ RG[j]
            tQ = RG[i].T @ (tG[j] - tG[i])
            RE = RQ.T @ RP
            tE = RQ.T @ (tP - tQ)
            L = L + torch.sqrt((se3_log(RE, tE) ** 2).sum())
    return L
