"""Pins of the pose-loss oracle (Sec. 3.4, Eq. 7) against what the mathematics
fixes: the Log/Exp round trip, zero loss at the ground truth, the closed form of
pure translations, the scale convention, and agreement of its two independent
forms (matrix logarithm with finite differences; torch closed form with
autograd).  CPU only."""
import numpy as np
import torch
from scipy.spatial.transform import Rotation

from oracle import pose_loss as PL


def random_poses(rng, N, spread=1.0):
    q = Rotation.random(N, random_state=rng).as_quat()
    t = rng.normal(0, spread, (N, 3))
    return np.concatenate([t, q], 1)


def perturb(rng, G, rot=0.05, trans=0.05):
    T = G.copy()
    for a in range(len(G)):
        dR = Rotation.from_rotvec(rng.normal(0, rot, 3))
        T[a, 3:] = (dR * Rotation.from_quat(G[a, 3:])).as_quat()
        T[a, :3] += rng.normal(0, trans, 3)
    return T


def test_log_exp_round_trip():
    rng = np.random.default_rng(0)
    for _ in range(20):
        xi = np.concatenate([rng.normal(0, 1, 3), rng.normal(0, 0.8, 3)])
        assert np.allclose(PL.log_se3(PL.exp_se3(xi)), xi, atol=1e-10)


def test_zero_at_ground_truth():
    rng = np.random.default_rng(1)
    G = random_poses(rng, 6)
    assert PL.loss(G, G) < 1e-9
    assert np.abs(PL.grad_fd(G[:3], G[:3])).max() < 1e-3   # the norm's kink: subgradient bounded


def test_pure_translations_closed_form():
    rng = np.random.default_rng(2)
    N = 5
    G = np.zeros((N, 7)); G[:, 6] = 1; G[:, :3] = rng.normal(0, 1, (N, 3))
    T = G.copy(); T[:, :3] += rng.normal(0, 0.1, (N, 3))
    L, g = 0.0, np.zeros((N, 3))
    for i in range(N):
        for j in range(N):
            if i != j:
                d = (T[j, :3] - T[i, :3]) - (G[j, :3] - G[i, :3])
                L += np.linalg.norm(d)
                g[j] += d / np.linalg.norm(d)
                g[i] -= d / np.linalg.norm(d)
    assert abs(PL.loss(T, G) - L) < 1e-10 * L
    gf = PL.grad_fd(T, G)
    assert np.allclose(gf[:, :3], g, atol=1e-6)


def test_scale_multiplies_predicted_translations():
    rng = np.random.default_rng(3)
    G = random_poses(rng, 4)
    T = perturb(rng, G)
    Ts = T.copy(); Ts[:, :3] *= 0.7
    assert abs(PL.loss(T, G, 0.7) - PL.loss(Ts, G, 1.0)) < 1e-12


def test_fd_gradient_orthogonal_to_quaternion():
    rng = np.random.default_rng(4)
    G = random_poses(rng, 4)
    T = perturb(rng, G)
    g = PL.grad_fd(T, G)
    for a in range(4):
        q = T[a, 3:] / np.linalg.norm(T[a, 3:])
        assert abs(np.dot(g[a, 3:], q)) < 1e-6 * (1 + np.linalg.norm(g[a, 3:]))


def test_torch_form_matches_matrix_log_form_and_fd_gradient():
    rng = np.random.default_rng(5)
    G = random_poses(rng, 5)
    T = perturb(rng, G, 0.1, 0.1)
    Tt = torch.tensor(T, dtype=torch.float64, requires_grad=True)
    q = Tt[:, 3:] / Tt[:, 3:].norm(dim=1, keepdim=True)
    x, y, z, w = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], -2)
    L = PL.loss_torch(R, Tt[:, :3], G, 0.8)
    assert abs(float(L) - PL.loss(T, G, 0.8)) < 1e-10 * float(L)
    (g,) = torch.autograd.grad(L, [Tt])
    gf = PL.grad_fd(T, G, 0.8)
    assert np.abs(g.numpy() - gf).max() < 1e-6 * np.abs(gf).max()


def test_planted_transposed_relative_pose_is_caught():
    """A plausible slip (T_j T_i^-1 instead of T_i^-1 T_j) changes the loss."""
    rng = np.random.default_rng(6)
    G = random_poses(rng, 4)
    T = perturb(rng, G, 0.1, 0.1)
    wrong = 0.0
    for i in range(4):
        for j in range(4):
            if i != j:
                Ti, Tj, Gi, Gj = PL._mat(T[i]), PL._mat(T[j]), PL._mat(G[i]), PL._mat(G[j])
                E = np.linalg.inv(Gj @ np.linalg.inv(Gi)) @ (Tj @ np.linalg.inv(Ti))
                wrong += np.linalg.norm(PL.log_se3(E))
    assert abs(wrong - PL.loss(T, G)) > 1e-3 * PL.loss(T, G)
