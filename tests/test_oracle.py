"""Pins of the FP64 oracle against mathematics it does not contain (CPU only).

Sec. 3.1 Eq. 6 defines the objective, Eq. 2-3 the reprojection; the checks are
finite differences, an independent world-point residual, library least squares,
exact recovery of noiseless scenes, closed forms, the Schur identity and gauge
invariance.  The last group plants mistakes in the oracle and checks that at
least one pin catches each of them.
"""
import dataclasses

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from paper_2208_04726_b300 import scenes as S
from oracle import dense_gn as dg
from oracle import schur
from oracle import unrolled_grad as ug
from tests import oracle_pins as pins

TINY = S.SceneSpec(n_frames=4, patches_per_frame=3, radius=None, t0=2)
SMALL = S.SceneSpec(n_frames=6, patches_per_frame=5, radius=2, t0=2)


def tiny(seed=0, spec=TINY, **kw):
    return S.make_scene(dataclasses.replace(spec, **kw), seed, dtype=np.float64)


# --------------------------------------------------------------- SE(3) helpers

def test_quaternion_conversions_match_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = Rotation.random(random_state=rng).as_quat()
        assert np.allclose(dg.quat_to_matrix(q), Rotation.from_quat(q).as_matrix(), atol=1e-14)
        R = Rotation.from_quat(q).as_matrix()
        q2 = dg.matrix_to_quat(R)
        assert np.allclose(Rotation.from_quat(q2).as_matrix(), R, atol=1e-13)
        assert q2[3] >= 0


def test_exp_se3_special_cases():
    rng = np.random.default_rng(1)
    v, w = rng.normal(size=3), rng.normal(size=3)
    T = dg.exp_se3(np.concatenate([v, np.zeros(3)]))          # pure translation
    assert np.allclose(T[:3, :3], np.eye(3)) and np.allclose(T[:3, 3], v)
    T = dg.exp_se3(np.concatenate([np.zeros(3), w]))          # pure rotation = Rodrigues
    assert np.allclose(T[:3, :3], Rotation.from_rotvec(w).as_matrix(), atol=1e-13)
    # translation along the rotation axis is unchanged by V(w)
    T = dg.exp_se3(np.concatenate([0.7 * w, w]))
    assert np.allclose(T[:3, 3], 0.7 * w, atol=1e-13)
    xi = rng.normal(size=6)
    assert np.allclose(dg.exp_se3(xi) @ dg.exp_se3(-xi), np.eye(4), atol=1e-13)


def test_adjoint_identity():
    rng = np.random.default_rng(2)
    T = dg.exp_se3(rng.normal(size=6))
    xi = 1e-3 * rng.normal(size=6)
    lhs = T @ dg.exp_se3(xi) @ np.linalg.inv(T)
    rhs = dg.exp_se3(dg.adjoint(T) @ xi)
    assert np.allclose(lhs, rhs, atol=1e-13)


# --------------------------------------------------------------- residual model

def test_residual_matches_world_point_form():
    sc = tiny(0)
    assert pins.residual_error(sc) < 1e-9


def test_noiseless_scene_has_zero_residual_at_ground_truth():
    sc = tiny(3, spec=SMALL, noiseless=True)
    gt = dataclasses.replace(sc, poses=sc.poses_gt.copy(),
                             patches=np.concatenate([sc.patches[:, :2], sc.depth_gt[:, None]], 1))
    prob = dg.Problem.from_scene(gt)
    r, active = dg.residuals(prob, prob.T, prob.d)
    assert active.all()
    assert np.abs(r).max() < 1e-9


def test_jacobians_match_finite_differences():
    for seed in range(3):
        assert pins.jacobian_error(tiny(seed)) < 1e-6
    assert pins.jacobian_error(tiny(7, spec=SMALL)) < 1e-6


# --------------------------------------------------------------- one step

def test_gn_step_matches_lstsq_on_fd_jacobian():
    for seed in range(3):
        assert pins.gn_step_error(tiny(seed)) < 1e-6


def test_one_step_update_matches_lstsq_step_with_closed_form_exponential():
    for seed in range(3):
        assert pins.update_error(tiny(seed)) < 1e-6


def test_dense_solve_equals_schur_solve_on_tiny_graphs():
    for seed, spec in [(0, TINY), (1, SMALL), (2, dataclasses.replace(TINY, n_frames=3, patches_per_frame=2, t0=2)),
                       (3, dataclasses.replace(SMALL, n_frames=5, patches_per_frame=4, t0=2))]:
        assert pins.schur_error(tiny(seed, spec=spec)) < 1e-12


def test_all_poses_fixed_reduces_to_per_patch_weighted_least_squares():
    sc = tiny(4, spec=dataclasses.replace(SMALL, t0=SMALL.n_frames))
    assert pins.depth_only_error(sc) < 1e-6


def test_self_edges_contribute_nothing():
    sc = tiny(5)
    keep = sc.anchor[sc.kk] != sc.jj
    sc2 = dataclasses.replace(sc, kk=sc.kk[keep], jj=sc.jj[keep], target=sc.target[keep], weight=sc.weight[keep])
    a = dg.solve_scene(sc, n_iters=1)
    b = dg.solve_scene(sc2, n_iters=1)
    assert np.abs(a["dxi"][0] - b["dxi"][0]).max() < 1e-12
    assert np.abs(a["dd"][0] - b["dd"][0]).max() < 1e-12


def test_gauge_invariance_under_right_multiplication():
    """T_i -> T_i S leaves every relative pose, hence every increment, unchanged."""
    sc = tiny(6, spec=SMALL)
    prob = dg.Problem.from_scene(sc)
    Sg = dg.exp_se3(np.array([0.3, -0.2, 0.5, 0.4, -0.1, 0.2]))
    prob2 = dg.Problem.from_scene(sc)
    prob2.T = prob.T @ Sg
    a = dg.solve(prob, 2)
    b = dg.solve(prob2, 2)
    for t in range(2):
        assert np.abs(a["dxi"][t] - b["dxi"][t]).max() < 1e-9 * max(1.0, np.abs(a["dxi"][t]).max())
        assert np.abs(a["dd"][t] - b["dd"][t]).max() < 1e-9
    assert np.allclose(a["T"] @ Sg, b["T"], atol=1e-9)


# --------------------------------------------------------------- convergence

def test_fixed_point_at_ground_truth():
    sc = tiny(8, spec=SMALL, noiseless=True)
    gt = dataclasses.replace(sc, poses=sc.poses_gt.copy(),
                             patches=np.concatenate([sc.patches[:, :2], sc.depth_gt[:, None]], 1))
    out = dg.solve_scene(gt, n_iters=1)
    assert np.abs(out["dxi"][0]).max() < 1e-10
    assert np.abs(out["dd"][0]).max() < 1e-10


def test_exact_recovery_of_noiseless_scene():
    sc = tiny(9, spec=SMALL, noiseless=True)
    out = dg.solve_scene(sc, n_iters=12)
    assert np.abs(out["depths"] - sc.depth_gt).max() < 1e-9
    gt = sc.poses_gt.astype(np.float64)
    got = out["poses"].copy()
    got[:, 3:] *= np.sign((got[:, 3:] * gt[:, 3:]).sum(1))[:, None]
    assert np.abs(got - gt).max() < 1e-9


@pytest.mark.slow
def test_converged_state_is_the_least_squares_minimiser():
    for seed in range(2):
        assert pins.minimiser_error(tiny(10 + seed)) < 1e-8


# --------------------------------------------------------------- gradient twin

def test_autograd_twin_forward_matches_oracle():
    sc = S.make_scene(S.PLAIN_N8, 11)
    out = dg.solve_scene(sc)
    poses, depths = ug.final_state(sc)
    assert np.abs(poses - out["poses"]).max() < 1e-10
    assert np.abs(depths - out["depths"]).max() < 1e-10


def test_autograd_twin_forward_matches_oracle_with_edges_behind_the_camera():
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, near_frac=0.3), 4)
    assert (pins.wp_homogeneous_depth(sc) <= dg.Z_MIN).sum() >= 4
    out = dg.solve_scene(sc)
    poses, depths = ug.final_state(sc)
    assert np.abs(poses - out["poses"]).max() < 1e-10
    assert np.abs(depths - out["depths"]).max() < 1e-10


def _oracle_loss(sc, target, weight, n_iters=2):
    sc2 = dataclasses.replace(sc, target=target, weight=weight)
    out = dg.solve_scene(sc2, n_iters=n_iters)
    L = float(np.sum((out["depths"] - sc.depth_gt.astype(np.float64)) ** 2))
    gt = sc.poses_gt.astype(np.float64)
    for a in range(sc.t0, sc.n_frames):
        q = out["poses"][a, 3:]
        s = 1.0 if np.dot(q, gt[a, 3:]) >= 0 else -1.0
        L += np.sum((out["poses"][a, :3] - gt[a, :3]) ** 2) + np.sum((q - s * gt[a, 3:]) ** 2)
    return L


def test_autograd_twin_gradient_matches_central_differences():
    """FP64 central differences (h = 1e-6) of the numpy oracle on 32 random
    target / weight coordinates vs the twin's autograd gradient."""
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, patches_per_frame=16), 12, dtype=np.float64)
    gt_, gw_, L = ug.gradient(sc)
    assert abs(L - _oracle_loss(sc, sc.target, sc.weight)) < 1e-12
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(16):
        for which, grad in (("target", gt_), ("weight", gw_)):
            e, c = int(rng.integers(sc.n_edges)), int(rng.integers(2))
            if sc.anchor[sc.kk[e]] == sc.jj[e]:
                continue
            tp, tm = sc.target.copy(), sc.target.copy()
            wp, wm = sc.weight.copy(), sc.weight.copy()
            if which == "target":
                tp[e, c] += h; tm[e, c] -= h
            else:
                wp[e, c] += h; wm[e, c] -= h
            fd = (_oracle_loss(sc, tp, wp) - _oracle_loss(sc, tm, wm)) / (2 * h)
            scale = np.abs(grad).max()
            assert abs(fd - grad[e, c]) < 1e-6 * scale + 1e-9, (which, e, c, fd, grad[e, c])


NEAR_N8 = dataclasses.replace(S.PLAIN_N8, near_frac=0.3)
NEAR_N22 = dataclasses.replace(S.WINDOW_N22, near_frac=0.1)


@pytest.mark.parametrize("spec,seed,min_off", [(NEAR_N8, 4, 4), (NEAR_N8, 11, 4), (NEAR_N22, 1, 200)])
def test_edges_behind_the_camera_take_no_part(spec, seed, min_off):
    """Seeded scenes with patches close to their source camera, seen from behind
    by later cameras: every edge whose homogeneous depth (world-point form) is
    at most z_min contributes nothing to H, g, the increment or the cost.  The
    scenes keep every edge well away from the threshold, so the set does not
    hinge on rounding."""
    sc = S.make_scene(spec, seed)
    zh = pins.wp_homogeneous_depth(sc)
    assert np.abs(zh - dg.Z_MIN).min() > 0.1
    err, n_off = pins.inactive_edge_error(sc)
    assert n_off >= min_off, n_off
    assert err < 1e-12, err


# --------------------------------------------------------------- planted mistakes

@pytest.fixture
def plant(monkeypatch):
    return monkeypatch


def test_pins_catch_a_transposed_adjoint(plant):
    plant.setattr(dg, "adjoint", lambda T: np.swapaxes(_true_adjoint(T), -1, -2))
    assert pins.jacobian_error(tiny(0)) > 1e-3


def test_pins_catch_a_wrong_sign_in_the_rotation_jacobian(plant):
    plant.setattr(dg, "skew", lambda a: -_true_skew(a))
    assert pins.jacobian_error(tiny(0)) > 1e-3 or pins.residual_error(tiny(0)) > 1e-6


def test_pins_catch_dropped_damping(plant):
    plant.setattr(dg, "normal_equations", _normal_equations_without_damping)
    sc = tiny(4, spec=dataclasses.replace(SMALL, t0=SMALL.n_frames))
    sc = dataclasses.replace(sc, weight=sc.weight * 1e-6)   # make lambda matter
    assert pins.depth_only_error(sc) > 1e-3


def test_pins_catch_unweighted_gradient(plant):
    orig = dg.linearize

    def lin(prob, T, d):
        r, Ji, Jj, Jd, act = orig(prob, T, d)
        return r / np.where(prob.weight > 0, prob.weight, 1.0) ** 0.5, Ji, Jj, Jd, act
    plant.setattr(dg, "linearize", lin)
    assert pins.gn_step_error(tiny(1)) > 1e-3


def test_pins_catch_a_retraction_on_the_wrong_side(plant):
    def step(prob, T, d):
        H, g = dg.normal_equations(prob, T, d)
        idx = dg.free_index(prob)
        dx = dg.solve_dense(H[np.ix_(idx, idx)], g[idx])
        nf = prob.N - prob.t0
        dxi, dd = dx[:6 * nf].reshape(nf, 6), dx[6 * nf:]
        T_new = T.copy()
        for a in range(nf):
            T_new[prob.t0 + a] = T[prob.t0 + a] @ dg.exp_se3(dxi[a])
        return T_new, d + dd, dxi, dd
    plant.setattr(dg, "gn_step", step)
    assert pins.update_error(tiny(2)) > 1e-3


_true_adjoint = dg.adjoint
_true_skew = dg.skew
_true_normal_equations = dg.normal_equations


def _normal_equations_without_damping(prob, T, d):
    saved = prob.damping
    prob.damping = 0.0
    try:
        return _true_normal_equations(prob, T, d)
    finally:
        prob.damping = saved


def test_pins_catch_a_dropped_activity_mask(plant):
    orig = dg.reproject

    def rep(prob, T, d):
        G, X, uv, active = orig(prob, T, d)
        Z = X[:, 2]
        uv = np.stack([prob.fx * X[:, 0] / Z + prob.cx, prob.fy * X[:, 1] / Z + prob.cy], axis=1)
        return G, X, uv, np.ones_like(active)
    plant.setattr(dg, "reproject", rep)
    err, _ = pins.inactive_edge_error(S.make_scene(NEAR_N8, 4))
    assert err > 1e-3


def test_pins_catch_an_activity_mask_on_the_residual_only(plant):
    orig = dg.linearize

    def lin(prob, T, d):
        r, Ji, Jj, Jd, act = orig(prob, T, d)
        # Jacobians recomputed as if every edge took part
        G, X, _, _ = dg.reproject(prob, T, d)
        Z = X[:, 2]
        Jpi = np.zeros((X.shape[0], 2, 3))
        Jpi[:, 0, 0] = prob.fx / Z
        Jpi[:, 0, 2] = -prob.fx * X[:, 0] / (Z * Z)
        Jpi[:, 1, 1] = prob.fy / Z
        Jpi[:, 1, 2] = -prob.fy * X[:, 1] / (Z * Z)
        dXj = np.concatenate([X[:, 3, None, None] * np.eye(3)[None], -dg.skew(X[:, :3])], axis=2)
        Jj2 = Jpi @ dXj
        Ji2 = -Jj2 @ dg.adjoint(G)
        Jd2 = np.einsum('eab,eb->ea', Jpi, G[:, :3, 3])
        return r, Ji2, Jj2, Jd2, act
    plant.setattr(dg, "linearize", lin)
    err, _ = pins.inactive_edge_error(S.make_scene(NEAR_N8, 4))
    assert err > 1e-3
