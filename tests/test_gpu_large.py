"""Reduced systems beyond the fused path: more than 15 free poses (up to 32,
a 192 x 192 system), through the C ABI.

The linearise kernel stores the scaled Schur rows and adds the pose-pair
blocks to FP64 partials; the assembly kernel sums the patch products from the
stored rows (compensated FP32 on the CUDA cores by default, three TF32
products on the tensor cores in the TF32 Schur mode); the solve factors S in
FP32 and refines in FP64 (packed storage).  Sec. 3.1: the same Gauss-Newton
step, compared with the FP64 oracle.
"""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from oracle import dense_gn as dg
from oracle import schur
from oracle import unrolled_grad as ug
from tests.gpu_util import (TOL_DEPTH, TOL_GRAD, TOL_POSE, end_to_end_errors, iteration_abs_errors,
                            iteration_errors, err, loss_grads, oracle_loss, solve_gpu)

pytestmark = pytest.mark.gpu

# 40 frames, 32 patches each, radius 16, the last 32 poses free (192 x 192)
MID32 = dataclasses.replace(S.STRESS_N64, n_frames=40, patches_per_frame=32, radius=16, t0=8, n_iters=2)
# just past the fused path: 16 free poses (96 x 96)
MID16 = dataclasses.replace(S.WINDOW_N22, n_frames=24, patches_per_frame=48, radius=12, t0=8)
# 25 free poses (150 x 150): the tensor-core assembly's second product starts mid-frame
MID25 = dataclasses.replace(S.STRESS_N64, n_frames=33, patches_per_frame=32, radius=16, t0=8, n_iters=2)


@pytest.fixture(scope="module", params=[0, 2], ids=["tc-assembly", "fp32-assembly"])
def solver(request):
    """Beyond 15 free poses the default (mode 0) assembles on the tensor cores;
    mode 2 assembles in compensated FP32 on the CUDA cores."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = ba.Solver(schur_tf32=request.param)
    yield s
    s.close()


def schur_tol(solver):
    """Reduced system against the oracle's: compensated FP32 sums reach 2e-6;
    the tensor cores' FP32 accumulation over up to 2048 patches per CTA is
    looser."""
    return 2e-6 if solver.schur_mode == 2 else 2e-5


@pytest.mark.parametrize("spec,seed", [(MID32, 0), (MID16, 1), (MID25, 5)])
def test_reduced_system_matches_oracle_schur(solver, spec, seed):
    sc = S.make_scene(spec, seed)
    prob = ba.problem_from_scene(sc)
    Sg, vg = solver.reduced_system(prob)
    torch.cuda.synchronize()
    pr = dg.Problem.from_scene(sc)
    Sr, vr = schur.reduced_system(pr, pr.T, pr.d)
    print("reduced system rel err", err(Sg.cpu().numpy(), Sr), err(vg.cpu().numpy(), vr))
    assert err(Sg.cpu().numpy(), Sr) < schur_tol(solver)
    assert err(vg.cpu().numpy(), vr) < schur_tol(solver)


@pytest.mark.parametrize("spec,seed", [(MID32, 2), (MID16, 3), (MID25, 6)])
def test_each_iteration_matches_oracle_step(solver, spec, seed):
    sc = S.make_scene(spec, seed)
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for t, (e_xi, e_dd) in enumerate(iteration_errors(solver, sc, 0, sc.n_iters)):
        assert e_xi < TOL_POSE, (t, e_xi)
        assert e_dd < TOL_DEPTH, (t, e_dd)


def test_edges_behind_the_camera_match_oracle(solver):
    """16 free poses (the assembly path) on a scene whose near patches are seen
    from behind by later cameras: those edges are left out on both paths."""
    sc = S.make_scene(dataclasses.replace(MID16, near_frac=0.1), 4)
    pr = dg.Problem.from_scene(sc)
    Z = dg.reproject(pr, pr.T, pr.d)[1][:, 2]
    assert (Z <= dg.Z_MIN).sum() >= 400 and np.abs(Z - dg.Z_MIN).min() > 0.1
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    for t, (e_xi, e_dd) in enumerate(iteration_errors(solver, sc, 0, sc.n_iters)):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH, (t, e_xi, e_dd)
    e_pose, e_depth, _ = end_to_end_errors(sc, probs[0])
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)


def test_whole_solve_matches_oracle_four_iterations(solver):
    sc = S.make_scene(dataclasses.replace(MID32, n_iters=4), 4)
    probs = solve_gpu(solver, [sc])
    assert int(probs[0].status.item()) == 0
    e_pose, e_depth, _ = end_to_end_errors(sc, probs[0])
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)
    for e_xi, e_dd in iteration_abs_errors(solver, sc, 0, sc.n_iters):
        assert e_xi < TOL_POSE and e_dd < TOL_DEPTH


def test_batch_results_equal_results_alone(solver):
    """A mixed batch (16 and 32 free poses, 2 and 4 iterations): each problem
    as when solved by itself, within the tolerance."""
    scenes = [S.make_scene(MID32, 10), S.make_scene(MID16, 11), S.make_scene(dataclasses.replace(MID32, n_iters=4), 12)]
    batch = solve_gpu(solver, scenes)
    for sc, pb in zip(scenes, batch):
        alone = solve_gpu(solver, [sc])[0]
        assert int(pb.status.item()) == 0 and int(alone.status.item()) == 0
        p0 = torch.as_tensor(sc.poses)
        assert err((pb.poses.cpu() - p0).numpy(), (alone.poses.cpu() - p0).numpy()) < TOL_POSE
        d0 = torch.as_tensor(sc.patches[:, 2])
        assert err((pb.patches[:, 2].cpu() - d0).numpy(), (alone.patches[:, 2].cpu() - d0).numpy()) < TOL_DEPTH


def test_bitwise_repeatable(solver):
    sc = S.make_scene(MID32, 13)
    a = solve_gpu(solver, [sc])[0]
    b = solve_gpu(solver, [sc])[0]
    assert torch.equal(a.poses, b.poses) and torch.equal(a.patches, b.patches)


def test_no_alloc_path_refuses_more_than_15_free_poses():
    """The allocation-free entry point has no assembly kernel: EINVAL beyond
    15 free poses (the backward takes up to 32, tested below)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sc = S.make_scene(MID16, 14)
    p = ba.problem_from_scene(sc)
    d, c = p.dims(), p.cstruct()
    rc = ba.load().dpvo_ba_solve_noalloc(None, ctypes.byref(d), ctypes.byref(c),
                                         torch.cuda.current_stream().cuda_stream)
    assert rc == ba.EINVAL


def _grads(solver, sc):
    """Forward solve for the final state, then the adjoint of the
    ground-truth loss from the initial state (as tests/test_gpu_grad.py)."""
    fwd = ba.problem_from_scene(sc)
    solver.solve([fwd])
    torch.cuda.synchronize()
    gp, gd = loss_grads(sc, fwd.poses.cpu().numpy(), fwd.patches[:, 2].cpu().numpy())
    start = ba.problem_from_scene(sc)
    gts, gws = solver.backward([start], [torch.tensor(gp, dtype=torch.float32, device="cuda")],
                               [torch.tensor(gd, dtype=torch.float32, device="cuda")])
    torch.cuda.synchronize()
    assert torch.equal(start.poses.cpu(), torch.as_tensor(sc.poses))
    return gts[0].cpu().numpy(), gws[0].cpu().numpy()


@pytest.mark.parametrize("spec,seed", [(MID16, 15), (MID32, 16)])
def test_backward_beyond_15_free_poses_matches_autograd_twin(solver, spec, seed):
    """The adjoint through the assembly path (16 and 32 free poses, both
    assemblies): the forward keeps each iteration's FP64 factor, and the
    right-hand side sum_k E_k C_k^-1 dbar_k is assembled from the adjoint
    pass's rows.  Against the FP64 torch-autograd twin at 1e-3."""
    sc = S.make_scene(spec, seed)
    gt, gw = _grads(solver, sc)
    ref_t, ref_w, _ = ug.gradient(sc)
    assert err(gt, ref_t) < TOL_GRAD, err(gt, ref_t)
    assert err(gw, ref_w) < TOL_GRAD, err(gw, ref_w)


def test_backward_beyond_15_free_poses_matches_central_differences(solver):
    """FP64 central differences (h = 1e-6) of the dense oracle on 12 random
    target and weight coordinates of a 16-free-pose problem."""
    sc = S.make_scene(dataclasses.replace(MID16, patches_per_frame=16), 17)
    gt, gw = _grads(solver, sc)
    rng = np.random.default_rng(7)
    h, checked = 1e-6, 0
    scale_t, scale_w = np.abs(gt).max(), np.abs(gw).max()
    while checked < 12:
        e, c = int(rng.integers(sc.n_edges)), int(rng.integers(2))
        if sc.anchor[sc.kk[e]] == sc.jj[e]:
            continue
        which = "target" if checked % 2 == 0 else "weight"
        tp, tm = sc.target.astype(np.float64).copy(), sc.target.astype(np.float64).copy()
        wp, wm = sc.weight.astype(np.float64).copy(), sc.weight.astype(np.float64).copy()
        if which == "target":
            tp[e, c] += h; tm[e, c] -= h
        else:
            wp[e, c] += h; wm[e, c] -= h
        fd = (oracle_loss(sc, tp, wp) - oracle_loss(sc, tm, wm)) / (2 * h)
        g = gt[e, c] if which == "target" else gw[e, c]
        scale = scale_t if which == "target" else scale_w
        assert abs(g - fd) < TOL_GRAD * scale, (which, e, c, g, fd)
        checked += 1


@pytest.mark.slow
def test_stress_instance_matches_dense_oracle():
    """One full large-window instance: 64 frames, 256 patches each (16,384),
    radius 24 (649,216 edges), last 32 poses free, 4 iterations, 20% outliers,
    against the dense FP64 oracle (a 16,768-variable Cholesky per iteration),
    with both assembly variants (the default on the tensor cores, mode 2 in
    FP32 on the CUDA cores)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sc = S.make_scene(S.STRESS_N64, 1)
    assert sc.n_patches == 16384 and sc.n_edges == 649216
    ref = None
    for mode in (0, 2):
        s = ba.Solver(schur_tf32=mode)
        probs = solve_gpu(s, [sc])
        s.close()
        assert int(probs[0].status.item()) == 0
        e_pose, e_depth, ref = end_to_end_errors(sc, probs[0], ref)
        print("fp32" if mode == 2 else "tc", "stress errors", e_pose, e_depth)
        assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (mode, e_pose, e_depth)
