"""Reduced systems beyond the fused path: more than 15 free poses (up to 32,
a 192 x 192 system), through the C ABI.

The linearise kernel stores the scaled Schur rows and adds the pose-pair
blocks to FP64 partials; the assembly kernel sums the patch products from the
stored rows (compensated FP32 on the CUDA cores by default, three TF32
products on the tensor cores in the TF32 Schur mode); the solve factors S in
FP32 and refines in FP64 (packed storage).  Sec. 3.1: the same Gauss-Newton
step, compared with the FP64 oracle.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from oracle import dense_gn as dg
from oracle import schur
from tests.gpu_util import (TOL_DEPTH, TOL_POSE, end_to_end_errors, iteration_abs_errors, iteration_errors, err,
                            solve_gpu)

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


def test_backward_and_no_alloc_paths_refuse_more_than_15_free_poses(solver):
    sc = S.make_scene(MID16, 14)
    p = ba.problem_from_scene(sc)
    g = torch.zeros_like(p.poses)
    with pytest.raises(ba.BAError) as e:
        solver.backward([p], [g], [torch.zeros_like(p.patches[:, 2])])
    assert e.value.code == ba.EINVAL


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
