"""The paper's two system configurations on the device-maintained windows
(Sec. 4: Default = 96 patches per frame and a 10-frame optimisation window,
Fast = 48 patches and 7 frames; Sec. 3.3: initialisation on 8 frames with 12
update iterations).  Through the C ABI: a 12-iteration solve against the FP64
oracle, and a mixed Default/Fast batch of sliding windows against the same
windows solved one by one (update within the parity tolerance)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from tests.gpu_util import TOL_DEPTH, TOL_POSE, end_to_end_errors, err, solve_gpu

pytestmark = pytest.mark.gpu

INTR = (320.0, 320.0, 320.0, 240.0)
DEFAULT = dict(max_frames=22, max_new_patches=96, radius=13, free_poses=10)
FAST = dict(max_frames=22, max_new_patches=48, radius=13, free_poses=7)


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = ba.Solver()
    yield s
    s.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_twelve_iteration_initialisation_solve_matches_oracle(solver, seed):
    """An 8-frame problem solved with 12 Gauss-Newton iterations in one call."""
    sc = S.make_scene(dataclasses.replace(S.PLAIN_N8, n_iters=12), 50 + seed)
    p = solve_gpu(solver, [sc])[0]
    assert int(p.status.item()) == 0
    e_pose, e_depth, _ = end_to_end_errors(sc, p)
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)


def filled(kind, n_frames, rng):
    w = ba.Window(n_iters=2, intrinsics=INTR, **kind)
    for _ in range(n_frames):
        n = kind["max_new_patches"]
        w.append(torch.tensor(rng.uniform([16, 16], [624, 464], (n, 2)).astype(np.float32), device="cuda"))
    return w


def test_default_fast_mix_batch_equals_windows_alone(solver):
    rng = np.random.default_rng(3)
    kinds = [DEFAULT, FAST, DEFAULT, FAST, FAST]
    lens = [30, 30, 8, 8, 15]           # full windows, initialisation-sized ones, one in between
    ws = [filled(k, n, rng) for k, n in zip(kinds, lens)]
    try:
        probs = [w.problem() for w in ws]
        torch.cuda.synchronize()
        with torch.no_grad():
            for p in probs:
                p.target += torch.tensor(rng.normal(0, 0.7, tuple(p.target.shape)).astype(np.float32), device="cuda")
        start = [(p.poses.clone(), p.patches.clone()) for p in probs]
        solver.solve(probs)
        torch.cuda.synchronize()
        batch = [(p.poses.clone(), p.patches.clone(), int(p.status.item())) for p in probs]
        assert [p.t0 for p in probs] == [12, 15, 2, 2, 8]
        for p, (p0, q0), (pb, qb, st) in zip(probs, start, batch):
            assert st == 0
            with torch.no_grad():
                p.poses.copy_(p0)
                p.patches.copy_(q0)
            solver.solve([p])
            torch.cuda.synchronize()
            # alone the problem is split into more work items (other summation order): the
            # updates agree within the parity tolerance, not bit for bit
            assert int(p.status.item()) == 0
            assert err((pb - p0).cpu().numpy(), (p.poses - p0).cpu().numpy()) < TOL_POSE
            assert err((qb - q0)[:, 2].cpu().numpy(), (p.patches - q0)[:, 2].cpu().numpy()) < TOL_DEPTH
    finally:
        for w in ws:
            w.close()
