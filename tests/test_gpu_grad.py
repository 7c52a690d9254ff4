"""Hand-written adjoint (dpvo_ba_backward) vs the FP64 references, through the C ABI.

Sec. 3.1: the layer back-propagates through its Gauss-Newton iterations.  The
loss is the squared distance of the final free poses and all inverse depths
from ground truth; gradients w.r.t. the targets and the weights are compared
with (a) the FP64 torch-autograd twin of the unrolled iterations and (b) FP64
central finite differences (h = 1e-6) of the numpy oracle.  Tolerance 1e-3
relative.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from oracle import dense_gn as dg
from oracle import unrolled_grad as ug
from tests.gpu_util import TOL_GRAD, err, loss_grads, oracle_loss

pytestmark = pytest.mark.gpu

SMALL = dataclasses.replace(S.PLAIN_N8, patches_per_frame=16)


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = ba.Solver()
    yield s
    s.close()


def gpu_gradients(solver, scenes):
    """Forward solve (to get the final state), then the backward from the initial state."""
    fwd = [ba.problem_from_scene(sc) for sc in scenes]
    solver.solve(fwd)
    torch.cuda.synchronize()
    start = [ba.problem_from_scene(sc) for sc in scenes]
    gps, gds = [], []
    for sc, p in zip(scenes, fwd):
        gp, gd = loss_grads(sc, p.poses.cpu().numpy(), p.patches[:, 2].cpu().numpy())
        gps.append(torch.tensor(gp, dtype=torch.float32, device="cuda"))
        gds.append(torch.tensor(gd, dtype=torch.float32, device="cuda"))
    gts, gws = solver.backward(start, gps, gds)
    torch.cuda.synchronize()
    for sc, p in zip(scenes, start):   # the inputs are read, never written
        assert torch.equal(p.poses.cpu(), torch.as_tensor(sc.poses))
        assert torch.equal(p.patches.cpu(), torch.as_tensor(sc.patches))
    return [g.cpu().numpy() for g in gts], [g.cpu().numpy() for g in gws]


@pytest.mark.parametrize("spec,seed", [(SMALL, 1), (S.PLAIN_N8, 2)])
def test_backward_matches_autograd_twin(solver, spec, seed):
    sc = S.make_scene(spec, seed)
    gts, gws = gpu_gradients(solver, [sc])
    ref_t, ref_w, _ = ug.gradient(sc)
    assert err(gts[0], ref_t) < TOL_GRAD, err(gts[0], ref_t)
    assert err(gws[0], ref_w) < TOL_GRAD, err(gws[0], ref_w)


def test_backward_batch_of_sixteen_problems(solver):
    """The differentiation workload: 16 eight-frame problems in one batch."""
    scenes = [S.make_scene(S.PLAIN_N8, 100 + b) for b in range(16)]
    gts, gws = gpu_gradients(solver, scenes)
    for b in (0, 7, 15):
        ref_t, ref_w, _ = ug.gradient(scenes[b])
        assert err(gts[b], ref_t) < TOL_GRAD and err(gws[b], ref_w) < TOL_GRAD, b


def test_backward_matches_central_differences(solver):
    """FP64 central differences (h = 1e-6) of the oracle on 32 random coordinates."""
    sc = S.make_scene(SMALL, 3)
    gts, gws = gpu_gradients(solver, [sc])
    rng = np.random.default_rng(5)
    h = 1e-6
    scale_t, scale_w = np.abs(gts[0]).max(), np.abs(gws[0]).max()
    checked = 0
    while checked < 32:
        e, c = int(rng.integers(sc.n_edges)), int(rng.integers(2))
        if sc.anchor[sc.kk[e]] == sc.jj[e]:
            continue
        which = "target" if checked % 2 == 0 else "weight"
        t_p, t_m = sc.target.astype(np.float64), sc.target.astype(np.float64).copy()
        w_p, w_m = sc.weight.astype(np.float64), sc.weight.astype(np.float64).copy()
        t_p = t_p.copy(); w_p = w_p.copy()
        if which == "target":
            t_p[e, c] += h; t_m[e, c] -= h
        else:
            w_p[e, c] += h; w_m[e, c] -= h
        fd = (oracle_loss(sc, t_p, w_p) - oracle_loss(sc, t_m, w_m)) / (2 * h)
        g = gts[0][e, c] if which == "target" else gws[0][e, c]
        scale = scale_t if which == "target" else scale_w
        assert abs(g - fd) < TOL_GRAD * scale, (which, e, c, g, fd)
        checked += 1


def test_window_size_backward_matches_autograd_twin(solver):
    sc = S.make_scene(S.WINDOW_N22, 4)
    gts, gws = gpu_gradients(solver, [sc])
    ref_t, ref_w, _ = ug.gradient(sc)
    assert err(gts[0], ref_t) < TOL_GRAD and err(gws[0], ref_w) < TOL_GRAD


def test_autograd_function_gives_the_same_gradient(solver):
    sc = S.make_scene(SMALL, 6)
    p = ba.problem_from_scene(sc)
    target = p.target.clone().requires_grad_(True)
    weight = p.weight.clone().requires_grad_(True)
    poses, patches = ba.DPVOBAFunction.apply(p.poses, p.patches, target, weight, p.anchor, p.kk, p.jj,
                                             p.intrinsics, p.t0, 2, solver)
    gp, gd = loss_grads(sc, poses.detach().cpu().numpy(), patches[:, 2].detach().cpu().numpy())
    L = (poses * torch.tensor(gp, dtype=torch.float32, device="cuda")).sum() + \
        (patches[:, 2] * torch.tensor(gd, dtype=torch.float32, device="cuda")).sum()
    g_t, g_w = torch.autograd.grad(L, [target, weight])
    ref_t, ref_w, _ = ug.gradient(sc)
    assert err(g_t.cpu().numpy(), ref_t) < TOL_GRAD
    assert err(g_w.cpu().numpy(), ref_w) < TOL_GRAD


def test_tf32_schur_mode_gradient_matches_autograd_twin():
    """The same adjoint with the opt-in tensor-core Schur accumulation."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = ba.Solver(schur_tf32=True)
    try:
        sc = S.make_scene(S.WINDOW_N22, 8)
        gts, gws = gpu_gradients(s, [sc])
        ref_t, ref_w, _ = ug.gradient(sc)
        assert err(gts[0], ref_t) < TOL_GRAD and err(gws[0], ref_w) < TOL_GRAD
    finally:
        s.close()
