"""Pose supervision loss (Sec. 3.4, Eq. 7) on the device, through the C ABI
(dpvo_ba_pose_loss), against the FP64 oracle; and its gradient carried through
the layer's backward (dpvo_ba_backward) against the FP64 autograd twin of the
unrolled iterations with the same loss.  Tolerances: loss 1e-5 relative,
pose gradient 1e-4 relative (FP32 arithmetic vs FP64 central differences),
target/weight gradients 1e-3 relative."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from oracle import pose_loss as PL
from oracle import unrolled_grad as ug
from tests.gpu_util import TOL_GRAD, err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def poses_pair(seed, N, rot=0.05, trans=0.05, spread=1.0):
    rng = np.random.default_rng(seed)
    G = np.concatenate([rng.normal(0, spread, (N, 3)), Rotation.random(N, random_state=rng).as_quat()], 1)
    T = G.copy()
    for a in range(N):
        T[a, 3:] = (Rotation.from_rotvec(rng.normal(0, rot, 3)) * Rotation.from_quat(G[a, 3:])).as_quat()
        T[a, :3] += rng.normal(0, trans, 3)
    return T.astype(np.float32), G.astype(np.float32)


def gpu(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


@pytest.mark.parametrize("N,scale,seed", [(8, 1.0, 0), (12, 0.7, 1), (64, 1.3, 2)])
def test_loss_and_gradient_match_oracle(N, scale, seed):
    T, G = poses_pair(seed, N)
    loss, grads = ba.pose_loss([gpu(T)], [gpu(G)], scale)
    torch.cuda.synchronize()
    T64, G64 = T.astype(np.float64), G.astype(np.float64)
    ref = PL.loss(T64, G64, scale)
    assert abs(float(loss[0]) - ref) < 1e-5 * ref
    if N <= 12:   # central differences over 7 N parameters x N^2 logarithms
        gref = PL.grad_fd(T64, G64, scale)
        assert err(grads[0].cpu().numpy(), gref) < 1e-4


def test_large_rotation_errors():
    """Relative errors up to ~2.5 rad: the J_l^-1 series still converges."""
    T, G = poses_pair(3, 6, rot=1.2, trans=0.5)
    loss, grads = ba.pose_loss([gpu(T)], [gpu(G)])
    torch.cuda.synchronize()
    T64, G64 = T.astype(np.float64), G.astype(np.float64)
    twists = PL.pair_twists(T64, G64)
    assert max(np.linalg.norm(x[3:]) for x in twists.values()) > 1.5
    ref = PL.loss(T64, G64)
    assert abs(float(loss[0]) - ref) < 1e-5 * ref
    assert err(grads[0].cpu().numpy(), PL.grad_fd(T64, G64)) < 1e-4


def test_zero_at_ground_truth_and_single_frame():
    _, G = poses_pair(4, 5)
    loss, grads = ba.pose_loss([gpu(G), gpu(G[:1])], [gpu(G), gpu(G[:1])])
    torch.cuda.synchronize()
    assert float(loss[0]) < 1e-4 and float(loss[1]) == 0.0
    assert float(grads[0].abs().max()) == 0.0 and float(grads[1].abs().max()) == 0.0


def test_batch_beyond_one_launch_equals_problems_alone():
    """130 problems (more than one launch's descriptors) equal their solo results bitwise."""
    pairs = [poses_pair(100 + b, 3 + b % 5) for b in range(130)]
    loss, grads = ba.pose_loss([gpu(T) for T, _ in pairs], [gpu(G) for _, G in pairs])
    torch.cuda.synchronize()
    for b in (0, 64, 127, 128, 129):
        l1, g1 = ba.pose_loss([gpu(pairs[b][0])], [gpu(pairs[b][1])])
        torch.cuda.synchronize()
        assert float(l1[0]) == float(loss[b]) and torch.equal(g1[0], grads[b])
    T64, G64 = (x.astype(np.float64) for x in pairs[129])
    assert abs(float(loss[129]) - PL.loss(T64, G64)) < 1e-5 * PL.loss(T64, G64)


def test_invalid_arguments():
    T, G = poses_pair(5, 3)
    big = gpu(np.tile(T, (50, 1)))
    with pytest.raises(ba.BAError) as e:
        ba.pose_loss([big], [big])          # 150 frames > DPVO_BA_MAX_FRAMES
    assert e.value.code == ba.EINVAL


def test_pose_loss_gradient_through_the_layer_matches_twin():
    """L_pose(BA(targets, weights)) on an 8-frame problem: dL/dtarget, dL/dweight
    from dpvo_ba_pose_loss + dpvo_ba_backward vs autograd of the FP64 twin."""
    sc = S.make_scene(S.PLAIN_N8, 7)
    solver = ba.Solver()
    try:
        fwd = ba.problem_from_scene(sc)
        solver.solve([fwd])
        torch.cuda.synchronize()
        _, gp = ba.pose_loss([fwd.poses], [gpu(sc.poses_gt)])
        start = ba.problem_from_scene(sc)
        gts, gws = solver.backward([start], [gp[0]], [torch.zeros_like(start.patches[:, 2])])
        torch.cuda.synchronize()
    finally:
        solver.close()
    target = torch.tensor(np.asarray(sc.target, np.float64), requires_grad=True)
    weight = torch.tensor(np.asarray(sc.weight, np.float64), requires_grad=True)
    R, t, _ = ug.unrolled(sc, target, weight)
    L = PL.loss_torch(R, t, sc.poses_gt)
    rt, rw = torch.autograd.grad(L, [target, weight])
    assert err(gts[0].cpu().numpy(), rt.numpy()) < TOL_GRAD, err(gts[0].cpu().numpy(), rt.numpy())
    assert err(gws[0].cpu().numpy(), rw.numpy()) < TOL_GRAD, err(gws[0].cpu().numpy(), rw.numpy())


def test_eq7_backward_matches_twin_given_the_twins_final_state():
    """Where the 4-5e-4 of the test above comes from.  The Eq. 7 gradient
    xi / |xi| at the smallest active twists (2e-4 here) moves by ~1e-4 when the
    final poses move by 1e-7, the FP32 forward's distance from the FP64 twin's
    final state.  Fed the loss gradient at the twin's own final state (FP64
    central differences of the oracle's Eq. 7 loss), the layer's backward
    matches the twin to 1e-5; fed the gradient at its own final state, it
    carries the loss's sensitivity, and this device kernel's gradient equals the
    central differences at that state to 1e-4."""
    sc = S.make_scene(S.PLAIN_N8, 300)
    target = torch.tensor(np.asarray(sc.target, np.float64), requires_grad=True)
    weight = torch.tensor(np.asarray(sc.weight, np.float64), requires_grad=True)
    R, t, _ = ug.unrolled(sc, target, weight)
    rt, rw = torch.autograd.grad(PL.loss_torch(R, t, sc.poses_gt), [target, weight])
    solver = ba.Solver()
    try:
        fwd = ba.problem_from_scene(sc)
        solver.solve([fwd])
        torch.cuda.synchronize()
        T_gpu = fwd.poses.cpu().numpy().astype(np.float64)
        Rn, tn = R.detach().numpy(), t.detach().numpy()
        T_twin = np.zeros_like(T_gpu)
        for a in range(sc.n_frames):
            q = Rotation.from_matrix(Rn[a]).as_quat()
            T_twin[a] = np.r_[tn[a], q if np.dot(q, T_gpu[a, 3:]) >= 0 else -q]
        _, gp = ba.pose_loss([fwd.poses], [gpu(sc.poses_gt)])
        fd_ours = PL.grad_fd(T_gpu, sc.poses_gt)
        assert err(gp[0].cpu().numpy()[sc.t0:], fd_ours[sc.t0:]) < 1e-4
        start = ba.problem_from_scene(sc)
        g = torch.tensor(PL.grad_fd(T_twin, sc.poses_gt), dtype=torch.float32, device="cuda")
        gts, gws = solver.backward([start], [g], [torch.zeros_like(start.patches[:, 2])])
        torch.cuda.synchronize()
    finally:
        solver.close()
    assert err(gts[0].cpu().numpy(), rt.numpy()) < 1e-5, err(gts[0].cpu().numpy(), rt.numpy())
    assert err(gws[0].cpu().numpy(), rw.numpy()) < 1e-5, err(gws[0].cpu().numpy(), rw.numpy())
