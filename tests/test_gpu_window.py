"""Window maintenance on the device (Sec. 3.3; dpvo_ba_window_*) against the
oracle, append by append, through the C ABI.  Integer arrays (anchors, edges)
and the patch centres and inverse depths are compared bit for bit; poses
within 1e-5 (FP64 composition stored as FP32), targets within 2e-3 px."""
import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from oracle import window as W

pytestmark = pytest.mark.gpu

INTR = (320.0, 320.0, 320.0, 240.0)


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def check(win, o):
    p = win.problem()
    torch.cuda.synchronize()
    kk, jj = o.edges()
    assert p.poses.shape[0] == len(o.poses) and p.patches.shape[0] == len(o.patches) and p.kk.shape[0] == len(kk)
    assert p.t0 == o.t0()
    assert np.array_equal(p.anchor.cpu().numpy(), o.anchor)
    assert np.array_equal(p.kk.cpu().numpy(), kk) and np.array_equal(p.jj.cpu().numpy(), jj)
    assert np.array_equal(p.patches.cpu().numpy(), o.patches)
    gp = p.poses.cpu().numpy().astype(np.float64)
    op = o.poses.copy()
    op[:, 3:] *= np.sign((op[:, 3:] * gp[:, 3:]).sum(1))[:, None]
    assert np.abs(gp - op).max() < 1e-5
    if len(kk):
        assert np.abs(p.target.cpu().numpy() - o.targets()).max() < 2e-3
        assert torch.all(p.weight == 1.0)


def test_append_sequence_matches_oracle():
    rng = np.random.default_rng(0)
    win = ba.Window(8, 12, 3, 4, INTR)
    o = W.WindowOracle(8, 3, 4, INTR)
    try:
        for f in range(25):
            p = win.problem() if f > 0 else None
            if p is not None:   # a solve would move poses and depths: perturb them through the views
                with torch.no_grad():
                    p.poses[:, :3] += torch.tensor(rng.normal(0, 0.01, (p.poses.shape[0], 3)), dtype=torch.float32,
                                                   device="cuda")
                    if p.patches.shape[0]:
                        p.patches[:, 2] *= torch.tensor(rng.uniform(0.9, 1.1, p.patches.shape[0]),
                                                        dtype=torch.float32, device="cuda")
                torch.cuda.synchronize()
            n = int(rng.integers(0, 13)) if f % 5 else 0
            xy = rng.uniform([0, 0], [640, 480], (n, 2)).astype(np.float32)
            poses_now = p.poses.cpu().numpy() if p is not None else np.zeros((0, 7))
            depths_now = p.patches[:, 2].cpu().numpy() if p is not None else None
            win.append(torch.tensor(xy, device="cuda"))
            o.append(xy, poses_now=poses_now, depths_now=depths_now)
            check(win, o)
    finally:
        win.close()


def test_full_sliding_window_sizes_and_a_solve():
    """22 frames, 96 patches each, radius 13, 10 free poses: once full, the edge
    count is that of the sliding-window workload (39,552); a batched solve on
    the maintained windows runs with status OK."""
    rng = np.random.default_rng(1)
    wins = [ba.Window(22, 96, 13, 10, INTR) for _ in range(3)]
    try:
        for f in range(30):
            ba.append_windows(wins, [torch.tensor(rng.uniform([16, 16], [624, 464], (96, 2)).astype(np.float32),
                                                  device="cuda") for _ in wins])
        probs = [w.problem() for w in wins]
        assert all(p.kk.shape[0] == 39552 and p.poses.shape[0] == 22 and p.t0 == 12 for p in probs)
        with torch.no_grad():   # targets: the reprojection plus a small revision
            for p in probs:
                p.target += torch.randn_like(p.target) * 0.5
        solver = ba.Solver()
        solver.solve(probs)
        torch.cuda.synchronize()
        assert all(int(p.status.item()) == 0 for p in probs)
        solver.close()
    finally:
        for w in wins:
            w.close()


def test_batched_append_equals_single_appends():
    """Three windows appended together equal three appended alone (bitwise)."""
    rng = np.random.default_rng(2)
    a = [ba.Window(6, 10, 2, 3, INTR) for _ in range(3)]
    b = [ba.Window(6, 10, 2, 3, INTR) for _ in range(3)]
    try:
        for f in range(9):
            xs = [torch.tensor(rng.uniform(0, 400, (int(rng.integers(0, 11)), 2)).astype(np.float32), device="cuda")
                  for _ in range(3)]
            ba.append_windows(a, xs)
            for w, x in zip(b, xs):
                w.append(x)
            torch.cuda.synchronize()
            for wa, wb in zip(a, b):
                pa, pb = wa.problem(), wb.problem()
                for name in ("poses", "patches", "anchor", "kk", "jj", "target", "weight"):
                    assert torch.equal(getattr(pa, name), getattr(pb, name)), name
        with pytest.raises(ba.BAError):
            ba.append_windows([a[0], a[0]], [xs[0], xs[0]])
    finally:
        for w in a + b:
            w.close()


def test_invalid_arguments():
    with pytest.raises(ba.BAError):
        ba.Window(0, 8, 2, 2, INTR)
    win = ba.Window(4, 8, 2, 2, INTR)
    try:
        with pytest.raises(ba.BAError) as e:
            win.append(torch.zeros(9, 2, device="cuda"))
        assert e.value.code == ba.EINVAL
        with pytest.raises(ba.BAError):
            win.problem()                 # empty window
    finally:
        win.close()
