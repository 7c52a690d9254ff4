"""Pins of the window-maintenance oracle (Sec. 3.3): constant velocity reproduces
a constant-velocity trajectory, the lower median obeys its rank definition, the
edges equal the patch-graph rule computed another way, sliding keeps exactly the
newest frames, and a reprojection target equals the direct projection of the
world point.  CPU only."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import window as W

INTR = (320.0, 320.0, 320.0, 240.0)


def test_constant_velocity_extends_a_constant_velocity_trajectory():
    rng = np.random.default_rng(0)
    D = np.eye(4)
    D[:3, :3] = Rotation.from_rotvec(rng.normal(0, 0.05, 3)).as_matrix()
    D[:3, 3] = rng.normal(0, 0.1, 3)
    T0 = np.eye(4)
    T0[:3, :3] = Rotation.random(random_state=rng).as_matrix()
    T0[:3, 3] = rng.normal(0, 1, 3)
    Ts = [np.linalg.matrix_power(D, k) @ T0 for k in range(5)]
    o = W.WindowOracle(10, 2, 4, INTR)
    o.append(np.zeros((0, 2)), poses_now=np.zeros((0, 7)))
    o.append(np.zeros((0, 2)), poses_now=np.stack([W._pose(Ts[0])]))
    o.append(np.zeros((0, 2)), poses_now=np.stack([W._pose(T) for T in Ts[:2]]))
    assert np.allclose(W._mat(o.poses[2]), Ts[2], atol=1e-12)
    o.append(np.zeros((0, 2)), poses_now=np.stack([W._pose(T) for T in Ts[:3]]))
    assert np.allclose(W._mat(o.poses[3]), Ts[3], atol=1e-12)


def test_lower_median_rank_definition():
    rng = np.random.default_rng(1)
    for K in (1, 2, 3, 4, 7, 10, 288):
        a = rng.integers(0, 5, K).astype(np.float32)      # many ties
        v = W.lower_median(a)
        r = (K - 1) // 2
        assert np.sum(a < v) <= r < np.sum(a <= v)
    assert W.lower_median([]) == 1.0


def test_edges_equal_the_graph_rule():
    rng = np.random.default_rng(2)
    o = W.WindowOracle(7, 2, 3, INTR)
    for _ in range(12):
        o.append(rng.uniform(0, 600, (int(rng.integers(0, 6)), 2)))
    kk, jj = o.edges()
    N = len(o.poses)
    mask = np.abs(np.arange(N)[None, :] - o.anchor[:, None]) <= 2
    k2, j2 = np.nonzero(mask)
    assert np.array_equal(kk, k2) and np.array_equal(jj, j2)


def test_sliding_keeps_the_newest_frames_and_their_patches():
    rng = np.random.default_rng(3)
    o = W.WindowOracle(5, 1, 3, INTR)
    ns = [int(rng.integers(0, 5)) for _ in range(30)]
    ids = []
    for f, n in enumerate(ns):
        xy = np.stack([np.arange(n) + 1000.0 * f, np.full(n, float(f))], 1)
        o.append(xy)
    assert len(o.poses) == 5
    assert len(o.patches) == sum(ns[-5:])
    assert np.array_equal(o.patches[:, 1].astype(int), np.repeat(np.arange(25, 30), ns[-5:]))
    assert np.array_equal(o.anchor, np.repeat(np.arange(5), ns[-5:]))
    assert o.t0() == 2


def test_target_is_the_projection_of_the_world_point():
    rng = np.random.default_rng(4)
    o = W.WindowOracle(4, 3, 2, INTR)
    Ms = []
    for a in range(3):
        M = np.eye(4)
        M[:3, :3] = Rotation.from_rotvec(rng.normal(0, 0.1, 3)).as_matrix()
        M[:3, 3] = rng.normal(0, 0.2, 3)
        Ms.append(M)
    Xw = np.array([0.3, -0.2, 4.0, 1.0])
    Xa = Ms[1] @ Xw
    px = (320 * Xa[0] / Xa[2] + 320, 320 * Xa[1] / Xa[2] + 240)
    o.append(np.zeros((0, 2)), poses_now=np.zeros((0, 7)))
    o.append(np.array([px]), poses_now=np.stack([W._pose(Ms[0])]))
    o.poses = np.stack([W._pose(M) for M in Ms[:2]])
    o.patches[0, 2] = 1.0 / Xa[2]
    o.append(np.zeros((0, 2)))
    o.poses[2] = W._pose(Ms[2])
    kk, jj = o.edges()
    tg = o.targets()
    for e, j in enumerate(jj):
        Xj = Ms[j] @ Xw
        assert np.allclose(tg[e], (320 * Xj[0] / Xj[2] + 320, 320 * Xj[1] / Xj[2] + 240), atol=1e-9)
