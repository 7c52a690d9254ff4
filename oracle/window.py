"""Oracle of the sliding optimisation window (Sec. 3.3 "Expansion" and
"Optimization"), the rules written out in numpy.
TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

Appending a frame to a window of at most ``max_frames`` frames:

1. if the window is full, the oldest frame leaves with every patch extracted
   from it (frame indices shift down by one);
2. the new frame's pose from the constant-velocity model
   T_n = T_{n-1} T_{n-2}^-1 T_{n-1} (world -> camera 4x4 matrices, FP64; the
   previous pose for the second frame, identity for the first);
3. its patches at the given pixel centres, each with the median inverse depth
   of the patches extracted from the previous 3 frames -- the value of rank
   floor((K - 1) / 2) among the K values in sorted order, 1 when K = 0;
4. the edges: patch k to every frame j of the window with
   |j - anchor_k| <= radius, grouped by patch, frames increasing;
5. targets at the reprojection of Eq. 2 at the current state (the patch
   centre for self edges and for points behind the camera), weights 1;
6. t0 = min(n_frames, max(2, n_frames - free_poses)): the first two poses stay
   fixed (gauge and monocular scale).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation


def _mat(p):
    M = np.eye(4)
    q = np.asarray(p[3:7], np.float64)
    M[:3, :3] = Rotation.from_quat(q / np.linalg.norm(q)).as_matrix()
    M[:3, 3] = np.asarray(p[:3], np.float64)
    return M


def _pose(M):
    q = Rotation.from_matrix(M[:3, :3]).as_quat()
    return np.concatenate([M[:3, 3], q])


def lower_median(values):
    v = np.sort(np.asarray(values))
    return v[(len(v) - 1) // 2] if len(v) else np.float32(1.0)


class WindowOracle:
    def __init__(self, max_frames, radius, free_poses, intrinsics):
        self.max_frames, self.R, self.free = max_frames, radius, free_poses
        self.fx, self.fy, self.cx, self.cy = (float(v) for v in intrinsics)
        self.poses = np.zeros((0, 7))          # FP64 (t, q)
        self.patches = np.zeros((0, 3), np.float32)
        self.anchor = np.zeros(0, np.int64)

    def append(self, new_xy, poses_now=None, depths_now=None):
        """new_xy [n, 2]; poses_now / depths_now: the state as it stands before the
        append (the caller may have changed it since the last append)."""
        if poses_now is not None:
            self.poses = np.asarray(poses_now, np.float64).copy()
        if depths_now is not None:
            self.patches[:, 2] = depths_now
        N = len(self.poses)
        # median over the previous 3 frames (before dropping)
        d_new = lower_median(self.patches[self.anchor >= N - 3, 2])
        # constant velocity
        if N == 0:
            Tn = np.eye(4)
        elif N == 1:
            Tn = _mat(self.poses[0])
        else:
            T1, T2 = _mat(self.poses[N - 1]), _mat(self.poses[N - 2])
            Tn = T1 @ np.linalg.inv(T2) @ T1
        poses, patches, anchor = self.poses, self.patches, self.anchor
        if N == self.max_frames:
            keep = anchor >= 1
            poses, patches, anchor = poses[1:], patches[keep], anchor[keep] - 1
        n = len(new_xy)
        new = np.concatenate([np.asarray(new_xy, np.float32), np.full((n, 1), d_new, np.float32)], 1)
        self.poses = np.concatenate([poses, _pose(Tn)[None]], 0)
        self.patches = np.concatenate([patches, new], 0)
        self.anchor = np.concatenate([anchor, np.full(n, len(self.poses) - 1)])

    def edges(self):
        N = len(self.poses)
        kk, jj = [], []
        for k, a in enumerate(self.anchor):
            for j in range(max(0, a - self.R), min(N - 1, a + self.R) + 1):
                kk.append(k)
                jj.append(j)
        return np.array(kk, np.int64), np.array(jj, np.int64)

    def targets(self):
        kk, jj = self.edges()
        out = np.zeros((len(kk), 2))
        Ms = [_mat(p) for p in self.poses]
        for e, (k, j) in enumerate(zip(kk, jj)):
            x, y, d = (float(v) for v in self.patches[k])
            a = int(self.anchor[k])
            if j == a:
                out[e] = (x, y)
                continue
            Xa = np.array([(x - self.cx) / self.fx, (y - self.cy) / self.fy, 1.0]) / d
            Xw = np.linalg.inv(Ms[a]) @ np.append(Xa, 1.0)
            Xj = Ms[j] @ Xw
            if Xj[2] * d > 1e-9:
                out[e] = (self.fx * Xj[0] / Xj[2] + self.cx, self.fy * Xj[1] / Xj[2] + self.cy)
            else:
                out[e] = (x, y)
        return out

    def t0(self):
        return min(len(self.poses), max(2, len(self.poses) - self.free))
