"""Seeded synthetic bundle-adjustment scenes for the DPVO patch graph.

This module only draws random numbers and lays them out; it holds none of the
bundle-adjustment arithmetic (no inverse-depth reprojection, no Jacobians, no
normal equations, no Lie-group retraction).  Rotations come from
``scipy.spatial.transform.Rotation`` and the synthetic image measurements are
made with a plain world-point pinhole camera, which is how a scene is rendered,
not how the method solves it.  Both the CUDA path and the oracle consume the
float32 arrays returned here.

Scene recipe (the paper measures on TartanAir / EuRoC / TUM-RGBD / ICL-NUIM;
those recordings and the trained update operator that would produce the flow
revisions and confidences are not available, so seeded synthetic scenes of the
same shapes stand in for them):

* Intrinsics fx = fy = 320, cx = 320, cy = 240 (a 640x480 image).
* Trajectory: camera centre takes 0.1 m steps along a direction that turns by
  at most 15 degrees per frame; orientation turns by 2 degrees per frame about
  an axis that itself drifts by at most 15 degrees per frame.
* Patches (Sec. 3, Eq. 1): ``patches_per_frame`` random pixel centres per frame,
  uniform in the image, at a depth U[1, 10] m in their source frame.  A point is
  redrawn until its homogeneous depth (depth in frame j times the inverse depth
  in the source frame) is at least 0.5 in every frame it is connected to.
* Patch graph (Sec. 3 "Patch Graph"): patch k from frame i has an edge to every
  frame j with |i - j| <= r (all frames when r is None), self edge included.
  Edges are grouped by patch, patches by source frame, frames ascending.
* Factors (Eq. 6): target = true projection + N(0, 0.5 px^2) per component;
  a fraction of edges are outliers displaced by U[5, 30] px in a uniform random
  direction.  Weights are U[0, 1] per component (outliers U[0, 0.05] unless
  ``outlier_weights_uniform``).
* Near patches (``near_frac`` > 0, off in the benchmark workloads): that
  fraction of the patches, drawn from a separate stream, is placed 0.15-0.4 m
  in front of its source camera, so that cameras further along the path see
  it from behind.  Their edges are kept only where the true homogeneous depth
  is clearly on one side of the activity threshold (>= 0.5 or <= -0.5), so an
  edge's part in the solve does not hinge on rounding; the patches then have
  gaps in their frame lists.  A drawn near patch left with fewer than 4 clearly
  active edges to other frames stays a regular patch (its inverse depth would
  be poorly determined).
* Initial state: every free pose (index >= t0) is moved by a 2-degree rotation
  about a random axis and a 5 cm translation in a random direction (applied on
  the world->camera side); fixed poses stay at ground truth; inverse depths are
  scaled by U[0.8, 1.2].

Poses are world->camera, stored as [tx, ty, tz, qx, qy, qz, qw] with qw >= 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np
from scipy.spatial.transform import Rotation

FX, FY, CX, CY = 320.0, 320.0, 320.0, 240.0
WIDTH, HEIGHT = 640, 480


@dataclass(frozen=True)
class SceneSpec:
    n_frames: int
    patches_per_frame: int
    radius: Optional[int]  # None: every patch connects to every frame
    t0: int                # poses [0, t0) are fixed
    n_iters: int = 2
    outlier_frac: float = 0.10
    outlier_weights_uniform: bool = False
    noise_var: float = 0.5
    init_rot_deg: float = 2.0
    init_trans: float = 0.05
    noiseless: bool = False  # no pixel noise, no outliers, unit weights
    near_frac: float = 0.0   # patches placed close to their source camera (see the module docstring)

    @property
    def n_patches(self) -> int:
        return self.n_frames * self.patches_per_frame


# The five workloads of the benchmark suite, by what they are.
PLAIN_N8 = SceneSpec(n_frames=8, patches_per_frame=64, radius=None, t0=2)
WINDOW_N22 = SceneSpec(n_frames=22, patches_per_frame=96, radius=13, t0=12)
STRESS_N64 = SceneSpec(n_frames=64, patches_per_frame=256, radius=24, t0=32,
                       n_iters=4, outlier_frac=0.20, outlier_weights_uniform=True)


def serving_spec(rng: np.random.Generator) -> SceneSpec:
    """One session of the serving mix: N ~ U{8..32}, {48, 64, 96} patches per
    frame, radius ~ U{8..13}, the last min(10, N - 2) poses free."""
    n = int(rng.integers(8, 33))
    ppf = int(rng.choice([48, 64, 96]))
    r = int(rng.integers(8, 14))
    return SceneSpec(n_frames=n, patches_per_frame=ppf, radius=r, t0=n - min(10, n - 2))


@dataclass
class Scene:
    spec: SceneSpec
    seed: int
    intrinsics: np.ndarray   # [4] float32 fx fy cx cy
    poses: np.ndarray        # [N, 7] float32, initial state
    patches: np.ndarray      # [P, 3] float32 x y d (initial inverse depth)
    anchor: np.ndarray       # [P] int32 source frame
    kk: np.ndarray           # [E] int32 patch of each edge
    jj: np.ndarray           # [E] int32 frame of each edge
    target: np.ndarray       # [E, 2] float32
    weight: np.ndarray       # [E, 2] float32
    poses_gt: np.ndarray     # [N, 7] float32
    depth_gt: np.ndarray     # [P] float32 inverse depth
    outlier: np.ndarray = field(default=None)  # [E] bool
    uv_true: np.ndarray = field(default=None)  # [E, 2] float64 noiseless measurement

    @property
    def n_frames(self) -> int:
        return self.poses.shape[0]

    @property
    def n_patches(self) -> int:
        return self.patches.shape[0]

    @property
    def n_edges(self) -> int:
        return self.kk.shape[0]

    @property
    def t0(self) -> int:
        return self.spec.t0

    @property
    def n_iters(self) -> int:
        return self.spec.n_iters


def _unit(v):
    return v / np.linalg.norm(v)


def _turn(rng, v, max_deg):
    """Rotate unit vector v by a random angle <= max_deg about a random axis."""
    axis = _unit(rng.normal(size=3))
    ang = np.deg2rad(max_deg) * rng.uniform()
    return _unit(Rotation.from_rotvec(axis * ang).apply(v))


def _trajectory(rng, n, step_t=0.1, step_deg=2.0):
    """Camera-to-world rotations and centres of a smooth random walk."""
    rots = [Rotation.identity()]
    centres = [np.zeros(3)]
    direction = _unit(rng.normal(size=3))
    axis = _unit(rng.normal(size=3))
    for _ in range(1, n):
        direction = _turn(rng, direction, 15.0)
        axis = _turn(rng, axis, 15.0)
        centres.append(centres[-1] + step_t * direction)
        rots.append(rots[-1] * Rotation.from_rotvec(axis * np.deg2rad(step_deg)))
    return rots, np.array(centres)


def _pack(rot_wc: Rotation, t_wc: np.ndarray) -> np.ndarray:
    q = rot_wc.as_quat()  # x y z w
    if q[3] < 0:
        q = -q
    return np.concatenate([t_wc, q])


def _frames_of(i, n, radius):
    if radius is None:
        return np.arange(n)
    return np.arange(max(0, i - radius), min(n - 1, i + radius) + 1)


def _draw_factors(rng, spec, uv_true, E):
    target = uv_true.copy()
    weight = np.ones((E, 2))
    outlier = np.zeros(E, dtype=bool)
    if not spec.noiseless:
        target += rng.normal(scale=np.sqrt(spec.noise_var), size=(E, 2))
        outlier = rng.uniform(size=E) < spec.outlier_frac
        n_out = int(outlier.sum())
        ang = rng.uniform(0.0, 2 * np.pi, size=n_out)
        mag = rng.uniform(5.0, 30.0, size=n_out)
        target[outlier] += mag[:, None] * np.stack([np.cos(ang), np.sin(ang)], axis=1)
        weight = rng.uniform(0.0, 1.0, size=(E, 2))
        if not spec.outlier_weights_uniform:
            weight[outlier] = rng.uniform(0.0, 0.05, size=(n_out, 2))
    return target, weight, outlier


def make_scene(spec: SceneSpec, seed: int, dtype=np.float32) -> Scene:
    """Draw one scene; arrays are float32 unless ``dtype`` asks otherwise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n, ppf = spec.n_frames, spec.patches_per_frame
    rots_cw, centres = _trajectory(rng, n)
    # world->camera: R = R_cw^T, t = -R_cw^T c
    R_cw = np.stack([r.as_matrix() for r in rots_cw])
    R_wc = np.transpose(R_cw, (0, 2, 1))
    t_wc = -np.einsum('nab,nb->na', R_wc, centres)

    xs = np.empty((n, ppf)); ys = np.empty((n, ppf)); zs = np.empty((n, ppf))
    for i in range(n):
        frames = _frames_of(i, n, spec.radius)
        todo = np.arange(ppf)
        for _attempt in range(1000):
            m = todo.shape[0]
            x = rng.uniform(0.0, WIDTH, size=m)
            y = rng.uniform(0.0, HEIGHT, size=m)
            z = rng.uniform(1.0, 10.0, size=m)
            pc = z[:, None] * np.stack([(x - CX) / FX, (y - CY) / FY, np.ones(m)], axis=1)
            pw = pc @ R_cw[i].T + centres[i]
            zj = np.einsum('fb,mb->mf', R_wc[frames, 2, :], pw) + t_wc[frames, 2][None, :]
            ok = np.all(zj / z[:, None] >= 0.5, axis=1)
            xs[i, todo[ok]] = x[ok]; ys[i, todo[ok]] = y[ok]; zs[i, todo[ok]] = z[ok]
            todo = todo[~ok]
            if todo.shape[0] == 0:
                break
        else:
            raise RuntimeError("could not place patches in front of every connected frame")
    xs, ys, zs = xs.reshape(-1), ys.reshape(-1), zs.reshape(-1)
    anchor = np.repeat(np.arange(n), ppf)
    P = xs.shape[0]
    near = np.zeros(P, dtype=bool)
    zs_regular = zs.copy()
    if spec.near_frac > 0:
        nrng = np.random.Generator(np.random.PCG64(seed ^ 0x4EA2))
        near = nrng.uniform(size=P) < spec.near_frac
        zs[near] = nrng.uniform(0.15, 0.4, size=int(near.sum()))

    kk_list, jj_list = [], []
    for i in range(n):
        frames = _frames_of(i, n, spec.radius)
        ks = np.arange(i * ppf, (i + 1) * ppf)
        kk_list.append(np.repeat(ks, frames.shape[0]))
        jj_list.append(np.tile(frames, ppf))
    kk = np.concatenate(kk_list)
    jj = np.concatenate(jj_list)
    if near.any():
        # homogeneous depth of each edge at the true state: depth in frame j over depth in the source frame
        def hom_depth():
            pc = zs[:, None] * np.stack([(xs - CX) / FX, (ys - CY) / FY, np.ones(P)], axis=1)
            pw = np.einsum('pab,pb->pa', R_cw[anchor], pc) + centres[anchor]
            zj = np.einsum('eb,eb->e', R_wc[jj, 2, :], pw[kk]) + t_wc[jj, 2]
            return zj / zs[kk]
        # a near patch keeps its place only if at least 4 edges to other frames
        # stay clearly active (its inverse depth then stays well determined)
        zh = hom_depth()
        n_act = np.zeros(P, np.int64)
        np.add.at(n_act, kk, ((zh >= 0.5) & (jj != anchor[kk])).astype(np.int64))
        weak = near & (n_act < 4)
        zs[weak] = zs_regular[weak]
        near &= ~weak
        zh = hom_depth()
        keep = ~near[kk] | (zh >= 0.5) | (zh <= -0.5)
        kk, jj = kk[keep], jj[keep]
    E = kk.shape[0]

    # render the true measurement of every edge with a world-point pinhole camera
    pc = zs[:, None] * np.stack([(xs - CX) / FX, (ys - CY) / FY, np.ones(P)], axis=1)
    pw = np.einsum('pab,pb->pa', R_cw[anchor], pc) + centres[anchor]
    cam = np.einsum('eab,eb->ea', R_wc[jj], pw[kk]) + t_wc[jj]
    uv_true = np.stack([FX * cam[:, 0] / cam[:, 2] + CX, FY * cam[:, 1] / cam[:, 2] + CY], axis=1)

    target, weight, outlier = _draw_factors(rng, spec, uv_true, E)

    poses_gt = np.stack([_pack(rots_cw[i].inv(), t_wc[i]) for i in range(n)])
    poses = poses_gt.copy()
    for i in range(spec.t0, n):
        axis = _unit(rng.normal(size=3))
        dr = Rotation.from_rotvec(axis * np.deg2rad(spec.init_rot_deg))
        dt = spec.init_trans * _unit(rng.normal(size=3))
        poses[i] = _pack(dr * rots_cw[i].inv(), dr.apply(t_wc[i]) + dt)
    scale = rng.uniform(0.8, 1.2, size=P)

    f32 = dtype
    invd = 1.0 / zs
    return Scene(
        spec=spec, seed=seed,
        intrinsics=np.array([FX, FY, CX, CY], dtype=f32),
        poses=poses.astype(f32),
        patches=np.stack([xs, ys, invd * scale], axis=1).astype(f32),
        anchor=anchor.astype(np.int32),
        kk=kk.astype(np.int32), jj=jj.astype(np.int32),
        target=target.astype(f32), weight=weight.astype(f32),
        poses_gt=poses_gt.astype(f32), depth_gt=invd.astype(f32),
        outlier=outlier, uv_true=uv_true,
    )


def make_batch(spec: SceneSpec, count: int, base_seed: int = 0):
    return [make_scene(spec, base_seed + b) for b in range(count)]


def make_serving_mix(count: int, base_seed: int = 0):
    """Sessions of the serving workload, each with its own shape and seed."""
    rng = np.random.Generator(np.random.PCG64(base_seed ^ 0x5EED))
    return [make_scene(serving_spec(rng), base_seed + 1000 + s) for s in range(count)]


def refresh_factors(scene: Scene, seed: int) -> Scene:
    """A new request on a resident session: fresh pixel noise, outliers and
    weights around the same true measurements; graph and state unchanged."""
    rng = np.random.Generator(np.random.PCG64(seed))
    target, weight, outlier = _draw_factors(rng, scene.spec, scene.uv_true, scene.n_edges)
    return replace(scene, target=target.astype(np.float32),
                   weight=weight.astype(np.float32), outlier=outlier)
