"""Checks that pin the oracle to something other than itself.

Each function returns an error figure (0 when the oracle is right) so that the
tests can both assert that it is small and, with a mistake planted in the
oracle, that it becomes large.  The independent pieces written here:

* ``wp_residuals``: the Eq. 6 residual written in world-point form (back-project
  the patch centre to a 3-D point in world coordinates, then move it into frame
  j) with scipy rotations, not the oracle's relative-pose / inverse-depth form;
* finite differences of residuals under left pose perturbations built from
  scipy rotations;
* a Gauss-Newton step obtained by ``numpy.linalg.lstsq`` on the whitened,
  damped, finite-difference Jacobian (no normal equations, no Cholesky);
* the minimiser of the objective found by ``scipy.optimize.least_squares``;
* the set of edges behind (or nearly behind) the camera, found from the
  world-point form's depth in frame j, and the same problem with those edges
  deleted from the graph.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize
from scipy.spatial.transform import Rotation

from oracle import dense_gn as dg
from oracle import schur


def _rt(pose):
    return Rotation.from_quat(pose[3:7]).as_matrix(), np.asarray(pose[:3], np.float64)


def wp_residuals(scene, Rs, ts, d):
    """Residual target - pixel of every edge, via world points (independent form)."""
    fx, fy, cx, cy = (float(v) for v in scene.intrinsics)
    x, y = scene.patches[:, 0].astype(np.float64), scene.patches[:, 1].astype(np.float64)
    depth = 1.0 / d
    pc = depth[:, None] * np.stack([(x - cx) / fx, (y - cy) / fy, np.ones_like(x)], 1)
    i = scene.anchor
    pw = np.einsum('pba,pb->pa', Rs[i], pc - ts[i])           # R_i^T (p_c - t_i)
    k, j = scene.kk, scene.jj
    cam = np.einsum('eab,eb->ea', Rs[j], pw[k]) + ts[j]
    uv = np.stack([fx * cam[:, 0] / cam[:, 2] + cx, fy * cam[:, 1] / cam[:, 2] + cy], 1)
    return scene.target.astype(np.float64) - uv


def _state(scene):
    Rs, ts = zip(*[_rt(p.astype(np.float64)) for p in scene.poses])
    return np.stack(Rs), np.stack(ts), scene.patches[:, 2].astype(np.float64)


def _perturbed(Rs, ts, d, var, h):
    """Apply h along free variable ``var`` = ('pose', a, m) or ('depth', k)."""
    Rs, ts, d = Rs.copy(), ts.copy(), d.copy()
    if var[0] == 'pose':
        _, a, m = var
        if m < 3:          # left translation: t <- t + h e_m
            ts[a, m] += h
        else:              # left rotation: R <- Rot(h e) R, t <- Rot(h e) t
            e = np.zeros(3); e[m - 3] = h
            Q = Rotation.from_rotvec(e).as_matrix()
            Rs[a] = Q @ Rs[a]
            ts[a] = Q @ ts[a]
    else:
        d[var[1]] += h
    return Rs, ts, d


def free_vars(scene):
    N, P, t0 = scene.n_frames, scene.n_patches, scene.t0
    return [('pose', a, m) for a in range(t0, N) for m in range(6)] + [('depth', k) for k in range(P)]


def fd_jacobian(scene, h=1e-6):
    """Central-difference Jacobian of the world-point residual w.r.t. the free
    variables, shape (2E, nfree), d(pixel)/d(var) = -d(residual)/d(var)."""
    Rs, ts, d = _state(scene)
    cols = []
    for var in free_vars(scene):
        rp = wp_residuals(scene, *_perturbed(Rs, ts, d, var, h))
        rm = wp_residuals(scene, *_perturbed(Rs, ts, d, var, -h))
        cols.append(-(rp - rm).reshape(-1) / (2 * h))
    return np.stack(cols, 1)


def jacobian_error(scene):
    """Max relative difference between the oracle's analytic per-edge Jacobians
    (scattered into the free-variable columns) and finite differences."""
    prob = dg.Problem.from_scene(scene)
    r, Ji, Jj, Jd, active = dg.linearize(prob, prob.T, prob.d)
    N, t0 = scene.n_frames, scene.t0
    nf = N - t0
    E = scene.n_edges
    Ja = np.zeros((E, 2, 6 * nf + scene.n_patches))
    i = scene.anchor[scene.kk]
    for e in range(E):
        if i[e] >= t0:
            Ja[e, :, 6 * (i[e] - t0):6 * (i[e] - t0) + 6] += Ji[e]
        if scene.jj[e] >= t0:
            Ja[e, :, 6 * (scene.jj[e] - t0):6 * (scene.jj[e] - t0) + 6] += Jj[e]
        Ja[e, :, 6 * nf + scene.kk[e]] += Jd[e]
    Ja = Ja.reshape(2 * E, -1)
    Jn = fd_jacobian(scene)
    return np.abs(Ja - Jn).max() / np.abs(Jn).max()


def residual_error(scene):
    """Oracle residual vs the independent world-point residual (max abs, px)."""
    prob = dg.Problem.from_scene(scene)
    r, active = dg.residuals(prob, prob.T, prob.d)
    r2 = wp_residuals(scene, *_state(scene))
    return np.abs(r - r2).max()


def lstsq_step(scene, damping=dg.DAMPING):
    """The Gauss-Newton increment as a damped weighted linear least-squares
    problem solved by numpy's SVD-based lstsq on finite-difference Jacobians."""
    Rs, ts, d = _state(scene)
    r = wp_residuals(scene, Rs, ts, d).reshape(-1)
    J = fd_jacobian(scene)
    sw = np.sqrt(scene.weight.astype(np.float64).reshape(-1))
    nf6 = 6 * (scene.n_frames - scene.t0)
    P = scene.n_patches
    A = np.concatenate([sw[:, None] * J, np.concatenate([np.zeros((P, nf6)), np.sqrt(damping) * np.eye(P)], 1)], 0)
    b = np.concatenate([sw * r, np.zeros(P)])
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    return x[:nf6].reshape(-1, 6), x[nf6:]


def gn_step_error(scene):
    """Relative difference between the oracle's first increment and lstsq_step."""
    out = dg.solve_scene(scene, n_iters=1)
    dxi, dd = lstsq_step(scene)
    a = np.concatenate([out["dxi"][0].ravel(), out["dd"][0]])
    b = np.concatenate([dxi.ravel(), dd])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def schur_error(scene):
    prob = dg.Problem.from_scene(scene)
    _, _, dxi, dd = dg.gn_step(prob, prob.T, prob.d)
    sxi, sdd = schur.schur_step(prob, prob.T, prob.d)
    a = np.concatenate([dxi.ravel(), dd])
    b = np.concatenate([sxi.ravel(), sdd])
    return np.linalg.norm(a - b) / np.linalg.norm(a)


def depth_only_error(scene, damping=dg.DAMPING):
    """All poses fixed: each inverse depth solves a 1-D damped weighted least
    squares, dd_k = sum w J r / (sum w J^2 + lambda), with J from finite
    differences of the world-point residual."""
    assert scene.t0 == scene.n_frames
    Rs, ts, d = _state(scene)
    r = wp_residuals(scene, Rs, ts, d)
    h = 1e-7
    jd = -(wp_residuals(scene, Rs, ts, d + h) - wp_residuals(scene, Rs, ts, d - h)) / (2 * h)  # per edge, pixel slope
    w = scene.weight.astype(np.float64)
    num = np.zeros(scene.n_patches)
    den = np.full(scene.n_patches, damping)
    np.add.at(num, scene.kk, (w * jd * r).sum(1))
    np.add.at(den, scene.kk, (w * jd * jd).sum(1))
    ref = num / den
    out = dg.solve_scene(scene, n_iters=1)
    return np.abs(out["dd"][0] - ref).max() / np.abs(ref).max()


def minimiser_error(scene, iters=25):
    """Converged oracle state vs scipy.optimize.least_squares on the
    independent world-point objective (relative, over free variables).  At a
    minimum the gradient vanishes, so the depth damping does not move it."""
    out = dg.solve_scene(scene, n_iters=iters)
    Rs0, ts0, d0 = _state(scene)
    t0, N, P = scene.t0, scene.n_frames, scene.n_patches
    sw = np.sqrt(scene.weight.astype(np.float64))

    def unpack(z):
        Rs, ts = Rs0.copy(), ts0.copy()
        for a in range(t0, N):
            o = 6 * (a - t0)
            Q = Rotation.from_rotvec(z[o + 3:o + 6]).as_matrix()
            Rs[a] = Q @ Rs0[a]
            ts[a] = Q @ ts0[a] + z[o:o + 3]
        return Rs, ts, z[6 * (N - t0):]

    def fun(z):
        return (sw * wp_residuals(scene, *unpack(z))).ravel()

    z0 = np.concatenate([np.zeros(6 * (N - t0)), d0])
    sol = scipy.optimize.least_squares(fun, z0, xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=2000)
    Rs, ts, d = unpack(sol.x)
    T_ls = np.stack([np.concatenate([ts[a], Rotation.from_matrix(Rs[a]).as_quat()]) for a in range(N)])
    T_or = out["poses"]
    sgn = np.sign((T_ls[:, 3:] * T_or[:, 3:]).sum(1))[:, None]
    T_ls[:, 3:] *= sgn
    a = np.concatenate([T_or[t0:].ravel(), out["depths"]])
    b = np.concatenate([T_ls[t0:].ravel(), d])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def textbook_exp(xi):
    """Closed-form SE(3) exponential: R = Rodrigues(w), t = V(w) v with
    V = I + (1 - cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2."""
    v, w = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = np.linalg.norm(w)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-8:
        V = np.eye(3) + 0.5 * W
    else:
        V = np.eye(3) + (1 - np.cos(th)) / th**2 * W + (th - np.sin(th)) / th**3 * (W @ W)
    return Rotation.from_rotvec(w).as_matrix(), V @ v


def update_error(scene):
    """State after one oracle iteration vs the lstsq increment applied on the
    left with the closed-form exponential (relative, free poses and depths)."""
    out = dg.solve_scene(scene, n_iters=1)
    dxi, dd = lstsq_step(scene)
    Rs, ts, d = _state(scene)
    t0 = scene.t0
    ref = []
    for a in range(t0, scene.n_frames):
        R, t = textbook_exp(dxi[a - t0])
        Rn, tn = R @ Rs[a], R @ ts[a] + t
        q = Rotation.from_matrix(Rn).as_quat()
        q *= np.sign(np.dot(q, out["poses"][a, 3:]))
        ref.append(np.concatenate([tn, q]))
    a_ = np.concatenate([out["poses"][t0:].ravel(), out["depths"]])
    b_ = np.concatenate([np.stack(ref).ravel(), d + dd])
    return np.linalg.norm(a_ - b_) / np.linalg.norm(b_ - np.concatenate([np.stack([np.concatenate([ts[a], Rotation.from_matrix(Rs[a]).as_quat()]) for a in range(t0, scene.n_frames)]).ravel(), d]))


def wp_homogeneous_depth(scene):
    """Third homogeneous coordinate of every edge's reprojected centre, in the
    world-point form: depth of the back-projected point in frame j times the
    patch's inverse depth (the point's depth in its source frame is 1 / d)."""
    Rs, ts, d = _state(scene)
    fx, fy, cx, cy = (float(v) for v in scene.intrinsics)
    x, y = scene.patches[:, 0].astype(np.float64), scene.patches[:, 1].astype(np.float64)
    pc = (1.0 / d)[:, None] * np.stack([(x - cx) / fx, (y - cy) / fy, np.ones_like(x)], 1)
    i = scene.anchor
    pw = np.einsum('pba,pb->pa', Rs[i], pc - ts[i])
    k, j = scene.kk, scene.jj
    zj = np.einsum('eb,eb->e', Rs[j][:, 2, :], pw[k]) + ts[j][:, 2]
    return zj * d[k]


def without_edges(scene, drop):
    """The scene with the edges flagged in ``drop`` deleted from the graph."""
    import dataclasses
    keep = ~np.asarray(drop, bool)
    kw = dict(kk=scene.kk[keep], jj=scene.jj[keep], target=scene.target[keep], weight=scene.weight[keep])
    if scene.outlier is not None:
        kw["outlier"] = scene.outlier[keep]
    if scene.uv_true is not None:
        kw["uv_true"] = scene.uv_true[keep]
    return dataclasses.replace(scene, **kw)


def inactive_edge_error(scene, z_min=dg.Z_MIN):
    """An edge whose reprojected homogeneous depth is at most z_min takes no part
    (the reading of Eq. 2-3's division by the third coordinate for points
    behind or next to the camera): the oracle's first increment, its normal
    equations restricted to the free variables and its cost on the scene must
    equal those of the same scene with those edges deleted.  Returns the
    largest relative difference and the number of such edges."""
    drop = wp_homogeneous_depth(scene) <= z_min
    sub = without_edges(scene, drop)
    pa, pb = dg.Problem.from_scene(scene), dg.Problem.from_scene(sub)
    Ha, ga = dg.normal_equations(pa, pa.T, pa.d)
    Hb, gb = dg.normal_equations(pb, pb.T, pb.d)
    idx = dg.free_index(pa)
    eH = np.abs(Ha[np.ix_(idx, idx)] - Hb[np.ix_(idx, idx)]).max() / np.abs(Hb[np.ix_(idx, idx)]).max()
    eg = np.abs(ga[idx] - gb[idx]).max() / np.abs(gb[idx]).max()
    oa, ob = dg.solve_scene(scene, n_iters=1), dg.solve_scene(sub, n_iters=1)
    xa = np.concatenate([oa["dxi"][0].ravel(), oa["dd"][0]])
    xb = np.concatenate([ob["dxi"][0].ravel(), ob["dd"][0]])
    ex = np.abs(xa - xb).max() / np.abs(xb).max()
    ca, cb = dg.cost(pa, pa.T, pa.d), dg.cost(pb, pb.T, pb.d)
    ec = abs(ca - cb) / cb
    return max(eH, eg, ex, ec), int(drop.sum())
