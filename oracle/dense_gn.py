"""Plain FP64 Gauss-Newton over the patch graph, solving the full dense normal
equations.  TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

What it computes (Deep Patch Visual Odometry, Sec. 3.1 "Differentiable Bundle
Adjustment", Eq. 6, with the reprojection of Eq. 2-3):

    minimise  sum_{(k,j) in E}  || target_kj - omega_ij(T, P_k) ||^2_{diag(w_kj)}

over the camera poses T (world->camera, SE(3)) and the inverse depth d_k of every
patch, the patch centre pixel (x_k, y_k) held constant.  Each iteration linearises
the residuals, forms the normal equations H dx = g with H = sum J^T W J (+ the
damping 1e-4 on the inverse-depth diagonal, Appendix "Bundle Adjustment Layer")
and g = sum J^T W r, drops the rows and columns of the fixed poses (the gauge:
only the last poses of the window are free, Sec. 3.3 "Optimization"), solves by
dense Cholesky and retracts.  Two iterations are the paper's default.

Readings of points the paper leaves open (the CUDA path takes the same ones):
* poses map world -> camera, so T_j T_i^-1 maps camera i to camera j (Eq. 2);
* pose increments are left perturbations xi = (v, w), translation first, applied
  as T <- Exp(xi) T with the SE(3) group exponential;
* residual r = target - pi(X); weights are the two components of Sigma_kj
  applied as a diagonal precision;
* damping lambda is added to the inverse-depth diagonal only;
* an edge takes part iff the homogeneous depth of the reprojected centre
  (third component of T_j T_i^-1 K^-1 P_k with the patch's inverse depth as the
  fourth) exceeds z_min; other edges contribute nothing;
* no clamping of depths after the update.

Nothing here is blocked, fused or reordered beyond that definition: the dense
Hessian is built from per-edge 13x13 blocks, the Cholesky is LAPACK's.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse

DAMPING = 1e-4
Z_MIN = 0.1


# --------------------------------------------------------------------------- SE(3)

def skew(a):
    """[a]x for a (..., 3) array."""
    a = np.asarray(a, dtype=np.float64)
    z = np.zeros(a.shape[:-1])
    return np.stack([
        np.stack([z, -a[..., 2], a[..., 1]], -1),
        np.stack([a[..., 2], z, -a[..., 0]], -1),
        np.stack([-a[..., 1], a[..., 0], z], -1),
    ], -2)


def quat_to_matrix(q):
    """Rotation matrix of the unit quaternion q = (qx, qy, qz, qw)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def matrix_to_quat(R):
    """Unit quaternion (qx, qy, qz, qw), qw >= 0, of a rotation matrix."""
    R = np.asarray(R, dtype=np.float64)
    tr = np.trace(R)
    if tr > 0:
        s = 2.0 * np.sqrt(1.0 + tr)
        q = np.array([(R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s,
                      (R[1, 0] - R[0, 1]) / s, 0.25 * s])
    else:
        a = int(np.argmax(np.diag(R)))
        b, c = (a + 1) % 3, (a + 2) % 3
        s = 2.0 * np.sqrt(1.0 + R[a, a] - R[b, b] - R[c, c])
        q = np.empty(4)
        q[a] = 0.25 * s
        q[b] = (R[b, a] + R[a, b]) / s
        q[c] = (R[c, a] + R[a, c]) / s
        q[3] = (R[c, b] - R[b, c]) / s
    q /= np.linalg.norm(q)
    return -q if q[3] < 0 else q


def pose_to_matrix(p):
    """4x4 world->camera matrix of a stored pose [tx ty tz qx qy qz qw]."""
    T = np.eye(4)
    T[:3, :3] = quat_to_matrix(p[3:7])
    T[:3, 3] = p[:3]
    return T


def matrix_to_pose(T):
    return np.concatenate([T[:3, 3], matrix_to_quat(T[:3, :3])])


def hat(xi):
    """4x4 twist matrix of xi = (v, w)."""
    M = np.zeros((4, 4))
    M[:3, :3] = skew(xi[3:6])
    M[:3, 3] = xi[0:3]
    return M


def exp_se3(xi):
    """SE(3) group exponential, taken literally as the matrix exponential of the twist."""
    return scipy.linalg.expm(hat(np.asarray(xi, dtype=np.float64)))


def adjoint(T):
    """Adjoint of T for twists ordered (v, w): Exp(Ad(T) xi) = T Exp(xi) T^-1."""
    R, t = T[..., :3, :3], T[..., :3, 3]
    A = np.zeros(T.shape[:-2] + (6, 6))
    A[..., :3, :3] = R
    A[..., :3, 3:] = skew(t) @ R
    A[..., 3:, 3:] = R
    return A


# --------------------------------------------------------------------------- problem

class Problem:
    """One bundle-adjustment problem in FP64 (inputs promoted from the float32
    arrays both paths receive)."""

    def __init__(self, poses, patches, anchor, kk, jj, target, weight, intrinsics, t0,
                 damping=DAMPING, z_min=Z_MIN):
        self.T = np.stack([pose_to_matrix(p) for p in np.asarray(poses, np.float64)])
        patches = np.asarray(patches, np.float64)
        self.x, self.y, self.d = patches[:, 0].copy(), patches[:, 1].copy(), patches[:, 2].copy()
        self.anchor = np.asarray(anchor, np.int64)
        self.kk = np.asarray(kk, np.int64)
        self.jj = np.asarray(jj, np.int64)
        self.target = np.asarray(target, np.float64)
        self.weight = np.asarray(weight, np.float64)
        self.fx, self.fy, self.cx, self.cy = (float(v) for v in intrinsics)
        self.t0 = int(t0)
        self.damping = float(damping)
        self.z_min = float(z_min)

    @classmethod
    def from_scene(cls, scene, **kw):
        return cls(scene.poses, scene.patches, scene.anchor, scene.kk, scene.jj,
                   scene.target, scene.weight, scene.intrinsics, scene.t0, **kw)

    @property
    def N(self):
        return self.T.shape[0]

    @property
    def P(self):
        return self.d.shape[0]


def reproject(prob, T, d):
    """Eq. 2: X = T_j T_i^-1 K^-1 P_k for every edge, P_k's centre taken as the
    homogeneous point (xbar, ybar, 1, d).  Returns the relative poses G (E,4,4),
    the homogeneous points X (E,4) and the pixel coordinates (E,2) after the
    division by the third component (Eq. 3 and the text after it)."""
    i = prob.anchor[prob.kk]
    j = prob.jj
    G = T[j] @ np.linalg.inv(T[i])
    Pk = np.stack([(prob.x - prob.cx) / prob.fx, (prob.y - prob.cy) / prob.fy,
                   np.ones(prob.P), d], axis=1)[prob.kk]
    X = np.einsum('eab,eb->ea', G, Pk)
    Z = X[:, 2]
    active = Z > prob.z_min
    Zs = np.where(active, Z, 1.0)
    uv = np.stack([prob.fx * X[:, 0] / Zs + prob.cx, prob.fy * X[:, 1] / Zs + prob.cy], axis=1)
    return G, X, uv, active


def residuals(prob, T, d):
    """r = target - omega_ij(T, P_k) (Eq. 6), zero on edges that take no part."""
    _, _, uv, active = reproject(prob, T, d)
    r = prob.target - uv
    r[~active] = 0.0
    return r, active


def linearize(prob, T, d):
    """Residuals and their Jacobians w.r.t. the left perturbation of pose i, of
    pose j, and the inverse depth d_k, for every edge (Eq. 6 linearised)."""
    G, X, uv, active = reproject(prob, T, d)
    r = prob.target - uv
    Z = np.where(active, X[:, 2], 1.0)
    fx, fy = prob.fx, prob.fy
    E = X.shape[0]
    # d pi / d X_xyz
    Jpi = np.zeros((E, 2, 3))
    Jpi[:, 0, 0] = fx / Z
    Jpi[:, 0, 2] = -fx * X[:, 0] / (Z * Z)
    Jpi[:, 1, 1] = fy / Z
    Jpi[:, 1, 2] = -fy * X[:, 1] / (Z * Z)
    # d X_xyz / d xi_j for the homogeneous point X = (X_xyz, W): [W I, -[X_xyz]x]
    dXj = np.concatenate([X[:, 3, None, None] * np.eye(3)[None], -skew(X[:, :3])], axis=2)
    Jj = Jpi @ dXj
    # T_i <- Exp(xi_i) T_i gives G <- G Exp(-xi_i) = Exp(-Ad(G) xi_i) G
    Ji = -Jj @ adjoint(G)
    # d X_xyz / d d = translation column of G
    Jd = np.einsum('eab,eb->ea', Jpi, G[:, :3, 3])
    off = ~active
    r[off] = 0.0
    Ji[off] = 0.0
    Jj[off] = 0.0
    Jd[off] = 0.0
    return r, Ji, Jj, Jd, active


def normal_equations(prob, T, d):
    """Full dense H (6N+P square) and g over all poses and inverse depths, with
    the damping on the inverse-depth diagonal.  Variable order: pose 0..N-1 (6
    each, (v, w)), then d_0..d_{P-1}."""
    r, Ji, Jj, Jd, active = linearize(prob, T, d)
    N, P = prob.N, prob.P
    n = 6 * N + P
    i = prob.anchor[prob.kk]
    j = prob.jj
    cols = np.concatenate([6 * i[:, None] + np.arange(6), 6 * j[:, None] + np.arange(6),
                           (6 * N + prob.kk)[:, None]], axis=1)          # (E, 13)
    J = np.concatenate([Ji, Jj, Jd[:, :, None]], axis=2)                  # (E, 2, 13)
    WJ = prob.weight[:, :, None] * J
    Hloc = np.einsum('eca,ecb->eab', J, WJ)                               # (E, 13, 13)
    gloc = np.einsum('eca,ec->ea', WJ, r)                                 # (E, 13)
    rows_idx = np.broadcast_to(cols[:, :, None], Hloc.shape).ravel()
    cols_idx = np.broadcast_to(cols[:, None, :], Hloc.shape).ravel()
    H = scipy.sparse.coo_matrix((Hloc.ravel(), (rows_idx, cols_idx)), shape=(n, n)).toarray()
    g = np.zeros(n)
    np.add.at(g, cols.ravel(), gloc.ravel())
    H[6 * N + np.arange(P), 6 * N + np.arange(P)] += prob.damping
    return H, g


def free_index(prob):
    """Indices of the free variables: poses t0..N-1, then every inverse depth."""
    N, P = prob.N, prob.P
    return np.concatenate([np.arange(6 * prob.t0, 6 * N), 6 * N + np.arange(P)])


class NotSPD(RuntimeError):
    pass


def solve_dense(H, g):
    """Solve H x = g by dense Cholesky (LAPACK potrf/potrs)."""
    try:
        c = scipy.linalg.cho_factor(H, lower=True, check_finite=True)
    except np.linalg.LinAlgError as e:
        raise NotSPD(str(e))
    return scipy.linalg.cho_solve(c, g)


def gn_step(prob, T, d):
    """One Gauss-Newton iteration from (T, d); returns (T', d', dxi, dd)."""
    H, g = normal_equations(prob, T, d)
    idx = free_index(prob)
    dx = solve_dense(H[np.ix_(idx, idx)], g[idx])
    nf = prob.N - prob.t0
    dxi = dx[:6 * nf].reshape(nf, 6)
    dd = dx[6 * nf:]
    T_new = T.copy()
    for a in range(nf):
        T_new[prob.t0 + a] = exp_se3(dxi[a]) @ T[prob.t0 + a]
    return T_new, d + dd, dxi, dd


def solve(prob, n_iters=2):
    """Run n_iters Gauss-Newton iterations from the problem's initial state.

    Returns a dict with per-iteration pose increments ``dxi`` (list of
    (N - t0, 6)), inverse-depth increments ``dd`` (list of (P,)), the final
    ``T`` (N,4,4), ``poses`` (N,7) and ``depths`` (P,)."""
    T, d = prob.T.copy(), prob.d.copy()
    out = {"dxi": [], "dd": []}
    for _ in range(n_iters):
        T, d, dxi, dd = gn_step(prob, T, d)
        out["dxi"].append(dxi)
        out["dd"].append(dd)
    out["T"] = T
    out["poses"] = np.stack([matrix_to_pose(t) for t in T])
    out["depths"] = d
    return out


def solve_scene(scene, n_iters=None, **kw):
    prob = Problem.from_scene(scene, **kw)
    return solve(prob, scene.n_iters if n_iters is None else n_iters)


def cost(prob, T, d):
    """Value of the Eq. 6 objective at (T, d)."""
    r, _ = residuals(prob, T, d)
    return float(np.sum(prob.weight * r * r))
