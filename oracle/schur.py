"""FP64 Schur-complement solve of the dense normal equations.  TEST INFRASTRUCTURE
(see ``oracle/__init__.py``).

Sec. 3.1 states that the layer eliminates the inverse depths with the Schur
complement.  Because every residual involves exactly one patch, the
inverse-depth block C of the free-variable Hessian is diagonal, and

    [ B   E ] [dxi]   [v]        S = B - E C^-1 E^T,   v' = v - E C^-1 w,
    [ E^T C ] [dd ] = [w]   =>   S dxi = v',           dd = C^-1 (w - E^T dxi).

This is an exact rearrangement of the dense solve in ``dense_gn``; the tests use
it to pin that solve (equality on small graphs) and to compare the reduced pose
system (S, v') that the CUDA path factorises.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import dense_gn as dg


def blocks(prob, T, d):
    """Split the free-variable normal equations into B, E, diag(C), v, w."""
    H, g = dg.normal_equations(prob, T, d)
    idx = dg.free_index(prob)
    Hf = H[np.ix_(idx, idx)]
    gf = g[idx]
    m = 6 * (prob.N - prob.t0)
    B, E, Cblk = Hf[:m, :m], Hf[:m, m:], Hf[m:, m:]
    C = np.diag(Cblk).copy()
    off = Cblk - np.diag(C)
    if np.any(off != 0.0):
        raise AssertionError("inverse-depth block is not diagonal")
    return B, E, C, gf[:m], gf[m:]


def reduced_system(prob, T, d):
    """The reduced pose system (S, v') after eliminating every inverse depth."""
    B, E, C, v, w = blocks(prob, T, d)
    S = B - (E / C[None, :]) @ E.T
    vr = v - E @ (w / C)
    return S, vr


def schur_step(prob, T, d):
    """One Gauss-Newton increment (dxi, dd) computed through the Schur complement."""
    B, E, C, v, w = blocks(prob, T, d)
    S = B - (E / C[None, :]) @ E.T
    vr = v - E @ (w / C)
    c = scipy.linalg.cho_factor(S, lower=True)
    dxi = scipy.linalg.cho_solve(c, vr)
    dd = (w - E.T @ dxi) / C
    nf = prob.N - prob.t0
    return dxi.reshape(nf, 6), dd
