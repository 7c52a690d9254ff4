"""FP64 oracle of the correlation features (Sec. 3.2 "Correlation", Eq. 4;
Appendix "Correlation Operation").
TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

For edge e = (k, j), level l (scale s_0 = 1, s_1 = the pooling factor), patch
pixel q with level-0 coordinates (x, y), and grid offsets (a, b) in 0..6:

    C[e, l, q, a, b] = < g_kq , f_lj( x / s_l + b - 3 , y / s_l + a - 3 ) >

f bilinear with pixel centres at integer coordinates and zero outside the map.
``correlation`` writes this definition out directly (every sample interpolated,
then the inner product).  ``correlation_by_volume`` is the second form the paper
names as equivalent: the full volume of integer-pixel inner products, sampled
bilinearly.  Both read the same bfloat16 values, widened exactly to FP64.
"""
from __future__ import annotations

import numpy as np


def from_bf16(u) -> np.ndarray:
    """bfloat16 bit patterns (uint16) widened exactly to float32: a bfloat16 is
    the upper half of the float32 with the same sign, exponent and leading
    mantissa bits."""
    return (np.asarray(u, np.uint16).astype(np.uint32) << 16).view(np.float32)


def _bilinear(F, x, y):
    """F [H, W, D] float64; x, y arrays of one shape S -> [*S, D]."""
    H, W = F.shape[:2]
    x0, y0 = np.floor(x), np.floor(y)
    out = np.zeros(x.shape + (F.shape[2],))
    for dy in (0, 1):
        for dx in (0, 1):
            px, py = (x0 + dx).astype(np.int64), (y0 + dy).astype(np.int64)
            w = (x - x0 if dx else 1 - (x - x0)) * (y - y0 if dy else 1 - (y - y0))
            inside = (px >= 0) & (px < W) & (py >= 0) & (py < H)
            vals = np.zeros(x.shape + (F.shape[2],))
            vals[inside] = F[py[inside], px[inside]]
            out += w[..., None] * vals
    return out


def correlation(inp, edges=None):
    """[len(edges), 2, 9, 7, 7] float64."""
    edges = np.arange(inp.n_edges) if edges is None else np.asarray(edges)
    maps = [from_bf16(inp.fmap0).astype(np.float64), from_bf16(inp.fmap1).astype(np.float64)]
    g = from_bf16(inp.gpatch).astype(np.float64)
    off = np.arange(7) - 3.0
    out = np.zeros((len(edges), 2, 9, 7, 7))
    for n, e in enumerate(edges):
        k, j = int(inp.kk[e]), int(inp.jj[e])
        for l, s in enumerate((1.0, float(inp.scale))):
            xy = inp.coords[e].astype(np.float64) / s
            X = xy[:, 0][:, None, None] + off[None, None, :]      # [9, 7 (a), 7 (b)]
            Y = xy[:, 1][:, None, None] + off[None, :, None]
            X, Y = np.broadcast_to(X, (9, 7, 7)), np.broadcast_to(Y, (9, 7, 7))
            f = _bilinear(maps[l][j], X, Y)                       # [9, 7, 7, D]
            out[n, l] = np.einsum("qabd,qd->qab", f, g[k])
    return out


def correlation_by_volume(inp, edges):
    """The same through the correlation volume V[q, py, px] = <g_kq, f_lj[py, px]>,
    sampled bilinearly at the grid positions (zero outside)."""
    maps = [from_bf16(inp.fmap0).astype(np.float64), from_bf16(inp.fmap1).astype(np.float64)]
    g = from_bf16(inp.gpatch).astype(np.float64)
    off = np.arange(7) - 3.0
    out = np.zeros((len(edges), 2, 9, 7, 7))
    for n, e in enumerate(edges):
        k, j = int(inp.kk[e]), int(inp.jj[e])
        for l, s in enumerate((1.0, float(inp.scale))):
            V = np.einsum("hwd,qd->qhw", maps[l][j], g[k])        # [9, H, W]
            xy = inp.coords[e].astype(np.float64) / s
            for q in range(9):
                X = np.broadcast_to(xy[q, 0] + off[None, :], (7, 7))
                Y = np.broadcast_to(xy[q, 1] + off[:, None], (7, 7))
                out[n, l, q] = _bilinear(V[q][:, :, None], X, Y)[..., 0]
    return out
