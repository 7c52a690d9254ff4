"""Seeded synthetic inputs of the correlation features (Sec. 3.2 "Correlation").

This module only draws random numbers and lays them out; it holds none of the
correlation arithmetic (no bilinear sampling, no inner products).  The paper's
inputs come from its feature network on real video (not available), so seeded
arrays of the same shapes stand in for them:

* Level-0 matching features: H0 x W0 x 128 per frame (a quarter of the image
  in each direction in the paper: 120 x 160 for 640 x 480), N(0, 1) entries
  stored as bfloat16 (round to nearest even).
* Level 1: level 0 average-pooled over s x s blocks (Sec. 3.1 builds the
  pyramid by 4 x 4 average pooling with stride 4), stored as bfloat16.
* Patch features: 3 x 3 pixels x 128 per patch, N(0, 1), bfloat16; pixel
  q = 3 u + v for row u and column v of the patch.
* Patch graph: ``patches_per_frame`` patches per frame; patch k from frame i
  has an edge to every frame j with |i - j| <= radius, grouped by patch.
* Reprojected pixel coordinates (level-0 pixels, (x, y)): a patch centre
  uniform in the map, moved per edge by N(0, (0.5 + 0.5 |i - j|)^2) pixels;
  the 3 x 3 pattern about it scaled by U[0.8, 1.25], turned by U[-0.15, 0.15]
  rad, plus N(0, 0.05^2) per coordinate.  A fraction ``wide_frac`` of the edges
  spread the pattern by U[3, 4] instead (their windows are far apart).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DIM = 128


def to_bf16(x) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def from_bf16(u) -> np.ndarray:
    return (np.asarray(u, np.uint16).astype(np.uint32) << 16).view(np.float32)


@dataclass
class CorrInputs:
    n_frames: int
    n_patches: int
    n_edges: int
    height: int
    width: int
    scale: int
    fmap0: np.ndarray     # [N, H0, W0, 128] uint16 (bfloat16 bits)
    fmap1: np.ndarray     # [N, H1, W1, 128] uint16
    gpatch: np.ndarray    # [P, 9, 128] uint16
    kk: np.ndarray        # [E] int32
    jj: np.ndarray        # [E] int32
    coords: np.ndarray    # [E, 9, 2] float32


def make_corr_inputs(n_frames, patches_per_frame, radius, height, width, scale, seed, wide_frac=0.0):
    rng = np.random.default_rng(seed)
    N, P = n_frames, n_frames * patches_per_frame
    f0 = rng.standard_normal((N, height, width, DIM), dtype=np.float32)
    fmap0 = to_bf16(f0)
    H1, W1 = height // scale, width // scale
    f0b = from_bf16(fmap0)[:, :H1 * scale, :W1 * scale]
    f1 = f0b.reshape(N, H1, scale, W1, scale, DIM).mean(axis=(2, 4))
    fmap1 = to_bf16(f1)
    gpatch = to_bf16(rng.standard_normal((P, 9, DIM), dtype=np.float32))
    anchor = np.repeat(np.arange(N), patches_per_frame)
    kk, jj = [], []
    for k in range(P):
        i = anchor[k]
        for j in range(max(0, i - radius), min(N - 1, i + radius) + 1):
            kk.append(k)
            jj.append(j)
    kk, jj = np.array(kk, np.int32), np.array(jj, np.int32)
    E = len(kk)
    centre = rng.uniform([2, 2], [width - 3, height - 3], (P, 2))
    du, dv = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0], indexing="ij")   # rows u, columns v
    pattern = np.stack([dv.ravel(), du.ravel()], 1)                            # (x, y) offsets of q = 3u + v
    dist = np.abs(anchor[kk] - jj).astype(np.float64)
    c = centre[kk] + rng.standard_normal((E, 2)) * (0.5 + 0.5 * dist)[:, None]
    sc = rng.uniform(0.8, 1.25, E)
    wide = rng.random(E) < wide_frac
    sc[wide] = rng.uniform(3.0, 4.0, int(wide.sum()))
    th = rng.uniform(-0.15, 0.15, E)
    R = np.stack([np.stack([np.cos(th), -np.sin(th)], -1), np.stack([np.sin(th), np.cos(th)], -1)], -2)
    coords = c[:, None, :] + sc[:, None, None] * np.einsum("eij,qj->eqi", R, pattern)
    coords += rng.standard_normal(coords.shape) * 0.05
    return CorrInputs(N, P, E, height, width, scale, fmap0, fmap1, gpatch, kk, jj, coords.astype(np.float32))
