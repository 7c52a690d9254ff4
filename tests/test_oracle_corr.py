"""Pins of the correlation oracle (Sec. 3.2, Eq. 4): integer coordinates give
plain inner products, the definition equals the correlation-volume form the
paper names as equivalent, the features are linear in the patch features, and
samples outside the map read zero.  CPU only."""
import dataclasses

import numpy as np

from oracle import corr as C
from paper_2208_04726_b300 import corr_inputs as CI


def small(seed=0, scale=2):
    return CI.make_corr_inputs(3, 4, 1, 12, 16, scale, seed)


def test_integer_coordinates_give_inner_products():
    inp = small()
    inp.coords[:] = np.round(inp.coords)
    e = 5
    out = C.correlation(inp, [e])[0]
    k, j = inp.kk[e], inp.jj[e]
    f = CI.from_bf16(inp.fmap0[j]).astype(np.float64)
    g = CI.from_bf16(inp.gpatch[k]).astype(np.float64)
    for q in range(9):
        x, y = (int(v) for v in inp.coords[e, q])
        for a in range(7):
            for b in range(7):
                py, px = y + a - 3, x + b - 3
                ref = f[py, px] @ g[q] if 0 <= py < 12 and 0 <= px < 16 else 0.0
                assert abs(out[0, q, a, b] - ref) < 1e-9


def test_definition_equals_the_correlation_volume_form():
    for scale in (2, 4):
        inp = small(1, scale)
        edges = np.arange(0, inp.n_edges, 3)
        assert np.abs(C.correlation(inp, edges) - C.correlation_by_volume(inp, edges)).max() < 1e-9


def test_linear_in_patch_features():
    """Scaling the patch features by -2 (exact in bfloat16) scales every output by -2."""
    inp = small(2)
    e = [0, 7, 11]
    a = C.correlation(inp, e)
    g2 = CI.to_bf16(-2.0 * CI.from_bf16(inp.gpatch))
    assert np.array_equal(CI.from_bf16(g2), -2.0 * CI.from_bf16(inp.gpatch))
    b = C.correlation(dataclasses.replace(inp, gpatch=g2), e)
    assert np.abs(b + 2.0 * a).max() < 1e-9


def test_far_outside_reads_zero():
    inp = small(3)
    inp.coords[:] = -100.0
    assert np.abs(C.correlation(inp, [0, 1])).max() == 0.0
