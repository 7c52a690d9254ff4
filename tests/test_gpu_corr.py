"""Correlation features (Sec. 3.2, Eq. 4) on the tensor cores through the C ABI
(dpvo_ba_correlation) against the FP64 oracle on the same bfloat16 inputs.
Tolerance: 1e-5 relative (norm over an edge set) and 1e-3 absolute per output
(FP32 accumulation of 128 bfloat16 products of unit-variance features)."""
import numpy as np
import pytest
import torch

from oracle import corr as C
from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import corr_inputs as CI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def to_dev(inp):
    bf = lambda a: torch.from_numpy(a.view(np.int16)).view(torch.bfloat16).cuda()
    return (bf(inp.fmap0), bf(inp.fmap1), bf(inp.gpatch), torch.from_numpy(inp.kk).cuda(),
            torch.from_numpy(inp.jj).cuda(), torch.from_numpy(inp.coords).cuda())


def run(inp):
    out, st = ba.correlation(*to_dev(inp), inp.scale)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), int(st.item())


def compare(got, ref):
    assert np.abs(got - ref).max() < 1e-3, np.abs(got - ref).max()
    assert np.linalg.norm(got - ref) < 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("scale,seed", [(2, 0), (4, 1)])
def test_small_problem_every_edge(scale, seed):
    inp = CI.make_corr_inputs(4, 6, 2, 24, 32, scale, seed)
    got, st = run(inp)
    assert st == 0
    compare(got, C.correlation(inp))


def test_wide_windows_use_the_cuda_core_path():
    inp = CI.make_corr_inputs(3, 5, 1, 40, 48, 4, 2, wide_frac=0.5)
    got, st = run(inp)
    assert st == 0
    compare(got, C.correlation(inp))


def test_borders_nonfinite_and_bad_indices():
    inp = CI.make_corr_inputs(3, 4, 1, 16, 20, 2, 3)
    inp.coords[0] += 40.0                      # far outside: zeros
    inp.coords[1, 4] = np.nan                  # non-finite: zeros
    inp.coords[2] -= np.array([inp.coords[2, 4, 0], inp.coords[2, 4, 1]], np.float32)   # centred on the corner
    got, st = run(inp)
    ref = C.correlation(inp)
    ref[1] = 0.0
    assert st == 0
    compare(got, ref)
    assert np.abs(got[0]).max() == 0.0 and np.abs(got[1]).max() == 0.0
    inp.kk[3] = 10_000
    got, st = run(inp)
    assert st & ba.STATUS_BAD_INPUT and np.abs(got[3]).max() == 0.0


def test_sliding_window_sized_problem_sampled():
    """22 frames of 120 x 160 x 128 features, 2112 patches, radius 13 (39,552
    edges), level 1 pooled by 4: 64 sampled edges against the oracle."""
    inp = CI.make_corr_inputs(22, 96, 13, 120, 160, 4, 4)
    assert inp.n_edges == 39552
    got, st = run(inp)
    assert st == 0
    edges = np.random.default_rng(0).choice(inp.n_edges, 64, replace=False)
    compare(got[edges], C.correlation(inp, edges))


def test_unaligned_feature_maps_are_rejected():
    """Features are read in 16-byte pieces (TMA boxes and copies): maps that
    start 8 bytes past a 16-byte boundary return EINVAL and nothing runs."""
    inp = CI.make_corr_inputs(3, 6, 1, 40, 48, 4, 5)
    args = list(to_dev(inp))
    for i in (0, 1, 2):
        shifted = list(args)
        t = args[i]
        big = torch.zeros(t.numel() + 8, dtype=t.dtype, device=t.device)
        shifted[i] = big[4:4 + t.numel()].view(t.shape)
        assert shifted[i].data_ptr() % 16 == 8
        with pytest.raises(ba.BAError) as e:
            ba.correlation(*shifted, inp.scale)
        assert e.value.code == ba.EINVAL
