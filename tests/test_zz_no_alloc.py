"""The allocation-free entry point (dpvo_ba_solve_noalloc) against the regular
one (dpvo_ba_solve), through the C ABI.

dpvo_ba_solve_noalloc exists for callers that may not allocate device memory
while they run (fixed-budget embedded pipelines, processes whose device memory
belongs to another allocator, real-time loops that cannot take cudaMalloc's
synchronisation).  It keeps its workspace in one fixed device array that all
calls share, so the test makes two calls in a row on different problems and
checks that each matches the regular entry point, i.e. that nothing left in
the shared array by the first call leaks into the second.

This file is named to be collected last, so that a run that stops at the first
failure has already run every other test.
"""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from tests.gpu_util import TOL_DEPTH, TOL_POSE, err

pytestmark = pytest.mark.gpu


def _noalloc(lib, prob, stream, cfg=None):
    d = prob.dims()
    p = prob.cstruct()
    return lib.dpvo_ba_solve_noalloc(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(d),
                                     ctypes.byref(p), stream.cuda_stream)


def _update_errors(a, b, scene):
    """Relative error of a's update (final - initial) against b's."""
    t0 = scene.t0
    pa, pb = a.poses.cpu().numpy().astype(np.float64), b.poses.cpu().numpy().astype(np.float64)
    p0 = scene.poses.astype(np.float64)
    e_pose = err(pa[t0:] - p0[t0:], pb[t0:] - p0[t0:])
    da, db = a.patches[:, 2].cpu().numpy(), b.patches[:, 2].cpu().numpy()
    d0 = scene.patches[:, 2]
    e_depth = err(da.astype(np.float64) - d0, db.astype(np.float64) - d0)
    return e_pose, e_depth


@pytest.mark.parametrize("tf32", [False, True], ids=["fp32-schur", "tf32-schur"])
def test_noalloc_entry_point_matches_regular_solve_twice_in_a_row(tf32):
    """Both Schur modes (the tensor-core mode stores its Schur rows in its own
    per-chunk layout in the shared array)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lib = ba.load()
    stream = torch.cuda.current_stream()
    scenes = [S.make_scene(S.WINDOW_N22, 900), S.make_scene(dataclasses.replace(S.PLAIN_N8, t0=3), 901)]
    solver = ba.Solver(schur_tf32=tf32)
    cfg = ba.Config(1e-4, 0.1, 0, 0, 1) if tf32 else None
    try:
        for sc in scenes:
            ref = ba.problem_from_scene(sc)
            solver.solve([ref])
            got = ba.problem_from_scene(sc)
            assert _noalloc(lib, got, stream, cfg) == ba.OK
            torch.cuda.synchronize()
            assert int(got.status.item()) == int(ref.status.item()) == 0
            e_pose, e_depth = _update_errors(got, ref, sc)
            assert e_pose < TOL_POSE and e_depth < TOL_DEPTH, (e_pose, e_depth)
    finally:
        solver.close()


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lib = ba.load()
    sc = S.make_scene(S.PLAIN_N8, 902)
    prob = ba.problem_from_scene(sc)
    d = prob.dims()
    d.n_patches = 3_000_000          # workspace far beyond the fixed array; nothing is launched
    p = prob.cstruct()
    before = prob.poses.clone()
    rc = lib.dpvo_ba_solve_noalloc(None, ctypes.byref(d), ctypes.byref(p), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == ba.EINVAL
    assert torch.equal(prob.poses, before)


def test_noalloc_rejects_more_than_15_free_poses_and_leaves_the_state():
    """Beyond 15 free poses the Schur complement needs the separate assembly
    pass, which this entry point does not have: EINVAL, nothing launched."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lib = ba.load()
    sc = S.make_scene(dataclasses.replace(S.WINDOW_N22, n_frames=24, patches_per_frame=16, t0=8), 903)
    prob = ba.problem_from_scene(sc)
    before_p, before_q = prob.poses.clone(), prob.patches.clone()
    rc = _noalloc(lib, prob, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rc == ba.EINVAL
    assert torch.equal(prob.poses, before_p) and torch.equal(prob.patches, before_q)
