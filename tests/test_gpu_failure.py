"""Failure detection without a GPU fault.

The pipelined kernels (the TF32 Schur path, both assembly kernels, the
correlation kernel) wait on mbarriers with a bounded number of polls and
report DPVO_BA_STATUS_TIMEOUT rather than hang.  Here the same bounded wait
runs on a phase that nothing completes: it must give up, report the status,
and leave the context usable.
"""
import pytest
import torch

from paper_2208_04726_b300 import ba
from paper_2208_04726_b300 import scenes as S
from tests.gpu_util import TOL_DEPTH, TOL_POSE, end_to_end_errors, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_bounded_wait_gives_up_and_reports_timeout():
    assert ba.selftest_bounded_wait(arrive=False, polls=1000) == ba.STATUS_TIMEOUT


def test_bounded_wait_returns_when_the_phase_completes():
    assert ba.selftest_bounded_wait(arrive=True, polls=1000) == 0


def test_context_stays_usable_after_a_timeout():
    assert ba.selftest_bounded_wait(arrive=False, polls=1000) == ba.STATUS_TIMEOUT
    sc = S.make_scene(S.PLAIN_N8, 80)
    s = ba.Solver()
    probs = solve_gpu(s, [sc])
    s.close()
    assert int(probs[0].status.item()) == 0
    e_pose, e_depth, _ = end_to_end_errors(sc, probs[0])
    assert e_pose < TOL_POSE and e_depth < TOL_DEPTH


def test_selftest_rejects_bad_arguments():
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = ba.load()
    assert lib.dpvo_ba_selftest_bounded_wait(st.data_ptr(), 0, 0, None) == ba.EINVAL
    assert lib.dpvo_ba_selftest_bounded_wait(None, 0, 10, None) == ba.EINVAL
