"""Failure detection without a GPU fault: every wait of the library's kernels is bounded and
reports GBPCG_TIMEOUT to the host instead of hanging.  The self-test runs that wait on an
mbarrier nobody arrives at (a short poll limit), checks the reported status and that the
context stays usable.  Faults are injected on the host only (NaN weights and sign-flipped
networks are in test_gpu_fcg.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_23343_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(gpu_lib):
    st, _ = gpu_lib.wait_selftest(True, 1 << 10)
    assert st == gpu_lib.OK
    st1, ms1 = gpu_lib.wait_selftest(False, 1 << 12)
    st2, ms2 = gpu_lib.wait_selftest(False, 1 << 15)
    assert st1 == gpu_lib.TIMEOUT and st2 == gpu_lib.TIMEOUT
    assert "bounded wait" in gpu_lib.last_error()
    assert ms2 > ms1  # the wait gives up after its polls, not earlier
    print(f"2^15 polls: {ms2:.3f} ms; the production limit of 2^18 polls ~ {ms2 * 8 / 1e3:.2f} s")
    st3, ms3 = gpu_lib.wait_selftest(False, 1 << 18)  # the production limit itself
    assert st3 == gpu_lib.TIMEOUT and 0.05e3 <= ms3 <= 5e3
    # the context is still usable: a solve right after succeeds
    b = inputs.poisson_problem(32, 0)
    x, res = gpu_lib.pcg_solve(torch.from_numpy(b).cuda(), tol=1e-6, maxit=2000)
    assert res["status"] == gpu_lib.OK
    assert oracle.true_relres(b.astype(np.float64), x.cpu().double().numpy()) <= 1e-6


def test_selftest_argument_checks(gpu_lib):
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.wait_selftest(False, 0)
    with pytest.raises(gpu_lib.GbpcgError):
        gpu_lib.wait_selftest(False, (1 << 18) + 1)
