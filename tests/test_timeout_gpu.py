"""Failure detection without a GPU fault: a bounded device wait that runs out
records LU_ERR_TIMEOUT, the kernel returns, and the device keeps working."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import EPS64, factor_gpu, dev

pytestmark = pytest.mark.gpu


def test_withheld_block_times_out_and_device_stays_usable(oracle_mod):
    import torch

    import paper_1611_06365_gb300 as lu
    assert lu.lu_last_device_status(reset=True) == 0
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    rc = lu.lu_wait_selftest(5_000_000)          # 5 ms bound
    t1.record()
    torch.cuda.synchronize()
    assert rc == lu.LU_ERR_TIMEOUT
    assert t0.elapsed_time(t1) >= 4.0             # the wait really ran to its bound
    assert lu.lu_last_device_status() == 0        # the library-wide status is untouched
    assert lu.lu_get_status() == lu.LU_OK
    # the context is intact: a factorization and a solve still give the oracle's answer
    n = 300
    A = li.uniform(n, n, seed=77)
    b = li.ones_rhs(A)
    LU, ipiv, info, dA, dpiv = factor_gpu(A, "f64")
    dB = torch.from_numpy(b).to(dev()).view(1, n).clone()
    lu.lu_solve(dA, dpiv, dB, n)
    torch.cuda.synchronize()
    x = dB.view(-1).cpu().numpy()
    assert info == 0 and oracle_mod.backward_error(A, x, b) <= 10 * n * EPS64


def test_selftest_rejects_bad_bound():
    import paper_1611_06365_gb300 as lu
    assert lu.lu_wait_selftest(0) == -1


@pytest.mark.parametrize("code", [0, 1])
def test_substitution_quotient_equals_ieee_division(code):
    """The back substitution divides by u(j, j) with Markstein's correction from a
    precomputed reciprocal; over 2^24 hashed operand pairs (every exponent, both
    signs, significands near 2) it gives the IEEE quotient bit for bit."""
    import paper_1611_06365_gb300 as lu
    assert lu.lu_div_selftest(code, 1 << 24, seed=12345) == 0
