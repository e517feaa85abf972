"""Failure detection without a GPU fault: a kernel waits on an mbarrier that
nothing arrives at; its bounded wait gives up after the limit, the host reads
STP_ERR_TIMEOUT, and the context keeps working (a plan runs afterwards).
Capacity overflow and invalid arguments are covered in test_gpu_plan.py and
test_abi.py."""
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    from paper_2609_30533_gb300 import build as B
    B.build()
    from paper_2609_30533_gb300 import stp
    status, us = stp.selftest_bounded_wait(20_000_000)   # 20 ms
    assert status == stp.STP_ERR_TIMEOUT
    assert 15_000 <= us <= 2_000_000, us
    prob, prm = WL.disc2d(0)
    P = stp.problem_from(prob, prm, precision=0, max_iters=5)
    out = P.plan()
    assert out.status in (stp.STP_OK, stp.STP_NO_SOLUTION)
    P.close()
