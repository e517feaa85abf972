"""Closed-form (continuous) edge validation on the GPU against the oracle:
verdicts and exact clearances on random point-robot edges among obstacles
with interior waypoints (FP64 to 1e-9, FP32 within the 1e-5 m band), and
planner trees node for node in FP64 with continuous validation."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as WL
from test_gpu_plan import CASES, _compare_arena
from test_oracle_continuous import _random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


@pytest.mark.parametrize("precision,tol", [(1, 1e-9), (0, 1e-5)])
def test_continuous_verdicts_match_oracle(precision, tol):
    from paper_2609_30533_gb300 import stp
    P, qa, ta, qb, tb = _random_case(7, n=2000)
    rv, rclr = O.check_edges_continuous(P, qa, ta, qb, tb)
    prm = WL.Params(variant=0, n_roots=2, workers=64, max_iters=1, eta=0.1, res=0.01, dt=0.02, H=12.0)
    Q = stp.problem_from(P, prm, precision=precision, continuous=1)
    cast = np.float64 if precision else np.float32
    v, clr, _ = Q.check_edges(qa.astype(cast), ta.astype(cast), qb.astype(cast), tb.astype(cast), clearance=True)
    far = np.abs(rclr) > tol
    assert np.array_equal(v[far], rv[far]), int((v[far] != rv[far]).sum())
    assert np.max(np.abs(clr - rclr)) < (1e-9 if precision else 2e-5)
    assert (v == 0).sum() > 100 and (v == 1).sum() > 100
    Q.close()


@pytest.mark.parametrize("case", ["disc2d-interval", "disc2d-recycling", "disc2d-norecycling"])
def test_continuous_fp64_trees_match_oracle(case):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    ref = O.plan(prob, prm, continuous=True)
    P = stp.problem_from(prob, prm, precision=1, continuous=1)
    out = P.plan()
    assert out.status == (stp.STP_OK if ref.status == 0 else stp.STP_NO_SOLUTION)
    assert out.stats["nodes"] == ref.inserted
    _compare_arena(P.tree(-1), ref.fwd, 1e-9)
    for i in range(prm.n_roots):
        _compare_arena(P.tree(i), ref.seg[i], 1e-9)
    if ref.status == 0:
        assert abs(out.U - ref.U) < 1e-9
    P.close()


def test_continuous_fp32_paths_are_exactly_free():
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES["disc2d-interval"]()
    P = stp.problem_from(prob, prm, precision=0, continuous=1)
    out = P.plan()
    assert out.status == stp.STP_OK
    d = prob.dof
    v, clr = O.check_edges_continuous(prob, out.path[:-1, :d], out.path[:-1, d], out.path[1:, :d], out.path[1:, d])
    assert np.all(v.astype(bool) | (np.abs(clr) <= 1e-5))
    P.close()
