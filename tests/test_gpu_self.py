"""Arm self-collision on the GPU against the oracle: verdicts on random UR5e
edges (FP64 exact away from |clearance| <= 1e-9; FP32 within the clearance and
box bands), and planner trees node for node in FP64 with self-collision on."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as WL
from test_gpu_plan import _compare_arena

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


def _arm():
    prob, prm = WL.ur5e(0, n_obs=4, candidate=0)
    prob.qg = prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4])
    prob.self_collision = True
    return prob, dataclasses.replace(prm, workers=64, max_iters=30)


@pytest.mark.parametrize("precision", [1, 0])
def test_self_collision_verdicts_match_oracle(precision):
    from paper_2609_30533_gb300 import stp
    prob, prm = _arm()
    qa, ta, qb, tb = WL.microbench_edges(prob, 2000, 0.5, 15.0, seed=3)
    cast = np.float64 if precision else np.float32
    qa, ta, qb, tb = (x.astype(cast).astype(np.float64) for x in (qa, ta, qb, tb))
    rv, rclr, _, _, rbm = O.check_edges(prob, qa, ta, qb, tb, prm.res, bounds=True)
    P = stp.problem_from(prob, prm, precision=precision)
    v, _, _ = P.check_edges(qa, ta, qb, tb)
    band = 1e-9 if precision else 1e-5
    bad = (v != rv) & (np.abs(rclr) > band) & (np.abs(rbm) > (0 if precision else 1e-6))
    assert not bad.any(), int(bad.sum())
    # self-collision changes verdicts on this batch
    plain = dataclasses.replace(prob, self_collision=False)
    pv, _, _, _ = O.check_edges(plain, qa, ta, qb, tb, prm.res)
    assert (pv != rv).sum() > 100
    P.close()


def test_self_collision_fp64_trees_match_oracle():
    from paper_2609_30533_gb300 import stp
    prob, prm = _arm()
    ref = O.plan(prob, prm)
    P = stp.problem_from(prob, prm, precision=1)
    out = P.plan()
    assert ref.status == 0 and out.status == stp.STP_OK
    assert out.stats["nodes"] == ref.inserted
    _compare_arena(P.tree(-1), ref.fwd, 1e-9)
    for i in range(prm.n_roots):
        _compare_arena(P.tree(i), ref.seg[i], 1e-9)
    assert abs(out.U - ref.U) < 1e-9
    P.close()
