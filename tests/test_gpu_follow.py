"""GPU planner (FP32 and FP64) against the FP64 oracle in follow mode, through
the C ABI.

The device records one decision record per worker and iteration
(stp_set_trace). The oracle replays the same batch-synchronous run
(Algorithms 1-3) and, wherever its FP64 margin of a decision lies below the
flag threshold (NN near-tie, admissibility or horizon boundary, check-count
rounding, clearance within 1e-5 m of contact, interval emptiness, bridge rank,
improvement or publish near-tie), adopts the device's recorded choice; any
other difference is an unflagged mismatch. The tests require:

* zero unflagged mismatches over every iteration of the run;
* trees equal node for node (counts, parent indices, insertion iterations,
  tree ids exactly; coordinates, root times and costs within the FP32 bound
  below), statistics and U history equal;
* FP64 device mode: no flagged decision differs either (the device computes
  what the oracle computes).

This covers the timed configuration (UR5e, W 1024, 32 iterations, root
recycling with 8 trees), the 7-DoF configuration at W 4096 (root recycling
with 16 trees and interval root) for its first iterations, the batched form
(each member of a mixed batch), and the learned branch.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

# FP32 coordinates: every node coordinate, time and cost comes from a chain of
# steering steps, each rounding to float32 (relative 2^-24). With the device's
# choices adopted at flagged decisions, the trees agree to within
# 1e-5 + 1e-5 |value| (observed: below 2e-7 + 1e-5 |value| on every case).
ATOL32, RTOL32 = 1e-5, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


def _small_arm(n_obs=4, workers=64, iters=30):
    prob, prm = WL.ur5e(0, n_obs=n_obs, candidate=0)
    prob.qg = prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4])
    return prob, dataclasses.replace(prm, workers=workers, max_iters=iters)


CASES = {
    "disc2d-interval": lambda: (WL.disc2d(0)[0], dataclasses.replace(WL.disc2d(0)[1], max_iters=120)),
    "disc2d-recycling": lambda: (WL.disc2d(1)[0], dataclasses.replace(WL.disc2d(1)[1], variant=1, max_iters=80,
                                                                       eta=0.05)),
    "ur5e-small-recycling": lambda: _small_arm(),
    "ur5e-small-interval": lambda: (_small_arm()[0], dataclasses.replace(_small_arm()[1], variant=0, eta=0.3)),
    "ur5e-small-norecycling": lambda: (_small_arm()[0], dataclasses.replace(_small_arm()[1], variant=2)),
    "ragged-workers": lambda: (WL.disc2d(2)[0], dataclasses.replace(WL.disc2d(2)[1], workers=1500, max_iters=4)),
}


def _arenas(P, ref, prm):
    return [(P.tree(a), ref.fwd if a < 0 else ref.seg[a]) for a in range(-1, prm.n_roots)]


def _compare_trees(P, ref, prm, atol, rtol):
    for g, r in _arenas(P, ref, prm):
        assert len(g["x"]) == len(r.x), (len(g["x"]), len(r.x))
        assert np.array_equal(g["parent"], r.parent)
        assert np.array_equal(g["iter"], r.iter)
        assert np.array_equal(g["tree"], r.tree)
        for k, rv in (("x", r.x), ("troot", r.troot), ("cost", r.cost)):
            assert np.allclose(g[k], rv, rtol=rtol, atol=atol), (k, float(np.max(np.abs(g[k] - rv))))


def follow_check(P, prob, prm, precision, proposal=None, trace_iters=None):
    """Plan (already done by the caller), read the device trace and goal grid,
    replay the oracle in follow mode, and check everything listed above.
    Returns (oracle result, device output stats, follow report)."""
    rec = P.trace()
    _, grid = P.goal_grid()
    ref = O.plan(prob, prm, proposal=proposal, follow=(rec, grid))
    f = ref.follow
    assert f["unflagged"] == [], f["unflagged"][:20]
    if precision == 1:
        assert sum(f["flagged_diff"].values()) == 0, f["flagged_diff"]
    return ref, rec, f


def _stats_equal(st, ref):
    assert st["iterations"] == ref.iters
    assert st["first_solution_iter"] == ref.first_iter
    assert st["nodes"] == ref.inserted
    assert st["edges_validated"] == ref.ext_checked
    assert st["bridges_validated"] == ref.bridge_checked
    assert st["root_checks"] == ref.root_checked


def _run(prob, prm, precision, **over):
    from paper_2609_30533_gb300 import stp
    P = stp.problem_from(prob, prm, precision=precision, **over)
    P.set_trace(prm.max_iters)
    out = P.plan()
    return P, out


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("case", list(CASES))
def test_follow_mode_matches_oracle(case, precision):
    prob, prm = CASES[case]()
    P, out = _run(prob, prm, precision)
    ref, rec, f = follow_check(P, prob, prm, precision)
    assert len(rec) == ref.iters
    _stats_equal(out.stats, ref)
    tol = (1e-9, 0.0) if precision == 1 else (ATOL32, RTOL32)
    _compare_trees(P, ref, prm, *tol)
    assert np.allclose(P.history(), ref.U_hist, rtol=0, atol=tol[0])
    print("%s fp%d: %d iterations, %d nodes compared; followed %s; differing %s" % (
        case, 64 if precision else 32, ref.iters, ref.inserted + 1,
        {k: v for k, v in f["followed"].items() if v}, {k: v for k, v in f["flagged_diff"].items() if v}))
    P.close()


def test_follow_mode_timed_configuration():
    """The timed workload: UR5e, 32 link spheres, 16 moving obstacles, W 1024,
    root recycling with 8 trees, 32 iterations, FP32."""
    prob, prm = WL.ur5e(0)
    prm = dataclasses.replace(prm, max_iters=32)
    assert prm.workers == 1024 and prm.variant == 1 and prm.n_roots == 8
    P, out = _run(prob, prm, 0)
    ref, rec, f = follow_check(P, prob, prm, 0)
    assert ref.iters == out.stats["iterations"] and ref.iters >= 1
    assert len(rec) == ref.iters
    _stats_equal(out.stats, ref)
    _compare_trees(P, ref, prm, ATOL32, RTOL32)
    assert np.allclose(P.history(), ref.U_hist, rtol=0, atol=ATOL32)
    n_nodes = sum(len(g["x"]) for g, _ in _arenas(P, ref, prm))
    print("timed config: %d iterations, %d nodes, %d extension + %d bridge edges compared; followed %s; "
          "differing %s" % (ref.iters, n_nodes, ref.ext_checked, ref.bridge_checked,
                            {k: v for k, v in f["followed"].items() if v},
                            {k: v for k, v in f["flagged_diff"].items() if v}))
    assert n_nodes > 1000
    P.close()


@pytest.mark.parametrize("variant", [1, 0])
def test_follow_mode_arm7_w4096(variant):
    """7-DoF arm (48 spheres, 64 obstacles on 8-waypoint paths, H 60 s) at
    W 4096: root recycling with 16 trees and interval root, first iterations."""
    prob, prm = WL.arm7(0, variant=variant)
    prm = dataclasses.replace(prm, workers=4096, max_iters=3 if variant == 1 else 2)
    P, out = _run(prob, prm, 0)
    ref, rec, f = follow_check(P, prob, prm, 0)
    assert len(rec) == ref.iters >= 1
    _stats_equal(out.stats, ref)
    _compare_trees(P, ref, prm, ATOL32, RTOL32)
    print("arm7 variant %d: %d iterations, %d extension edges; followed %s" % (
        variant, ref.iters, ref.ext_checked, {k: v for k, v in f["followed"].items() if v}))
    P.close()


def test_follow_mode_batched_members():
    """Every member of a mixed batch (point robot and arms, both variants)
    against the oracle: the batch kernels write the same decision records."""
    from paper_2609_30533_gb300 import stp
    cases = [CASES["disc2d-interval"](), CASES["disc2d-recycling"](), CASES["ur5e-small-recycling"](),
             CASES["ur5e-small-interval"]()]
    p, q = WL.arm7(1, variant=0)
    cases.append((p, dataclasses.replace(q, workers=128, max_iters=5)))
    probs = []
    for prob, prm in cases:
        P = stp.problem_from(prob, prm, precision=0, iters_per_graph=8)
        P.set_trace(prm.max_iters)
        probs.append(P)
    B = stp.Batch(probs, nn_ctas=4, validate_ctas=4)
    _, stats = B.plan()
    for P, (prob, prm), st in zip(probs, cases, stats):
        ref, rec, f = follow_check(P, prob, prm, 0)
        assert len(rec) == ref.iters
        _stats_equal(st, ref)
        _compare_trees(P, ref, prm, ATOL32, RTOL32)
    B.close()
    for P in probs:
        P.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_follow_mode_learned(variant):
    """Learned branch (seeded stand-in network output): FP32 trees against
    the oracle in follow mode."""
    from paper_2609_30533_gb300 import stp
    prob, prm = _small_arm(workers=128, iters=20)
    prm = dataclasses.replace(prm, variant=variant, eta=0.3 if variant == 0 else prm.eta)
    y32 = WL.random_proposal(prob, seed=11)
    P = stp.problem_from(prob, prm, precision=0, learned=1)
    P.set_proposal(y32)
    P.set_trace(prm.max_iters)
    out = P.plan()
    ref, rec, f = follow_check(P, prob, prm, 0, proposal=y32.astype(np.float64))
    _stats_equal(out.stats, ref)
    _compare_trees(P, ref, prm, ATOL32, RTOL32)
    assert np.any(rec[:, :, 0] & O.TRACE_FLAGS["learned"])
    P.close()
