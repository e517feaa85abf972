"""GPU planner vs the FP64 oracle, through the C ABI.

FP64 device mode: trees equal the oracle's node for node (same counts, parent
indices, tree ids, insertion iterations; coordinates, root times and costs to
1e-9), same incumbent, history, slot states and statistics.

FP32 device mode: node-for-node equality holds until the first iteration in
which the oracle recorded a decision whose FP64 margin is below the flag
threshold (NN near-tie, admissibility boundary, check-count rounding, clearance
within 1e-5 m, ...); every path it returns satisfies the problem's invariants
re-checked by the oracle.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu


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
    "ur5e-recycling": lambda: (WL.ur5e(0)[0], dataclasses.replace(WL.ur5e(0)[1], workers=200, max_iters=6)),
    "arm7-interval": lambda: (WL.arm7(0)[0], dataclasses.replace(WL.arm7(0)[1], variant=0, workers=96,
                                                                  max_iters=5)),
    "ragged-workers": lambda: (WL.disc2d(2)[0], dataclasses.replace(WL.disc2d(2)[1], workers=1500, max_iters=4)),
    "ur5e-small-norecycling": lambda: (_small_arm()[0], dataclasses.replace(_small_arm()[1], variant=2)),
    "disc2d-norecycling": lambda: (WL.disc2d(1)[0], dataclasses.replace(WL.disc2d(1)[1], variant=2, max_iters=80,
                                                                        eta=0.05)),
}


def _compare_arena(g, r, atol, upto_iter=None):
    n = len(r.x) if upto_iter is None else int(np.sum(r.iter < upto_iter))
    if upto_iter is None:
        assert len(g["x"]) == len(r.x), (len(g["x"]), len(r.x))
    gi = g["iter"][:n]
    assert np.array_equal(g["parent"][:n], r.parent[:n])
    assert np.array_equal(gi, r.iter[:n])
    assert np.array_equal(g["tree"][:n], r.tree[:n])
    assert np.allclose(g["x"][:n], r.x[:n], rtol=0, atol=atol)
    assert np.allclose(g["troot"][:n], r.troot[:n], rtol=0, atol=atol)
    assert np.allclose(g["cost"][:n], r.cost[:n], rtol=0, atol=atol)


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_trees_match_oracle_node_for_node(case):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    ref = O.plan(prob, prm)
    P = stp.problem_from(prob, prm, precision=1)
    # A fresh plan and a replay of the captured graph both equal the oracle.
    for _ in range(2):
        out = P.plan()
        _check_fp64_plan(P, out, ref, prm, stp)
    st = out.stats
    print(case, "U=%.6f iters=%d nodes=%d ext=%d bridge=%d" % (ref.U, st["iterations"], st["nodes"],
                                                               st["edges_validated"], st["bridges_validated"]))
    P.close()


def _check_fp64_plan(P, out, ref, prm, stp):
    assert out.status == (stp.STP_OK if ref.status == 0 else stp.STP_NO_SOLUTION)
    st = out.stats
    assert st["iterations"] == ref.iters
    assert st["first_solution_iter"] == ref.first_iter
    assert st["nodes"] == ref.inserted
    assert st["edges_validated"] == ref.ext_checked
    assert st["bridges_validated"] == ref.bridge_checked
    assert st["root_checks"] == ref.root_checked
    _compare_arena(P.tree(-1), ref.fwd, 1e-9)
    for i in range(prm.n_roots):
        _compare_arena(P.tree(i), ref.seg[i], 1e-9)
    assert np.allclose(P.history(), ref.U_hist, rtol=0, atol=1e-9)
    if ref.status == 0:
        assert abs(out.U - ref.U) < 1e-9 and abs(out.C - ref.C) < 1e-9
        assert np.allclose(out.path, ref.path, rtol=0, atol=1e-9)
    if prm.variant != 0:
        sl = P.slots()
        for k in ("has_root", "active", "gen"):
            assert np.array_equal(sl[k], ref.slots[k]), k
        fin = ref.slots["has_root"] == 1
        assert np.allclose(sl["T"][fin], ref.slots["T"][fin])


def _first_flag(ref, tol=1e-5, band=1e-5):
    for k in range(ref.iters):
        if ref.margin_hist[k] < tol or ref.clear_hist[k] < band:
            return k
    return ref.iters


def _first_mismatch(P, ref, prm, atol=2e-4):
    """Earliest iteration at which the FP32 trees differ from the oracle's."""
    worst = ref.iters
    arenas = [(-1, ref.fwd)] + [(i, ref.seg[i]) for i in range(prm.n_roots)]
    for a, r in arenas:
        g = P.tree(a)
        n = min(len(g["x"]), len(r.x))
        for i in range(n):
            same = (g["parent"][i] == r.parent[i] and g["iter"][i] == r.iter[i]
                    and np.allclose(g["x"][i], r.x[i], rtol=0, atol=atol))
            if not same:
                worst = min(worst, int(min(g["iter"][i], r.iter[i])))
                break
        if len(g["x"]) != len(r.x):
            it = g["iter"][n] if len(g["x"]) > n else r.iter[n]
            worst = min(worst, int(it))
    return worst


@pytest.mark.parametrize("case", ["disc2d-interval", "ur5e-small-recycling", "ur5e-small-interval",
                                  "ur5e-recycling"])
def test_fp32_trees_match_until_first_flagged_decision(case):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    ref = O.plan(prob, prm)
    P = stp.problem_from(prob, prm, precision=0)
    out = P.plan()
    flag = _first_flag(ref)
    mism = _first_mismatch(P, ref, prm)
    print("%s: first flagged iteration %d, first FP32 mismatch %d of %d" % (case, flag, mism, ref.iters))
    assert mism >= flag
    P.close()


@pytest.mark.parametrize("case", ["disc2d-interval", "ur5e-small-recycling", "ur5e-small-interval"])
def test_fp32_paths_satisfy_invariants(case):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    P = stp.problem_from(prob, prm, precision=0)
    out = P.plan()
    assert out.status == stp.STP_OK
    d = prob.dof
    path = out.path
    assert np.allclose(path[0, :d], prob.qs, atol=1e-6) and abs(path[0, d]) < 1e-12
    assert np.allclose(path[-1, :d], prob.qg, atol=1e-6) and abs(path[-1, d] - out.U) < 1e-5
    dq = np.linalg.norm(np.diff(path[:, :d], axis=0), axis=1)
    dt = np.diff(path[:, d])
    assert np.all(dt > 0)
    assert np.all(dq <= prob.vmax * dt * (1 + 1e-4) + 1e-5)
    assert abs(dq.sum() - out.C) < 1e-3
    Lg = np.linalg.norm(prob.qg - prob.qs) / prob.vmax
    assert out.U >= Lg - 1e-5
    v, clr, _, _ = O.check_edges(prob, path[:-1, :d], path[:-1, d], path[1:, :d], path[1:, d], prm.res)
    assert np.all(v.astype(bool) | (np.abs(clr) <= 1e-5))
    assert np.all(np.diff(P.history()) <= 0)
    P.close()


def test_fp32_full_size_plan_sampled():
    """The timed UR5e configuration (W 1024, 32 iterations, root recycling with
    8 trees, FP32), checked through properties that hold at any size on sampled
    nodes: every sampled tree edge is collision-free by the FP64 oracle at the
    problem's resolution (clearance band 1e-5 m), runs forward in time within
    the velocity bound, and its child stores the parent's cost plus the edge's
    configuration distance, the parent's root time and tree id."""
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.ur5e(0)
    prm = dataclasses.replace(prm, max_iters=32)
    assert prm.workers == 1024 and prm.variant == 1 and prm.n_roots == 8
    P = stp.problem_from(prob, prm, precision=0)
    out = P.plan()
    assert out.status in (stp.STP_OK, stp.STP_NO_SOLUTION)
    st = out.stats
    assert st["iterations"] == 32 or out.status == stp.STP_OK
    d = prob.dof
    rng = np.random.default_rng(7)
    qa, ta, qb, tb = [], [], [], []
    n_total = 0
    for arena in [-1] + list(range(prm.n_roots)):
        t = P.tree(arena)
        n_total += len(t["x"])
        kids = np.flatnonzero(t["parent"] >= 0)
        if len(kids) == 0:
            continue
        pick = rng.choice(kids, size=min(len(kids), 300 if arena < 0 else 60), replace=False)
        for i in pick:
            p = t["parent"][i]
            dist = np.linalg.norm(t["x"][i, :d] - t["x"][p, :d])
            assert abs(t["cost"][i] - (t["cost"][p] + dist)) <= 1e-4 * (1 + t["cost"][i])
            assert t["troot"][i] == t["troot"][p] and t["tree"][i] == t["tree"][p]
            a, b = (p, i) if arena < 0 else (i, p)      # forward: parent earlier; backward: parent later
            qa.append(t["x"][a, :d]); ta.append(t["x"][a, d]); qb.append(t["x"][b, :d]); tb.append(t["x"][b, d])
    assert n_total > prm.workers
    qa, qb, ta, tb = map(np.asarray, (qa, qb, ta, tb))
    assert len(qa) >= 300
    dt = tb - ta
    assert np.all(dt > 0)
    assert np.all(np.linalg.norm(qb - qa, axis=1) <= prob.vmax * dt * (1 + 1e-4) + 1e-5)
    v, clr, _, _ = O.check_edges(prob, qa, ta, qb, tb, prm.res)
    bad = ~v.astype(bool) & (np.abs(clr) > 1e-5)
    assert not bad.any(), int(bad.sum())
    P.close()


def test_degenerate_queries():
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.disc2d(0)
    prob.qg = prob.qs.copy()
    P = stp.problem_from(prob, prm, precision=0)
    out = P.plan()
    assert out.status == stp.STP_OK and out.U == 0.0 and out.C == 0.0 and len(out.path) == 1
    P.close()
    prob, prm = WL.disc2d(0)
    prob.qs = prob.way[0, 0, 1:3].copy()          # start inside a disc at t = 0
    P = stp.problem_from(prob, prm, precision=0)
    out = P.plan()
    assert out.status == stp.STP_NO_SOLUTION and math.isinf(out.U)
    P.close()
    # Horizon below the travel-time bound: no iteration runs (L_g >= H).
    prob, prm = WL.disc2d(0)
    P = stp.problem_from(prob, prm, precision=0, t_max=2.0)
    out = P.plan()
    assert out.status == stp.STP_NO_SOLUTION and out.stats["iterations"] == 0
    P.close()


def test_capacity_overflow_is_reported():
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.disc2d(0)
    P = stp.problem_from(prob, prm, precision=0, capacity=8, max_iters=50)
    with pytest.raises(stp.StpError) as e:
        P.plan()
    assert e.value.status == stp.STP_ERR_CAPACITY
    P.close()


def _snapshot(P, prm, out):
    trees = [P.tree(a) for a in [-1] + list(range(prm.n_roots))]
    keys = ("iterations", "first_solution_iter", "nodes", "edges_validated", "bridges_validated", "check_points")
    return out.U, out.C, [dict((k, v.copy()) for k, v in t.items()) for t in trees], \
        tuple(out.stats[k] for k in keys), out.path.copy()


def _same(a, b):
    assert a[0] == b[0] and a[1] == b[1] and a[3] == b[3] and np.array_equal(a[4], b[4])
    for ta, tb in zip(a[2], b[2]):
        for k in ta:
            assert np.array_equal(ta[k], tb[k]), k


def test_replanning_is_deterministic():
    """FP32: the first plan, a replay of the captured graph, and a new problem
    created after the first was freed (reusing its cached device block and
    stream) give bit-identical trees, statistics and paths."""
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES["ur5e-small-recycling"]()
    P = stp.problem_from(prob, prm, precision=0)
    a = _snapshot(P, prm, P.plan())
    b = _snapshot(P, prm, P.plan())
    _same(a, b)
    P.close()
    Q = stp.problem_from(prob, prm, precision=0)
    _same(a, _snapshot(Q, prm, Q.plan()))
    Q.close()
    stp.release_cached()
    R = stp.problem_from(prob, prm, precision=0)
    _same(a, _snapshot(R, prm, R.plan()))
    R.close()


@pytest.mark.parametrize("which", ["disc", "arm"])
def test_goal_sequence_matches_oracle(which):
    """Goal sequences chained on the device (FP64) equal the oracle's chain."""
    from paper_2609_30533_gb300 import sequence as SQ
    from paper_2609_30533_gb300 import stp
    if which == "disc":
        prob, prm = WL.disc2d(0)
        prm = dataclasses.replace(prm, max_iters=150)
        goals = [np.array([0.95, 0.95]), np.array([0.1, 0.9])]
    else:
        prob, prm = WL.ur5e(0, n_obs=4, candidate=0)
        prm = dataclasses.replace(prm, workers=64, max_iters=40)
        goals = [prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4]),
                 prob.qs + np.array([0.2, 0.3, -0.2, 0.1, 0.4, -0.3])]
    st, path, visits, _ = O.plan_sequence(prob, prm, goals)
    res = SQ.plan_sequence(prob, prm, goals, precision=1)
    assert st == 0 and res.status == stp.STP_OK
    assert np.allclose(res.visits, visits, rtol=0, atol=1e-9)
    assert res.path.shape == path.shape and np.allclose(res.path, path, rtol=0, atol=1e-9)
    r32 = SQ.plan_sequence(prob, prm, goals, precision=0)
    assert r32.status == stp.STP_OK
    d = prob.dof
    v, clr, _, _ = O.check_edges(prob, r32.path[:-1, :d], r32.path[:-1, d], r32.path[1:, :d], r32.path[1:, d],
                                 prm.res)
    assert np.all(v.astype(bool) | (np.abs(clr) <= 1e-5))
