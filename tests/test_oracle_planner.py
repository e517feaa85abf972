"""Oracle pins for the space-time metric, NN and the planner loops.

* The directed metric (Eq. space-time-metric) on hand-computed cases: infinite
  unless the step goes forward in sigma-time and respects v_max.
* Invariants fixed by the problem statement (Sec. "Problem Formulation") on every
  returned path: starts at (q_s, 0), ends at (q_g, U), strictly increasing time,
  speed <= v_max on every edge, U >= L_g, every edge free at resolution, C equal
  to the recomputed length, U non-increasing over iterations.
* Tree invariants from Algorithm 1 (steering fraction, rho(x_n, x_new) <= eta),
  Eq. max-speed-extension (recycling edges at exactly v_max, step <= eta),
  and the activity rules of Algorithms 2 and 3.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as WL


# --- metric and NN -----------------------------------------------------------

def test_nn_spacetime_hand_cases():
    # v_max = 1, sample x_r = ((1, 0), 2), sigma = +1.
    x = np.array([
        [0.0, 0.0, 0.0],    # D=1,   Delta=2:   admissible, rho^2 = (1+4)/2 = 2.5
        [1.0, 0.5, 1.9],    # D=0.5, Delta=0.1: too fast, infinite
        [0.5, 0.0, 1.0],    # D=0.5, Delta=1:   rho^2 = (0.25+1)/2 = 0.625  <- argmin
        [1.0, 0.0, 2.5],    # later than the sample: infinite forward
    ])
    i, rho = O.nn_spacetime(x, [1.0, 0.0], 2.0, +1, 1.0)
    assert i == 2 and abs(rho - math.sqrt(0.625)) < 1e-15
    # Backward (sigma = -1): only vertices later than the sample qualify.
    i, rho = O.nn_spacetime(x, [1.0, 0.0], 2.0, -1, 1.0)
    assert i == 3 and abs(rho - math.sqrt(0.25 / 2)) < 1e-15
    # v_max scales the time term: v = 2 makes node 1 admissible (0.5 <= 0.2? no) and
    # node 0: rho^2 = (1 + 4*4)/2 = 8.5, node 2: (0.25 + 4)/2 = 2.125.
    i, rho = O.nn_spacetime(x, [1.0, 0.0], 2.0, +1, 2.0)
    assert i == 2 and abs(rho - math.sqrt(2.125)) < 1e-15
    # Nothing admissible -> -1.
    i, rho = O.nn_spacetime(x[[1, 3]], [1.0, 0.0], 2.0, +1, 1.0)
    assert i == -1 and rho == float("inf")
    # Ties: lowest index.
    i, _ = O.nn_spacetime(np.array([[0.5, 0.0, 1.0], [0.5, 0.0, 1.0]]), [1.0, 0.0], 2.0, +1, 1.0)
    assert i == 0
    # Activity filter: troot >= U excluded.
    i, _ = O.nn_spacetime(x, [1.0, 0.0], 2.0, +1, 1.0, troot=np.array([1.0, 1.0, 5.0, 1.0]), U=5.0)
    assert i == 0


# --- planner invariants ------------------------------------------------------

def _check_path(prob, prm, r):
    d = prob.dof
    P = r.path
    assert len(P) >= 2
    assert np.allclose(P[0, :d], prob.qs) and P[0, d] == 0.0
    assert np.allclose(P[-1, :d], prob.qg) and abs(P[-1, d] - r.U) < 1e-12
    Lg = np.linalg.norm(prob.qg - prob.qs) / prob.vmax
    assert r.U >= Lg - 1e-12
    dq = np.linalg.norm(np.diff(P[:, :d], axis=0), axis=1)
    dtt = np.diff(P[:, d])
    assert np.all(dtt > 0)
    assert np.all(dq <= prob.vmax * dtt * (1 + 1e-9) + 1e-12)
    assert abs(dq.sum() - r.C) < 1e-9
    v, _, _, _ = O.check_edges(prob, P[:-1, :d], P[:-1, d], P[1:, :d], P[1:, d], prm.res)
    assert v.all()
    ok, _ = O.state_free(prob, prob.qs, 0.0)
    assert ok
    ok, _ = O.state_free(prob, prob.qg, r.U)
    assert ok


def _check_trees(prob, prm, r):
    d = prob.dof
    v = prob.vmax
    arenas = [(r.fwd, +1)] + [(s, -1) for s in r.seg]
    for A, sigma in arenas:
        for i in range(len(A.x)):
            p = A.parent[i]
            if p < 0:
                assert A.cost[i] == 0.0
                continue
            assert p < i
            dq = np.linalg.norm(A.x[i, :d] - A.x[p, :d])
            dtt = sigma * (A.x[i, d] - A.x[p, d])
            assert dtt > 0
            assert dq <= v * dtt * (1 + 1e-9) + 1e-12
            assert abs(A.cost[i] - (A.cost[p] + dq)) < 1e-9
            assert A.troot[i] == A.troot[p] and A.tree[i] == A.tree[p]
            assert 0.0 <= A.x[i, d] <= prm.H
            if prm.variant == 0:
                rho = math.sqrt((dq * dq + v * v * dtt * dtt) / 2)
                assert rho <= prm.eta * (1 + 1e-12)
            else:
                assert abs(dq - v * dtt) < 1e-9 and dq <= prm.eta * (1 + 1e-12)


@pytest.fixture(scope="module")
def disc_run():
    prob, prm = WL.disc2d(0)
    prm = dataclasses.replace(prm, max_iters=150)
    return prob, prm, O.plan(prob, prm)


def test_interval_root_path_invariants(disc_run):
    prob, prm, r = disc_run
    assert r.status == 0 and np.isfinite(r.U)
    _check_path(prob, prm, r)
    assert np.all(np.diff(r.U_hist) <= 0)
    assert r.U_hist[r.first_iter] < float("inf") and (r.first_iter == 0 or r.U_hist[r.first_iter - 1] == float("inf"))


def test_interval_root_tree_invariants(disc_run):
    prob, prm, r = disc_run
    _check_trees(prob, prm, r)


def test_interval_root_only_active_trees_grow(disc_run):
    # A node inserted in iteration k extends a tree whose root time was below the
    # incumbent at the start of k (trees rooted at T >= U are inactive).
    prob, prm, r = disc_run
    U_start = np.concatenate([[np.inf], r.U_hist])
    for s in r.seg:
        for i in range(len(s.x)):
            if s.parent[i] >= 0 and s.parent[i] < i:
                k = s.iter[i]
                root_made_now = s.iter[s.parent[i]] == k and s.parent[s.parent[i]] < 0
                if not root_made_now:
                    assert s.troot[i] < U_start[k]
    # Materialised roots are goal states at their root time.
    for s in r.seg:
        roots = s.parent < 0
        assert np.allclose(s.x[roots, :prob.dof], prob.qg)
        assert np.array_equal(s.x[roots, prob.dof], s.troot[roots])


def test_planner_is_deterministic_and_seeded(disc_run):
    prob, prm, r = disc_run
    r2 = O.plan(prob, prm)
    assert r2.U == r.U and np.array_equal(r2.fwd.x, r.fwd.x)
    r3 = O.plan(prob, dataclasses.replace(prm, seed=prm.seed + 1))
    assert len(r3.fwd.x) != len(r.fwd.x) or not np.array_equal(r3.fwd.x, r.fwd.x)


def _small_arm():
    """UR5e with four obstacles and a nearby goal: solvable in a few iterations."""
    prob, prm = WL.ur5e(0, n_obs=4, candidate=0)
    prob.qg = prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4])
    prm = dataclasses.replace(prm, workers=64, max_iters=40)
    return prob, prm


@pytest.fixture(scope="module")
def arm_run():
    prob, prm = _small_arm()
    return prob, prm, O.plan(prob, prm)


def test_root_recycling_invariants(arm_run):
    prob, prm, r = arm_run
    assert r.status == 0, "small arm case should solve"
    _check_path(prob, prm, r)
    _check_trees(prob, prm, r)
    # Slots: every slot root is a goal state at a grid time with a free goal check.
    for i, s in enumerate(r.seg):
        if r.slots["has_root"][i]:
            assert len(s.x) >= 1 and s.parent[0] == -1
            T = r.slots["T"][i]
            assert abs(T / prm.dt - round(T / prm.dt)) < 1e-9
            assert np.all(s.troot == T)
            ok, _ = O.state_free(prob, prob.qg, T)
            assert ok
            # active iff its root time is below the final incumbent
            assert bool(r.slots["active"][i]) == (T < r.U)
        # Replaced slots hold only the new generation.
        assert np.all(s.tree == r.slots["gen"][i])


def test_no_recycling_keeps_a_fixed_forest(arm_run):
    """Variant 2 (the paper's allocation ablation): the initial roots are those
    of root recycling and are never replaced; roots at T >= U turn inactive."""
    prob, prm, r1 = arm_run
    r2 = O.plan(prob, dataclasses.replace(prm, variant=2))
    assert r2.status == 0
    _check_path(prob, prm, r2)
    _check_trees(prob, prm, r2)
    assert np.all(r2.slots["gen"] == 0)
    for i in range(prm.n_roots):
        if r2.slots["has_root"][i]:
            assert bool(r2.slots["active"][i]) == (r2.slots["T"][i] < r2.U)
            assert np.all(r2.seg[i].tree == 0)
            if r1.slots["gen"][i] == 0 and r1.slots["has_root"][i]:
                assert r2.slots["T"][i] == r1.slots["T"][i]
    # recycling replaced at least one root on this case; the ablation did not
    assert np.any(r1.slots["gen"] > 0)


def test_early_return_and_blocked_start():
    prob, prm = WL.disc2d(0)
    prob.qg = prob.qs.copy()
    r = O.plan(prob, prm, max_iters=5)
    assert r.status == 0 and r.U == 0.0 and r.C == 0.0 and len(r.path) == 1
    prob, prm = WL.disc2d(0)
    prob.qs = prob.way[0, 0, 1:3].copy()     # start inside a disc at t=0
    r = O.plan(prob, prm, max_iters=5)
    assert r.status == 5 and r.iters == 0
