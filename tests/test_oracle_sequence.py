"""Goal sequences in the oracle (Sec. "Problem Formulation"): each goal is a
single-goal query from the previous arrival state, local time restarting at 0,
obstacles shifted by the absolute start time, the remaining horizon. Pins: the
chained path satisfies the sequence feasibility conditions in ABSOLUTE time
(starts at (q_s, 0), visits the goals in order at the reported times, speed
bound, every edge free when checked against the unshifted obstacles), and a
query with offset tau equals the unshifted query on the problem whose obstacles
have been moved by hand."""
import dataclasses

import numpy as np

import oracle as O
import workloads as WL


def _disc_seq():
    prob, prm = WL.disc2d(0)
    prm = dataclasses.replace(prm, max_iters=150)
    goals = [np.array([0.95, 0.95]), np.array([0.1, 0.9])]
    return prob, prm, goals


def _check_sequence(prob, prm, goals, status, path, visits):
    assert status == 0
    d = prob.dof
    assert np.allclose(path[0, :d], prob.qs) and path[0, d] == 0.0
    t = path[:, d]
    assert np.all(np.diff(t) > 0)
    dq = np.linalg.norm(np.diff(path[:, :d], axis=0), axis=1)
    assert np.all(dq <= prob.vmax * np.diff(t) * (1 + 1e-9) + 1e-12)
    for g, tv in zip(goals, visits):
        i = int(np.argmin(np.abs(t - tv)))
        assert abs(t[i] - tv) < 1e-12 and np.allclose(path[i, :d], g)
    assert visits[-1] <= prm.H + 1e-12 and np.all(np.diff(visits) > 0)
    v, clr, _, _ = O.check_edges(prob, path[:-1, :d], t[:-1], path[1:, :d], t[1:], prm.res)
    assert np.all(v == 1), clr[v == 0]


def test_disc_sequence_is_feasible_in_absolute_time():
    prob, prm, goals = _disc_seq()
    status, path, visits, res = O.plan_sequence(prob, prm, goals)
    _check_sequence(prob, prm, goals, status, path, visits)
    assert len(res) == 2 and res[1].U > 0


def test_arm_sequence_is_feasible_in_absolute_time():
    prob, prm = WL.ur5e(0, n_obs=4, candidate=0)
    prm = dataclasses.replace(prm, workers=64, max_iters=40)
    goals = [prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4]),
             prob.qs + np.array([0.2, 0.3, -0.2, 0.1, 0.4, -0.3])]
    status, path, visits, _ = O.plan_sequence(prob, prm, goals)
    _check_sequence(prob, prm, goals, status, path, visits)


def test_offset_equals_hand_shifted_obstacles():
    prob, prm, _ = _disc_seq()
    tau = 3.25
    a = O.plan(prob, dataclasses.replace(prm, max_iters=40), t_offset=tau)
    moved = dataclasses.replace(prob, way=prob.way.copy())
    moved.way[:, :, 0] -= tau
    b = O.plan(moved, dataclasses.replace(prm, max_iters=40))
    assert a.status == b.status and a.inserted == b.inserted
    assert np.array_equal(a.fwd.x, b.fwd.x)
    assert (np.isinf(a.U) and np.isinf(b.U)) or a.U == b.U
