"""Host logic of goal sequences on CPU (Sec. "Problem Formulation": goals
visited in order), with the library's problem replaced by a fake planner
that moves in a straight line at unit speed: each query starts at the
previous goal with the obstacles shifted by the absolute start time
(t_offset) and the remaining horizon, query i gets problem_id + i, the
segments join into one path in absolute time without repeating the junction
states, and a failing query or an exhausted horizon ends the sequence with
its status."""
import dataclasses

import numpy as np
import pytest

from paper_2609_30533_gb300 import sequence as SQ
from paper_2609_30533_gb300 import stp


@dataclasses.dataclass
class Prob:
    dof: int
    qs: np.ndarray
    qg: np.ndarray


@dataclasses.dataclass
class Params:
    H: float
    problem_id: int


def _fake(calls, fail_at=None):
    class FakeProblem:
        def __init__(self, prob, params, **over):
            self.prob, self.params, self.over = prob, params, over
            self.closed = False
            calls.append(self)

        def plan(self):
            i = len(calls) - 1
            if fail_at is not None and i == fail_at:
                return stp.PlanOutput(stp.STP_NO_SOLUTION, float("inf"), float("inf"), np.zeros((0, 3)), {})
            qs, qg = self.prob.qs, self.prob.qg
            T = float(np.linalg.norm(qg - qs))      # unit speed
            mid = 0.5 * (qs + qg)
            path = np.array([[*qs, 0.0], [*mid, 0.5 * T], [*qg, T]])
            return stp.PlanOutput(stp.STP_OK, T, T, path, {})

        def close(self):
            self.closed = True

    return lambda prob, params, **over: FakeProblem(prob, params, **over)


def test_queries_chain_in_absolute_time(monkeypatch):
    calls = []
    monkeypatch.setattr(stp, "problem_from", _fake(calls))
    prob = Prob(2, np.array([0.0, 0.0]), np.array([9.0, 9.0]))
    goals = [np.array([3.0, 4.0]), np.array([3.0, 0.0]), np.array([0.0, 0.0])]
    r = SQ.plan_sequence(prob, Params(H=20.0, problem_id=7), goals, precision=1)
    assert r.status == stp.STP_OK
    assert r.visits == pytest.approx([5.0, 9.0, 12.0])
    assert [c.over["t_offset"] for c in calls] == pytest.approx([0.0, 5.0, 9.0])
    assert [c.params.H for c in calls] == pytest.approx([20.0, 15.0, 11.0])
    assert [c.params.problem_id for c in calls] == [7, 8, 9]
    assert all(c.over["precision"] == 1 and c.closed for c in calls)
    assert np.allclose(calls[1].prob.qs, goals[0]) and np.allclose(calls[1].prob.qg, goals[1])
    # 3 states for the first segment, 2 new ones for each later segment.
    assert r.path.shape == (7, 3)
    assert np.allclose(r.path[:, 2], [0.0, 2.5, 5.0, 7.0, 9.0, 10.5, 12.0])
    assert np.allclose(r.path[-1, :2], goals[-1])
    assert np.all(np.diff(r.path[:, 2]) > 0)


def test_failing_query_ends_the_sequence(monkeypatch):
    calls = []
    monkeypatch.setattr(stp, "problem_from", _fake(calls, fail_at=1))
    prob = Prob(2, np.array([0.0, 0.0]), np.array([1.0, 0.0]))
    r = SQ.plan_sequence(prob, Params(H=50.0, problem_id=0), [np.array([3.0, 4.0]), np.array([3.0, 0.0]),
                                                             np.array([0.0, 0.0])])
    assert r.status == stp.STP_NO_SOLUTION and r.path is None
    assert len(calls) == 2 and all(c.closed for c in calls)
    assert r.visits == pytest.approx([5.0]) and len(r.queries) == 2


def test_exhausted_horizon_stops_before_planning(monkeypatch):
    calls = []
    monkeypatch.setattr(stp, "problem_from", _fake(calls))
    prob = Prob(2, np.array([0.0, 0.0]), np.array([1.0, 0.0]))
    r = SQ.plan_sequence(prob, Params(H=5.0, problem_id=0), [np.array([3.0, 4.0]), np.array([3.0, 0.0])])
    assert r.status == stp.STP_NO_SOLUTION and r.path is None
    assert len(calls) == 1 and r.visits == pytest.approx([5.0])
