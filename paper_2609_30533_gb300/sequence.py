"""Goal sequences: the robot must reach q_g^1, ..., q_g^m in order (Sec.
"Problem Formulation"). With the preceding segments fixed, each goal is a
single-goal query from the previous arrival state: local time restarts at 0,
the obstacle trajectories are shifted by the query's absolute start time
(stp_params.t_offset) and the remaining horizon is the query's t_max. Every
query runs in the library (stp_create_problem / stp_plan); this module only
chains them.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from . import stp


@dataclasses.dataclass
class SequenceResult:
    status: int                  # STP_OK, or the failing query's status
    path: Optional[np.ndarray]   # [n][d+1] (q..., absolute t), None on failure
    visits: List[float]          # absolute arrival time at each reached goal
    queries: List["stp.PlanOutput"]


def plan_sequence(prob, params, goals: Sequence[np.ndarray], **over) -> SequenceResult:
    """prob / params: objects with the fields of workloads.Problem / Params
    (params.H is the sequence's horizon); goals: configurations in visit order.
    Query i uses problem_id params.problem_id + i; **over goes to every query."""
    t_abs = 0.0
    q = np.asarray(prob.qs, float)
    segs, visits, outs = [], [], []
    for i, g in enumerate(goals):
        H = params.H - t_abs
        if not H > 0:
            return SequenceResult(stp.STP_NO_SOLUTION, None, visits, outs)
        pi = dataclasses.replace(prob, qs=q.copy(), qg=np.asarray(g, float).copy())
        pr = dataclasses.replace(params, H=H, problem_id=params.problem_id + i)
        P = stp.problem_from(pi, pr, t_offset=t_abs, **over)
        try:
            out = P.plan()
        finally:
            P.close()
        outs.append(out)
        if out.status != stp.STP_OK:
            return SequenceResult(out.status, None, visits, outs)
        path = out.path.copy()
        path[:, prob.dof] += t_abs
        segs.append(path if i == 0 else path[1:])
        t_abs += out.U
        visits.append(t_abs)
        q = np.asarray(g, float)
    return SequenceResult(stp.STP_OK, np.concatenate(segs), visits, outs)
