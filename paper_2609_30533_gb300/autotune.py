"""Autotuner for the batched planner.

Chooses the extensions per problem (W, the Extend workers of every iteration)
and the launch form of the batch: the persistent work queue (launch_mode 0)
with its team size (CTAs per problem in flight), or the per-step kernels
(launch_mode 1) with their CTAs per problem for the NN and bridge scans and
for the collision kernel, by running each candidate on a sample of the
problems and timing it with the library's CUDA events.
Candidates are ranked by solved problems (more is better), then by the time of
the whole sample batch (throughput), then by the median first-solution time.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Callable, List, Sequence

import numpy as np

from . import stp


@dataclasses.dataclass
class Trial:
    workers: int
    launch_mode: int
    team_ctas: int
    nn_ctas: int
    validate_ctas: int
    batch_ms: float
    solved: int
    p50_first_ms: float
    edges_per_s: float


@dataclasses.dataclass
class Choice:
    workers: int
    launch_mode: int
    team_ctas: int
    nn_ctas: int
    validate_ctas: int
    trials: List[Trial]


def _rank(t: Trial):
    p50 = t.p50_first_ms if np.isfinite(t.p50_first_ms) else 1e30
    return (-t.solved, t.batch_ms, p50)


def autotune(make_problems: Callable[[int], Sequence["stp.Problem"]],
             workers: Sequence[int] = (256, 512, 1024),
             team_ctas: Sequence[int] = (4, 8, 16),
             nn_ctas: Sequence[int] = (4, 8, 16),
             validate_ctas: Sequence[int] = (1, 2, 4),
             iters_per_graph: int = 16) -> Choice:
    """make_problems(W) returns FP32 problems created with ext_per_iter = W.
    An empty team_ctas skips the persistent form, an empty nn_ctas or
    validate_ctas the per-step form."""
    trials = []
    shapes = [(0, t, 0, 0) for t in team_ctas] + [(1, 0, nn, vc) for nn, vc in
                                                  itertools.product(nn_ctas, validate_ctas)]
    for W in workers:
        probs = list(make_problems(W))
        for mode, team, nn, vc in shapes:
            B = stp.Batch(probs, nn_ctas=nn, validate_ctas=vc, iters_per_graph=iters_per_graph, launch_mode=mode,
                          team_ctas=team)
            B.plan()                       # warm-up (graph upload, caches)
            ms, stats = B.plan()
            B.close()
            fs = [s["first_solution_ms"] for s in stats if s["first_solution_iter"] >= 0]
            edges = sum(s["edges_validated"] + s["bridges_validated"] for s in stats)
            trials.append(Trial(W, mode, team, nn, vc, ms, len(fs), float(np.median(fs)) if fs else float("inf"),
                                edges / (ms * 1e-3) if ms > 0 else 0.0))
        for P in probs:
            P.close()
    best = min(trials, key=_rank)
    return Choice(best.workers, best.launch_mode, best.team_ctas, best.nn_ctas, best.validate_ctas, trials)
