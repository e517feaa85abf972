"""Autotuner for the batched planner.

Chooses the extensions per problem (W, the Extend workers of every iteration)
and the launch shape of the batched kernels (CTAs per problem for the NN and
bridge scans and for the collision kernel) by running each candidate on a
sample of the problems and timing it with the library's CUDA events.
Candidates are ranked by solved problems (more is better), then by the median
first-solution time, then by validated edges per second.
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
    nn_ctas: int
    validate_ctas: int
    batch_ms: float
    solved: int
    p50_first_ms: float
    edges_per_s: float


@dataclasses.dataclass
class Choice:
    workers: int
    nn_ctas: int
    validate_ctas: int
    trials: List[Trial]


def _rank(t: Trial):
    p50 = t.p50_first_ms if np.isfinite(t.p50_first_ms) else 1e30
    return (-t.solved, p50, -t.edges_per_s)


def autotune(make_problems: Callable[[int], Sequence["stp.Problem"]],
             workers: Sequence[int] = (256, 512, 1024),
             nn_ctas: Sequence[int] = (4, 8, 16),
             validate_ctas: Sequence[int] = (1, 2, 4),
             iters_per_graph: int = 16) -> Choice:
    """make_problems(W) returns FP32 problems created with ext_per_iter = W."""
    trials = []
    for W in workers:
        probs = list(make_problems(W))
        for nn, vc in itertools.product(nn_ctas, validate_ctas):
            B = stp.Batch(probs, nn_ctas=nn, validate_ctas=vc, iters_per_graph=iters_per_graph)
            B.plan()                       # warm-up (graph upload, caches)
            ms, stats = B.plan()
            B.close()
            fs = [s["first_solution_ms"] for s in stats if s["first_solution_iter"] >= 0]
            edges = sum(s["edges_validated"] + s["bridges_validated"] for s in stats)
            trials.append(Trial(W, nn, vc, ms, len(fs), float(np.median(fs)) if fs else float("inf"),
                                edges / (ms * 1e-3) if ms > 0 else 0.0))
        for P in probs:
            P.close()
    best = min(trials, key=_rank)
    return Choice(best.workers, best.nn_ctas, best.validate_ctas, trials)
