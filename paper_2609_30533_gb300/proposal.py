"""Learned proposal pipeline: training data from plain plans, training of the
proposal network on the tensor cores, and installation of its proposals into
problems for the learned sampling branch.

Every step runs in the library: plans (stp_batch_plan), problem summaries
(stp_problem_features), path targets (stp_problem_targets, a device kernel),
forward / backward / Adam (stp_mlp_*), proposal tables (stp_set_proposal).
This module only moves arrays between those calls.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Sequence, Tuple

import numpy as np

from . import stp


@dataclasses.dataclass
class Outcome:
    """Per-problem result of one batched plan."""
    solved: np.ndarray        # bool [n]
    first_ms: np.ndarray      # first-solution time from the batch start (inf if unsolved)
    first_iter: np.ndarray    # int, -1 if unsolved
    U: np.ndarray             # arrival time (inf if unsolved)
    batch_ms: float


def plan_batch(problems: Sequence["stp.Problem"], nn_ctas=4, validate_ctas=8, iters_per_graph=16,
               launch_mode=stp.STP_LAUNCH_STEPS, team_ctas=0) -> Outcome:
    """Plan the problems as one batch. The default launch form is the per-step
    kernels: at the hundreds to thousands of problems planned here they finish
    the batch sooner than the persistent work queue, and every problem starts
    at the batch's start, so first-solution times are not queue positions."""
    B = stp.Batch(problems, nn_ctas=nn_ctas, validate_ctas=validate_ctas, iters_per_graph=iters_per_graph,
                  launch_mode=launch_mode, team_ctas=team_ctas)
    ms, stats = B.plan()
    B.close()
    fi = np.array([s["first_solution_iter"] for s in stats])
    solved = fi >= 0
    fm = np.array([s["first_solution_ms"] if ok else np.inf for s, ok in zip(stats, solved)])
    U = np.array([s["U"] if ok else np.inf for s, ok in zip(stats, solved)])
    return Outcome(solved, fm, fi, U, ms)


def collect(problems: Sequence["stp.Problem"], outcome: Outcome) -> Tuple[np.ndarray, np.ndarray]:
    """Features and path targets of the solved problems of a finished plan."""
    X, T = [], []
    for P, ok in zip(problems, outcome.solved):
        if not ok:
            continue
        t = P.targets()
        if t is None:
            continue
        X.append(P.features())
        T.append(t)
    return (np.array(X, dtype=np.float32).reshape(-1, stp.MLP_IN),
            np.array(T, dtype=np.float32).reshape(-1, stp.MLP_NTGT))


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (flat)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in stp._MLP_SHAPES:
        if name.startswith("W"):
            lim = 1.0 / np.sqrt(shape[1])
            w = rng.uniform(-lim, lim, size=shape)
            if name == "W4":
                w[152:] = 0.0
            parts.append(w.reshape(-1))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


@dataclasses.dataclass
class TrainLog:
    losses: List[float]          # minibatch loss of every step
    val: List[Tuple[int, float]]  # (step, validation loss)
    best_step: int
    best_val: float


def train(net: "stp.Mlp", X: np.ndarray, T: np.ndarray, steps: int, batch: int, lr: float, seed: int = 0,
          val_frac: float = 0.15, eval_every: int = 25) -> TrainLog:
    """Adam steps on minibatches drawn with replacement from a training split;
    the parameters with the lowest loss on the held-back validation split
    (checked every eval_every steps) are restored at the end."""
    rng = np.random.default_rng(seed)
    n = len(X)
    perm = rng.permutation(n)
    nv = int(round(val_frac * n)) if n >= 8 else 0
    vi, ti = perm[:nv], perm[nv:]
    Xt, Tt = X[ti], T[ti]
    b = min(batch, len(ti))
    losses, val = [], []
    best = (0, loss(net, X[vi], T[vi]) if nv else float("inf"), net.get_params())
    val.append((0, best[1]))
    for k in range(1, steps + 1):
        idx = rng.integers(0, len(ti), size=b)
        losses.append(net.train_step(Xt[idx], Tt[idx], lr))
        if nv and (k % eval_every == 0 or k == steps):
            v = loss(net, X[vi], T[vi])
            val.append((k, v))
            if v < best[1]:
                best = (k, v, net.get_params())
    if nv:
        net.set_params(best[2])
    return TrainLog(losses, val, best[0], best[1])


def loss(net: "stp.Mlp", X: np.ndarray, T: np.ndarray) -> float:
    """Mean loss of the network on a set (no update)."""
    tot, n = 0.0, 0
    for i in range(0, len(X), net.max_batch):
        l, _ = net.gradients(X[i:i + net.max_batch], T[i:i + net.max_batch])
        k = len(X[i:i + net.max_batch])
        tot += l * k
        n += k
    return tot / max(n, 1)


def install(net: "stp.Mlp", problems: Sequence["stp.Problem"]) -> np.ndarray:
    """Network proposals for every problem (one forward pass per max_batch)."""
    X = np.array([P.features() for P in problems], dtype=np.float32)
    Y = np.concatenate([net.forward(X[i:i + net.max_batch]) for i in range(0, len(X), net.max_batch)])
    for P, y in zip(problems, Y):
        P.set_proposal(y)
    return Y
