"""Seeded synthetic planning problems (inputs only; none of the planner's arithmetic).

These stand in for the paper's Disc2D, Panda-spheres and Tabletop suites
(Sec. "Simulation Protocol", Table "benchmarks"), which are not available here.
Every problem is drawn from numpy's own generator with a fixed seed; the planner's
random draws (Philox4x32-10) are separate and live on each side of the
CUDA/oracle boundary.

Workloads (sizes follow the planning-problem shapes of the paper's suites):
  disc2d   2-DoF point robot in [0,1]^2, 8 discs r=0.05 at constant velocity
           U[-0.1,0.1]^2 /s, v_max 0.5, horizon 20 s, interval root N=4, W=64.
  ur5e     UR5e (standard DH), 32 link spheres r=0.05, 16 sphere obstacles r=0.06
           on 4-waypoint paths (<=0.5 m/s) in a 1.2 m cube, v_max pi/2 rad/s,
           horizon 15 s, root recycling N=8, W=1024.
  arm7     7-DoF serial arm with seeded DH (link lengths U[0.1,0.4] m), 48 link
           spheres r=0.04, 64 sphere obstacles r~U[0.04,0.1] on 8-waypoint paths,
           horizon 60 s, root recycling N=16 (or interval root), W=4096.
  mixed    problems drawn from the three families above with varied obstacle
           counts (4..128) and horizons (10..60 s).

Start/goal selection for the arms: candidates are drawn uniformly in the joint
box; the accepted candidate index per (workload, seed) is stored in
``accepted_candidates.json``, written by ``select_candidates.py`` (which decides
acceptance with the FP64 oracle: start clear at t=0 and goal clear at some time).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_ACCEPTED_PATH = os.path.join(HERE, "accepted_candidates.json")

# UR5e standard DH parameters (Universal Robots' published table):
# rows (a, alpha, d, theta_offset), metres / radians.
UR5E_DH = np.array([
    [0.0, math.pi / 2, 0.1625, 0.0],
    [-0.425, 0.0, 0.0, 0.0],
    [-0.3922, 0.0, 0.0, 0.0],
    [0.0, math.pi / 2, 0.1333, 0.0],
    [0.0, -math.pi / 2, 0.0997, 0.0],
    [0.0, 0.0, 0.0996, 0.0],
])


@dataclasses.dataclass
class Problem:
    """One planning query (Sec. "Problem Formulation")."""
    dof: int
    arm: bool
    dh: Optional[np.ndarray]      # [dof][4] (a, alpha, d, theta0) or None
    qlo: np.ndarray               # [dof]
    qhi: np.ndarray               # [dof]
    spheres: np.ndarray           # [S][5] frame index, x, y, z, r
    vmax: float
    obs_r: np.ndarray             # [M]
    way: np.ndarray               # [M][K][4] t, x, y, z
    qs: np.ndarray                # [dof]
    qg: np.ndarray                # [dof]
    name: str = ""
    self_collision: bool = False  # arms: also check the robot's own link spheres


@dataclasses.dataclass
class Params:
    """Planner settings (Sec. "Simulation Protocol" defaults p_new 0.05, p_guided 0.95)."""
    variant: int = 0              # 0 interval root, 1 root recycling
    n_roots: int = 4              # N groups / slots
    workers: int = 64             # W extensions per iteration
    max_iters: int = 2000
    eta: float = 0.1
    res: float = 0.01
    dt: float = 0.02
    p_new: float = 0.05
    p_guided: float = 0.95
    H: float = 20.0
    seed: int = 0
    problem_id: int = 0


def sphere_layout(dh: np.ndarray, n_spheres: int, radius: float) -> np.ndarray:
    """Place link spheres along each DH link (robot-model setup, not planning).

    Link j (frame j, 1-based) spans, in frame-j coordinates, the polyline
    (-a, -d sin(alpha), -d cos(alpha)) -> (-a, 0, 0) -> (0, 0, 0): the d-offset
    along the previous z axis, then the a-offset along x_j. Spheres are shared
    among links in proportion to |a| + |d| (largest remainder, at least one per
    link) and centred at equal arc-length spacing.
    """
    dof = dh.shape[0]
    lengths = np.abs(dh[:, 0]) + np.abs(dh[:, 2])
    lengths = np.maximum(lengths, 1e-6)
    counts = np.ones(dof, dtype=int)
    rest = n_spheres - dof
    share = lengths / lengths.sum() * rest
    base = np.floor(share).astype(int)
    counts += base
    left = rest - base.sum()
    order = np.argsort(-(share - base), kind="stable")
    counts[order[:left]] += 1
    out = []
    for j in range(dof):
        a, alpha, d, _ = dh[j]
        p0 = np.array([-a, -d * math.sin(alpha), -d * math.cos(alpha)])
        p1 = np.array([-a, 0.0, 0.0])
        p2 = np.zeros(3)
        l01 = np.linalg.norm(p1 - p0)
        l12 = np.linalg.norm(p2 - p1)
        total = l01 + l12
        for m in range(counts[j]):
            s = (m + 0.5) / counts[j] * total
            if s <= l01 and l01 > 0:
                c = p0 + (p1 - p0) * (s / l01)
            else:
                c = p1 + (p2 - p1) * ((s - l01) / l12 if l12 > 0 else 0.0)
            out.append([j + 1, c[0], c[1], c[2], radius])
    return np.array(out, dtype=np.float64)


def _waypoint_paths(rng, n_obs, n_way, lo, hi, H, vmax_obs, dims=3):
    """Piecewise-linear obstacle paths whose legs all respect vmax_obs.

    Waypoints are uniform in the box [lo, hi]^dims; leg durations are
    proportional to leg length and stretched over [0, H] (so every leg speed is
    total_length / H); if that exceeds vmax_obs the path is shrunk toward its
    first waypoint.
    """
    way = np.zeros((n_obs, n_way, 4))
    for m in range(n_obs):
        pts = rng.uniform(lo, hi, size=(n_way, dims))
        legs = np.linalg.norm(np.diff(pts, axis=0), axis=1)
        total = legs.sum()
        if total / H > vmax_obs:
            shrink = vmax_obs * H / total * 0.999
            pts = pts[0] + (pts - pts[0]) * shrink
            legs = legs * shrink
            total = legs.sum()
        times = np.concatenate([[0.0], np.cumsum(legs)]) / max(total, 1e-12) * H
        way[m, :, 0] = times
        way[m, :, 1:1 + dims] = pts
    return way


def _accepted(workload: str, seed: int) -> int:
    if not os.path.exists(_ACCEPTED_PATH):
        return 0
    with open(_ACCEPTED_PATH) as f:
        table = json.load(f)
    return int(table.get(workload, {}).get(str(seed), 0))


def arm_candidates(rng, dof, n):
    return rng.uniform(-math.pi, math.pi, size=(n, 2, dof))


N_CANDIDATES = 64


def disc2d(seed: int = 0, n_discs: int = 8, H: float = 20.0):
    """2-DoF point robot among discs moving at constant velocity."""
    rng = np.random.default_rng(1000 + seed)
    qs = np.array([0.05, 0.05])
    qg = np.array([0.95, 0.95])
    pos = []
    while len(pos) < n_discs:
        p = rng.uniform(0.0, 1.0, size=2)
        if np.linalg.norm(p - qs) < 0.1 or np.linalg.norm(p - qg) < 0.1:
            continue
        pos.append(p)
    pos = np.array(pos)
    vel = rng.uniform(-0.1, 0.1, size=(n_discs, 2))
    way = np.zeros((n_discs, 2, 4))
    way[:, 0, 0] = 0.0
    way[:, 0, 1:3] = pos
    way[:, 1, 0] = H
    way[:, 1, 1:3] = pos + H * vel
    prob = Problem(dof=2, arm=False, dh=None, qlo=np.zeros(2), qhi=np.ones(2),
                   spheres=np.array([[0, 0.0, 0.0, 0.0, 0.0]]), vmax=0.5,
                   obs_r=np.full(n_discs, 0.05), way=way, qs=qs, qg=qg,
                   name=f"disc2d-s{seed}")
    params = Params(variant=0, n_roots=4, workers=64, max_iters=2000, eta=0.1, res=0.01,
                    dt=0.02, H=H, seed=seed)
    return prob, params


def ur5e(seed: int = 0, n_obs: int = 16, H: float = 15.0, candidate: Optional[int] = None):
    """UR5e among sphere obstacles on 4-waypoint paths in a 1.2 m cube."""
    rng = np.random.default_rng(2000 + seed)
    spheres = sphere_layout(UR5E_DH, 32, 0.05)
    way = _waypoint_paths(rng, n_obs, 4, -0.6, 0.6, H, 0.5)
    obs_r = np.full(n_obs, 0.06)
    cands = arm_candidates(rng, 6, N_CANDIDATES)
    ci = _accepted("ur5e", seed) if candidate is None else candidate
    qs, qg = cands[ci, 0], cands[ci, 1]
    prob = Problem(dof=6, arm=True, dh=UR5E_DH.copy(), qlo=np.full(6, -math.pi),
                   qhi=np.full(6, math.pi), spheres=spheres, vmax=math.pi / 2,
                   obs_r=obs_r, way=way, qs=qs, qg=qg, name=f"ur5e-s{seed}")
    params = Params(variant=1, n_roots=8, workers=1024, max_iters=200, eta=0.5, res=0.01,
                    dt=0.02, H=H, seed=seed)
    return prob, params


def arm7_dh(rng) -> np.ndarray:
    lengths = rng.uniform(0.1, 0.4, size=7)
    dh = np.zeros((7, 4))
    dh[:, 1] = [math.pi / 2 if j % 2 == 0 else -math.pi / 2 for j in range(7)]
    dh[:, 2] = lengths
    return dh


def arm7(seed: int = 0, n_obs: int = 64, H: float = 60.0, variant: int = 1,
         candidate: Optional[int] = None, table: str = "arm7"):
    """7-DoF seeded-DH arm among 64 spheres on 8-waypoint paths."""
    rng = np.random.default_rng(3000 + seed)
    dh = arm7_dh(rng)
    spheres = sphere_layout(dh, 48, 0.04)
    way = _waypoint_paths(rng, n_obs, 8, -1.0, 1.0, H, 0.5)
    obs_r = rng.uniform(0.04, 0.1, size=n_obs)
    cands = arm_candidates(rng, 7, N_CANDIDATES)
    ci = _accepted(table, seed) if candidate is None else candidate
    qs, qg = cands[ci, 0], cands[ci, 1]
    prob = Problem(dof=7, arm=True, dh=dh, qlo=np.full(7, -math.pi), qhi=np.full(7, math.pi),
                   spheres=spheres, vmax=math.pi / 2, obs_r=obs_r, way=way, qs=qs, qg=qg,
                   name=f"arm7-s{seed}")
    params = Params(variant=variant, n_roots=16, workers=4096, max_iters=100, eta=0.5,
                    res=0.01, dt=0.02, H=H, seed=seed)
    return prob, params


# Learned-proposal study on the 7-DoF distribution: training problems use
# seeds C4_TRAIN_BASE + i, held-out problems C4_TEST_BASE + i.
C4_TRAIN_BASE, C4_TEST_BASE = 1_000_000, 2_000_000
C4_TRAIN_TABLED, C4_TEST_TABLED = 2048, 1000


def arm7_c4(split: str, i: int):
    """Problem i of the learned-proposal study ("train" or "test")."""
    base = C4_TRAIN_BASE if split == "train" else C4_TEST_BASE
    prob, params = arm7(seed=base + i, table="c4")
    params.problem_id = i
    return prob, params


def mixed(index: int):
    """One problem of the mixed batch: family by index mod 3, obstacle count in
    4..128 and horizon in 10..60 s drawn from the index."""
    rng = np.random.default_rng(4000 + index)
    family = index % 3
    H = float(rng.uniform(10.0, 60.0))
    n_obs = int(rng.integers(4, 129))
    if family == 0:
        prob, params = disc2d(seed=index, n_discs=min(n_obs, 32), H=H)
    elif family == 1:
        prob, params = ur5e(seed=index, n_obs=n_obs, H=H, candidate=_accepted("mixed", index))
    else:
        prob, params = arm7(seed=index, n_obs=n_obs, H=H, candidate=_accepted("mixed", index))
    params.problem_id = index
    prob.name = f"mixed-{index}"
    return prob, params


WORKLOADS = {"disc2d": disc2d, "ur5e": ur5e, "arm7": arm7}


def microbench_edges(prob: Problem, n_edges: int, eta: float, H: float, seed: int = 0):
    """Random space-time edges for the collision microbenchmark: start uniform
    in the joint box, a step of length eta in a random direction (components
    that would leave the box are reflected, so every step keeps length eta),
    duration D / v_max, start time uniform in [0, H - duration]."""
    rng = np.random.default_rng(5000 + seed)
    d = prob.dof
    qa = rng.uniform(prob.qlo, prob.qhi, size=(n_edges, d))
    direc = rng.normal(size=(n_edges, d))
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    step = eta * direc
    out = (qa + step > prob.qhi) | (qa + step < prob.qlo)
    step[out] = -step[out]
    qb = np.clip(qa + step, prob.qlo, prob.qhi)
    D = np.linalg.norm(qb - qa, axis=1)
    dur = D / prob.vmax
    ta = rng.uniform(0.0, 1.0, size=n_edges) * np.maximum(H - dur, 0.0)
    tb = ta + dur
    return qa, ta, qb, tb


def random_proposal(prob: Problem, seed: int = 0) -> np.ndarray:
    """A seeded stand-in for a proposal-network output y[160] (float32): random
    mixture logits, means of tau in [0.3, 0.9], log standard deviations in
    [-3, -1], and 16 small random waypoint offsets (normal, sd 0.05)."""
    rng = np.random.default_rng(seed)
    y = np.zeros(160)
    y[0:8] = rng.normal(size=8)
    y[8:16] = rng.uniform(0.3, 0.9, size=8)
    y[16:24] = rng.uniform(-3.0, -1.0, size=8)
    for i in range(16):
        f = (i + 1) / 17
        y[24 + 8 * i:24 + 8 * i + prob.dof] = rng.normal(scale=0.05, size=prob.dof)
        y[24 + 8 * i + 7] = f * 0.6
    return y.astype(np.float32)
