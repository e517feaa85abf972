"""Oracle pins for the per-worker decisions of an iteration.

Each pin is computed from the paper's definition, by hand or by brute force
over the oracle's own decision records, so that a plausible slip fails:

* Bridge rank (Algorithm 1; Sec. "Interval Root": earliest arrival first,
  the space-time metric breaks ties): hand cases where the earliest-arrival candidate
  has the larger rho, an inadmissible earlier arrival, ties on arrival broken
  by rho and on both by the lowest index; only the top candidate is validated
  (a blocked top candidate is not replaced by the runner-up); the improvement
  test (U, C) < (U0, C0).
* Publish (Sec. "GPU-Parallel Space-Time Forest"): lexicographic (U, C,
  worker) minimum of the successful bridges.
* Conditional query time (Eq. conditional-query-time): every drawn t_r lies in
  [D(q_s,q_r)/v, T - D(q_r,q_g)/v], recomputed from the Philox draws; an empty
  window skips the worker.
* Configuration-distance NN (Sec. "Practical Root Recycling"): hand cases with
  ties.
* Direction (forward iff w + k even), group draw, the new-root coin (empty
  group or u <= p_new; Algorithm 2) and the round-robin slot assignment
  (Algorithm 3) on W = 8 runs.
* Brute force over a whole interval-root run: every NN parent, bridge
  candidate, emitted bridge, bridge verdict and published winner equals the
  definition re-evaluated in numpy on the start-of-iteration trees.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as WL

F = O.TRACE_FLAGS
FLD = {n: i for i, n in enumerate(O.TRACE_FIELDS)}


def _point_problem(obstacles=(), dof=2, vmax=1.0):
    """Point robot (sphere radius 0) with static disc obstacles (r, x, y)."""
    obs = list(obstacles) or [(0.01, 50.0, 50.0)]
    way = np.zeros((len(obs), 1, 4))
    for m, (_, x, y) in enumerate(obs):
        way[m, 0] = (0.0, x, y, 0.0)
    return WL.Problem(dof=dof, arm=False, dh=None, qlo=np.full(dof, -10.0), qhi=np.full(dof, 10.0),
                      spheres=np.array([[0, 0, 0, 0, 0.0]]), vmax=vmax,
                      obs_r=np.array([r for r, _, _ in obs], dtype=float), way=way,
                      qs=np.zeros(dof), qg=np.ones(dof))


# --- bridge rank (hand cases) -------------------------------------------------

# Backward candidates seen from the forward node a = ((0, 0), t = 0), v = 1,
# rows (x, y, t), root time, cost, group.
_FWD_CANDS = [
    ((1.0, 0.0, 3.0), 9.0, 0.5, 0),   # arrival 9, rho^2 = (1 + 9) / 2 = 5
    ((0.5, 0.0, 1.0), 6.0, 0.7, 0),   # arrival 6, smallest rho: rho^2 = 0.625
    ((0.1, 0.0, 4.0), 5.0, 0.9, 1),   # arrival 5, rho^2 = (0.01 + 16) / 2 = 8.005
    ((2.0, 0.0, 2.5), 5.0, 1.5, 1),   # arrival 5, rho^2 = (4 + 6.25) / 2 = 5.125  <- winner
    ((3.0, 0.0, 2.0), 4.0, 0.1, 2),   # arrival 4 but D = 3 > v dt = 2: inadmissible
]


def _cands(rows):
    x = np.array([r[0] for r in rows], dtype=float)
    return x, np.array([r[1] for r in rows]), np.array([r[2] for r in rows]), np.array([r[3] for r in rows])


def test_bridge_rank_arrival_then_rho():
    prob = _point_problem()
    x, tr, co, sg = _cands(_FWD_CANDS)
    ok, s, i, imp, nval, U, C = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x, tr, co, sg, math.inf, math.inf,
                                        0.01)
    # Earliest admissible arrival (5) wins over the smallest rho (arrival 6);
    # between the two arrival-5 candidates the smaller rho (index 1 of group 1).
    assert (s, i) == (1, 1)
    assert U == 5.0 and abs(C - (0.0 + 2.0 + 1.5)) < 1e-15
    assert imp and nval == 1 and ok
    # Equal arrival and equal rho: the lowest (group, index).
    rows = [((2.0, 0.0, 2.5), 5.0, 1.0, 0), ((2.0, 0.0, 2.5), 5.0, 0.0, 0)]
    x2, tr2, co2, sg2 = _cands(rows)
    _, s, i, _, _, _, _ = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x2, tr2, co2, sg2, math.inf, math.inf,
                                   0.01)
    assert (s, i) == (0, 0)


def test_bridge_rank_activity_filter():
    # Trees whose root time is not below U0 are inactive: none left here.
    prob = _point_problem()
    x, tr, co, sg = _cands(_FWD_CANDS)
    ok, s, i, imp, nval, _, _ = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x, tr, co, sg, 4.0, 10.0, 0.01)
    assert (s, i) == (-1, -1) and not imp and nval == 0 and not ok
    # U0 = 5.5 keeps only the arrival-5 trees (and drops 6 and 9).
    ok, s, i, imp, nval, U, _ = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x, tr, co, sg, 5.5, 10.0, 0.01)
    assert (s, i) == (1, 1) and U == 5.0 and imp and nval == 1 and ok


def test_bridge_from_backward_node_and_improvement_rule():
    prob = _point_problem()
    # Backward node a = ((2, 0), t = 3), root time 5, cost 1; forward candidates:
    rows = [
        ((0.0, 0.0, 0.0), 0.0, 0.0, 0),   # rho^2 = (4 + 9) / 2 = 6.5
        ((1.5, 0.0, 2.0), 0.0, 1.5, 0),   # rho^2 = (0.25 + 1) / 2 = 0.625
        ((2.0, 0.4, 2.5), 0.0, 2.0, 0),   # rho^2 = (0.16 + 0.25) / 2 = 0.205  <- winner
        ((2.0, 0.0, 3.5), 0.0, 0.0, 0),   # later than a: inadmissible
        ((2.0, 0.4, 2.5), 0.0, 0.0, 0),   # ties with index 2: the lower index wins
    ]
    x, tr, co, _ = _cands(rows)
    ok, s, i, imp, nval, U, C = O.bridge(prob, [2.0, 0.0], 3.0, 5.0, 1.0, False, x, tr, co, None, math.inf,
                                        math.inf, 0.01)
    assert (s, i) == (-1, 2)
    assert U == 5.0 and abs(C - (2.0 + 0.4 + 1.0)) < 1e-12
    assert imp and nval == 1 and ok
    # (U, C) must improve lexicographically: equal U, larger C is rejected
    # without validation; equal U, smaller C is accepted.
    _, _, _, imp, nval, _, _ = O.bridge(prob, [2.0, 0.0], 3.0, 5.0, 1.0, False, x, tr, co, None, 5.0, 3.0, 0.01)
    assert not imp and nval == 0
    ok, _, _, imp, nval, _, _ = O.bridge(prob, [2.0, 0.0], 3.0, 5.0, 1.0, False, x, tr, co, None, 5.0, 3.5, 0.01)
    assert imp and nval == 1 and ok
    # A later arrival never improves.
    _, _, _, imp, nval, _, _ = O.bridge(prob, [2.0, 0.0], 3.0, 5.0, 1.0, False, x, tr, co, None, 4.9, 99.0, 0.01)
    assert not imp and nval == 0


def test_bridge_validates_only_the_top_candidate():
    # A static disc (r 0.1) at (0.5, 0) blocks the edge to the top-ranked
    # candidate (1, 0, t 1.5; arrival 3); the runner-up (0, 1, t 1.5; arrival
    # 3.5) is free but is not tried: the bridge fails with one validation.
    prob = _point_problem([(0.1, 0.5, 0.0)])
    rows = [((1.0, 0.0, 1.5), 3.0, 0.0, 0), ((0.0, 1.0, 1.5), 3.5, 0.0, 0)]
    x, tr, co, sg = _cands(rows)
    ok, s, i, imp, nval, U, _ = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x, tr, co, sg, math.inf, math.inf,
                                        0.01)
    assert (s, i) == (0, 0) and U == 3.0 and imp
    assert nval == 1 and not ok
    # Without the top candidate the runner-up is chosen and is free.
    ok, s, i, _, nval, U, _ = O.bridge(prob, [0.0, 0.0], 0.0, 0.0, 0.0, True, x[1:], tr[1:], co[1:], sg[1:],
                                       math.inf, math.inf, 0.01)
    assert (s, i) == (0, 0) and U == 3.5 and nval == 1 and ok


# --- publish -------------------------------------------------------------------

def test_publish_lexicographic_min():
    # Smallest U first, then C, then the lowest worker.
    assert O.publish_winner([5.0, 5.0, 6.0], [3.0, 2.0, 1.0], [4, 7, 1]) == 1
    assert O.publish_winner([5.0, 5.0], [2.0, 2.0], [9, 3]) == 1
    assert O.publish_winner([4.0, 4.0, 4.0], [2.0, 2.0, 1.0], [2, 1, 5]) == 2
    assert O.publish_winner([7.0, 4.0], [0.0, 9.0], [0, 1]) == 1
    assert O.publish_winner([], [], []) == -1


# --- configuration-distance NN ---------------------------------------------------

def test_nn_config_hand_cases():
    q0 = [0.0, 0.0]
    assert O.nn_config(np.array([[1, 0], [0, 1], [-1, 0]], float), q0) == (0, 1.0)        # three-way tie
    assert O.nn_config(np.array([[0, 5], [3, 4], [5, 0]], float), q0) == (0, 5.0)         # integer tie
    i, D = O.nn_config(np.array([[1, 0], [0, 1], [-1, 0], [0.5, 0.5]], float), q0)        # later and nearer
    assert i == 3 and abs(D - math.sqrt(0.5)) < 1e-15
    i, D = O.nn_config(np.array([[0.6, 0.8], [0.0, 0.9], [0.9, 0.0]], float), q0)
    assert i == 1 and abs(D - 0.9) < 1e-15
    assert O.nn_config(np.zeros((0, 2)), q0)[0] == -1
    # 7 coordinates: distance over all of them (no truncation to 3 or 6).
    x = np.zeros((2, 7))
    x[0, 6] = 0.5   # differs only in the last joint
    x[1, 0] = 0.4
    i, D = O.nn_config(x, np.zeros(7))
    assert i == 1 and abs(D - 0.4) < 1e-15


# --- Philox-derived decisions of small runs --------------------------------------

def _draws(prm, k, w, nslots):
    out = []
    for b in range((nslots + 3) // 4):
        out.extend(O.philox((b, w, k, prm.problem_id), (prm.seed & 0xFFFFFFFF, prm.seed >> 32)).tolist())
    return out


def _u(x):
    return (x >> 8) * 2.0 ** -24


def _wall(prob):
    """disc2d with its moving discs replaced by a static wall of discs on the
    anti-diagonal (gap at the lower right), so that the first solution takes
    many iterations and backward trees grow (exercises the new-root coin)."""
    xs = np.arange(0.0, 0.78, 0.07)
    way = np.zeros((len(xs), 1, 4))
    way[:, 0, 1] = xs
    way[:, 0, 2] = 1.0 - xs
    return dataclasses.replace(prob, way=way, obs_r=np.full(len(xs), 0.05))


def _interval_runs():
    prob, prm = WL.disc2d(0)
    out = []
    for pb, W, iters in [(prob, 8, 40), (_wall(prob), 8, 60)]:
        p = dataclasses.replace(prm, workers=W, max_iters=iters, p_new=0.3, seed=3)
        out.append((pb, p, O.plan(pb, p)))
    return out


def _group_active(r, prm, k, g):
    """Trees of group g created before iteration k with root time below U0."""
    U0 = r.U_hist[k - 1] if k > 0 else math.inf
    seg = r.seg[g]
    roots = (seg.parent == -1) & (seg.iter < k)
    return int(np.sum(seg.troot[roots] < U0))


def test_interval_direction_group_window_and_coin():
    n_skip = n_sampled = n_virtual = n_nn = 0
    for prob, prm, r in _interval_runs():
        n_skip, n_sampled, n_virtual, n_nn = _check_interval_run(prob, prm, r, n_skip, n_sampled, n_virtual, n_nn)
    # Every branch was exercised.
    assert n_skip > 20 and n_sampled > 50 and n_virtual > 5 and n_nn > 5, (n_skip, n_sampled, n_virtual, n_nn)


def _check_interval_run(prob, prm, r, n_skip, n_sampled, n_virtual, n_nn):
    d, v = prob.dof, prob.vmax
    for k in range(r.iters):
        for w in range(prm.workers):
            rec, rd = r.trace[k, w], r.trace_d[k, w]
            fl = rec[FLD["flags"]]
            raw = _draws(prm, k, w, 5 + d)
            # Direction: forward iff w + k even (Algorithm 2 alternates).
            assert bool(fl & F["fwd"]) == ((w + k) % 2 == 0)
            # Group: floor(u N) of slot 0.
            assert rec[FLD["group"]] == ((raw[0] >> 8) * prm.n_roots) >> 24
            if fl & F["root_hit"]:
                assert not fl & (F["sampled"] | F["emit"] | F["inserted"])
                continue
            # Conditional query time (Eq. conditional-query-time).
            qr = prob.qlo + np.array([_u(raw[4 + j]) for j in range(d)]) * (prob.qhi - prob.qlo)
            T = rd[0]
            lo = np.linalg.norm(qr - prob.qs) / v
            hi = T - np.linalg.norm(prob.qg - qr) / v
            assert abs(rd[2] - lo) < 1e-12 and abs(rd[3] - hi) < 1e-12
            if lo > hi:
                n_skip += 1
                assert not fl & F["sampled"] and np.isnan(rd[1])
                assert rec[FLD["parent"]] == -1 and not fl & (F["emit"] | F["virtual"] | F["inserted"])
                continue
            n_sampled += 1
            assert fl & F["sampled"]
            tr = rd[1]
            assert lo <= tr <= hi
            assert abs(tr - (lo + _u(raw[4 + d]) * (hi - lo))) < 1e-12
            # Reachable from the start and able to reach the goal by T.
            assert np.linalg.norm(qr - prob.qs) <= v * tr + 1e-12
            assert np.linalg.norm(prob.qg - qr) <= v * (T - tr) + 1e-12
            if not fl & F["fwd"]:
                g = rec[FLD["group"]]
                empty = _group_active(r, prm, k, g) == 0
                want = empty or _u(raw[3]) <= prm.p_new
                assert bool(fl & F["virtual"]) == want, (k, w)
                n_virtual += want
                n_nn += not want
    return n_skip, n_sampled, n_virtual, n_nn


def _parked(prob, until):
    """Adds a disc (r 0.05) parked on the goal from t = 0 to `until`, then
    gone: goal checks before `until` collide, so recycling slots whose grid
    range lies before it stay empty. Every obstacle gets three waypoints."""
    M = len(prob.obs_r)
    way = np.zeros((M + 1, 3, 4))
    for m in range(M):
        w = prob.way[m]
        way[m, :, 1:] = w[-1, 1:]
        way[m, :, 0] = (0.0, 1000.0, 2000.0)
    way[M] = [(0.0, prob.qg[0], prob.qg[1], 0.0), (until, prob.qg[0], prob.qg[1], 0.0),
              (until + 0.5, 5.0, 5.0, 0.0)]
    return dataclasses.replace(prob, way=way, obs_r=np.concatenate([prob.obs_r, [0.05]]))


def test_recycling_direction_and_round_robin_slots():
    base, prm = WL.disc2d(1)
    prm = dataclasses.replace(prm, variant=1, workers=8, max_iters=30, eta=0.05)
    wall = _wall(base)
    cases = [(wall, None), (_parked(wall, 12.0), [2, 3])]
    for prob, want_active in cases:
        r = O.plan(prob, prm)
        # No solution within the budget: the slots keep their initial roots.
        assert r.first_iter < 0
        active = [i for i in range(prm.n_roots) if r.slots["has_root"][i]]
        if want_active is not None:
            assert active == want_active
        else:
            assert active == list(range(prm.n_roots))
        for k in range(r.iters):
            for w in range(prm.workers):
                rec = r.trace[k, w]
                fwd = (w + k) % 2 == 0
                assert bool(rec[FLD["flags"]] & F["fwd"]) == fwd
                if fwd:
                    assert rec[FLD["group"]] == -1
                else:
                    # Backward ordinal floor(w/2) takes active slot ordinal mod #active.
                    assert rec[FLD["group"]] == active[(w // 2) % len(active)], (k, w)


# --- brute force over a whole interval-root run -----------------------------------

def _rho(qa, ta, qb, tb, v):
    """rho of the edges (qa, ta) -> (qb, tb) (rows broadcast against each
    other); inf unless the time step is positive and within the speed bound."""
    D = np.sqrt(np.sum((np.asarray(qb) - np.asarray(qa)) ** 2, axis=-1))
    dt = np.asarray(tb) - np.asarray(ta)
    ok = (dt > 0) & (D <= v * dt)
    r = np.sqrt((D * D + v * v * dt * dt) / 2.0)
    return np.where(ok, r, np.inf)


def _lexmin(k1, k2):
    """Index of the lexicographic (k1, k2, index) minimum with a finite k2, or
    -1; plus whether the runner-up key is within 1e-12 (an ambiguous tie)."""
    idx = np.flatnonzero(np.isfinite(k2))
    if len(idx) == 0:
        return -1, False
    order = sorted(idx, key=lambda i: (k1[i], k2[i], i))
    b = order[0]
    amb = len(order) > 1 and k1[order[1]] == k1[b] and abs(k2[order[1]] - k2[b]) < 1e-12
    return b, amb


@pytest.mark.parametrize("case", ["disc2d-seed0", "disc2d-seed5", "wall"])
def test_interval_run_decisions_by_brute_force(case):
    prob, prm = WL.disc2d(0)
    if case == "wall":
        prob = _wall(prob)
        prm = dataclasses.replace(prm, max_iters=150, p_new=0.3, seed=3)
    else:
        prm = dataclasses.replace(prm, max_iters=60, seed=int(case[-1]))
    r = O.plan(prob, prm)
    d, v, N = prob.dof, prob.vmax, prm.n_roots
    fx, fit = r.fwd.x, r.fwd.iter
    n_par = n_cand = n_emit = n_win = 0
    for k in range(r.iters):
        U0 = r.U_hist[k - 1] if k > 0 else math.inf
        C0 = r.C_hist[k - 1] if k > 0 else math.inf
        fset = np.flatnonzero(fit < k)
        succ = []
        for w in range(prm.workers):
            rec, rd = r.trace[k, w], r.trace_d[k, w]
            fl = rec[FLD["flags"]]
            g = rec[FLD["group"]]
            # NN parent (Algorithm 1): argmin rho over the start-of-iteration set.
            if fl & F["sampled"] and not fl & F["virtual"]:
                raw = _draws(prm, k, w, 5 + d)
                qr = prob.qlo + np.array([_u(raw[4 + j]) for j in range(d)]) * (prob.qhi - prob.qlo)
                tr = rd[1]
                if fl & F["fwd"]:
                    # sigma = +1: from an earlier tree node to the sample.
                    key = _rho(fx[fset, :d], fx[fset, d], qr, tr, v)
                    b, amb = _lexmin(np.zeros(len(fset)), key)
                    want = -1 if b < 0 else int(fset[b])
                else:
                    # sigma = -1: from the sample to a later node of group g's active trees.
                    A = r.seg[g]
                    sset = np.flatnonzero((A.iter < k) & (A.troot < U0))
                    key = _rho(qr, tr, A.x[sset, :d], A.x[sset, d], v)
                    b, amb = _lexmin(np.zeros(len(sset)), key)
                    want = -1 if b < 0 else int(sset[b])
                if not amb:
                    assert rec[FLD["parent"]] == want, (k, w)
                    n_par += 1
            if not fl & F["inserted"]:
                continue
            # Bridge rank against the opposite start-of-iteration set.
            fwd = bool(fl & F["fwd"])
            A = r.fwd if fwd else r.seg[g]
            a = A.x[rec[FLD["inserted"]]]
            a_cost = A.cost[rec[FLD["inserted"]]]
            a_troot = A.troot[rec[FLD["inserted"]]]
            if fwd:
                k1, k2, ids = [], [], []
                for s in range(N):
                    B = r.seg[s]
                    sset = np.flatnonzero((B.iter < k) & (B.troot < U0))
                    if len(sset):
                        k1.append(B.troot[sset])
                        k2.append(_rho(a[:d], a[d], B.x[sset, :d], B.x[sset, d], v))
                        ids += [(s, int(i)) for i in sset]
                k1 = np.concatenate(k1) if k1 else np.zeros(0)
                k2 = np.concatenate(k2) if k2 else np.zeros(0)
            else:
                k2 = _rho(fx[fset, :d], fx[fset, d], a[:d], a[d], v)
                k1 = np.full(len(fset), a_troot)
                ids = [(-1, int(i)) for i in fset]
            b, amb = _lexmin(k1, k2)
            if amb:
                continue
            assert bool(rec[FLD["flags"]] & F["br_cand"]) == (b >= 0), (k, w)
            if b < 0:
                continue
            n_cand += 1
            assert (rec[FLD["br_set"]], rec[FLD["br_idx"]]) == ids[b], (k, w)
            s, i = ids[b]
            vb = r.seg[s].x[i] if fwd else fx[i]
            cb = r.seg[s].cost[i] if fwd else r.fwd.cost[i]
            fnode, bnode = (a, vb) if fwd else (vb, a)
            Uc = r.seg[s].troot[i] if fwd else a_troot
            Cc = (a_cost if fwd else cb) + np.linalg.norm(fnode[:d] - bnode[:d]) + (cb if fwd else a_cost)
            improves = Uc < U0 or (Uc == U0 and Cc < C0)
            assert bool(fl & F["br_emit"]) == improves, (k, w)
            if not improves:
                continue
            n_emit += 1
            ok, _, _, _ = O.check_edges(prob, fnode[None, :d], [fnode[d]], bnode[None, :d], [bnode[d]], prm.res)
            assert bool(fl & F["br_hit"]) == (not ok[0]), (k, w)
            if ok[0]:
                succ.append((Uc, Cc, w))
        # Publish: lexicographic (U, C, worker) minimum of the successes.
        winners = [w for w in range(prm.workers) if r.trace[k, w, 0] & F["winner"]]
        if succ:
            best = min(succ)
            assert winners == [best[2]], (k, winners, best)
            assert abs(r.U_hist[k] - best[0]) < 1e-12
            n_win += 1
        else:
            assert winners == []
            assert r.U_hist[k] == U0 or (k == 0 and math.isinf(r.U_hist[k]))
    # Statistics: one validated edge per emitted bridge (only the top candidate).
    emitted = int(np.sum((r.trace[:, :, 0] & F["br_emit"]) != 0))
    assert r.bridge_checked == emitted
    assert n_par > 100 and n_cand > 100 and n_emit > 5 and n_win >= 1, (n_par, n_cand, n_emit, n_win)
