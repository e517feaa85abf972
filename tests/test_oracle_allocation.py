"""Oracle pins for goal-time allocation (interval root) and root recycling.

The interval-root partitions are pinned exactly by the worked example drawn in
Fig. interval-root; the recycling rule by the example drawn in Fig. method and
the rule that a slot whose root sits exactly at U is recycled only once U
improves strictly below it (Sec. "Practical Root Recycling").
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _num(x):
    return float(Fraction(x)) if isinstance(x, str) else float(x)


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _flags(ex):
    kmax = int(ex["H"] / ex["dt"])
    return np.array([1 if k in ex["free_k"] else 0 for k in range(ex["kmin"], kmax + 1)], dtype=np.uint8)


@pytest.mark.parametrize("panel", ["before", "after"])
def test_interval_root_worked_example(panel):
    ex = _load("interval_root_example.json")
    U = float("inf") if panel == "before" else ex["after"]["U"]
    uni, width, pieces = O.interval_partition(ex["Lg"], ex["H"], ex["dt"], ex["N"], U, ex["kmin"], _flags(ex))
    want = ex[panel]
    for g in range(ex["N"]):
        lo, hi = (_num(v) for v in want["uniform"][g])
        assert abs(uni[g] - lo) < 1e-12 and abs(uni[g] + width - hi) < 1e-12
        got = [(p[0], p[1]) for p in pieces if int(p[2]) == g]
        exp = [tuple(_num(v) for v in iv) for iv in want["guided"][g]]
        assert len(got) == len(exp), (g, got, exp)
        for (a, b), (c, d) in zip(got, exp):
            assert abs(a - c) < 1e-12 and abs(b - d) < 1e-12
        meas = sum(b - a for a, b in got)
        assert abs(meas - _num(want["guided_measure_each"])) < 1e-12


def test_interval_root_sampling_maps_into_pieces():
    ex = _load("interval_root_example.json")
    f = _flags(ex)
    args = (ex["Lg"], ex["H"], ex["dt"], ex["N"], float("inf"), ex["kmin"], f)
    # Group 0 guided pieces [0.5,1.5] u [3.5,4.5]: position u*2 walks the pieces.
    T, g = O.interval_sample(*args, 0, 0.1, 0.25, 0.95)
    assert g and abs(T - 1.0) < 1e-12
    T, g = O.interval_sample(*args, 0, 0.1, 0.75, 0.95)
    assert g and abs(T - 4.0) < 1e-12
    # Coin above p_guided: uniform interval I_1 = [4, 8).
    T, g = O.interval_sample(*args, 1, 0.96, 0.5, 0.95)
    assert (not g) and abs(T - 6.0) < 1e-12
    # After U = 9.5 group 2 guided = [35/6, 6.5] u [8.5, 9.5] (measure 5/3).
    args_u = (ex["Lg"], ex["H"], ex["dt"], ex["N"], 9.5, ex["kmin"], f)
    T, g = O.interval_sample(*args_u, 2, 0.0, 0.5, 0.95)
    assert g and abs(T - (8.5 + (5 / 6 - 2 / 3))) < 1e-12
    # No free check anywhere: guided portions empty, fall back to uniform.
    T, g = O.interval_sample(ex["Lg"], ex["H"], ex["dt"], 3, float("inf"), 0, np.zeros_like(f), 2, 0.0, 0.5,
                             0.95)
    assert (not g) and abs(T - 10.0) < 1e-12


def test_interval_root_guided_mean_is_piece_midpoint():
    ex = _load("interval_root_example.json")
    f = _flags(ex)
    us = (np.arange(2000) + 0.5) / 2000
    Ts = [O.interval_sample(ex["Lg"], ex["H"], ex["dt"], 3, float("inf"), 0, f, 1, 0.0, u, 0.95)[0] for u in us]
    assert abs(np.mean(Ts) - 5.5) < 1e-3          # group 2 = [4.5, 6.5]
    assert min(Ts) >= 4.5 and max(Ts) <= 6.5


def test_interval_windows_clip_to_Lg_and_H():
    # L_g = 0.3 (grid dt = 1): check at k=1 gives [0.5,1.5]; k = kmin..kmax = 1..3
    uni, w, pieces = O.interval_partition(0.3, 3.2, 1.0, 1, float("inf"), 1, np.array([1, 0, 1], np.uint8))
    got = [(round(p[0], 12), round(p[1], 12)) for p in pieces]
    assert got == [(0.5, 1.5), (2.5, 3.2)]
    assert abs(uni[0] - 0.3) < 1e-12 and abs(w - 2.9) < 1e-12
    # k = 1 adjacent to L_g = 0.8: window [0.5,1.5] clipped to [0.8,1.5].
    _, _, pieces = O.interval_partition(0.8, 3.0, 1.0, 2, float("inf"), 1, np.array([1, 1, 0], np.uint8))
    assert abs(pieces[0][0] - 0.8) < 1e-12 and abs(pieces[-1][1] - 2.5) < 1e-12


def _recycle_fixture():
    ex = _load("root_recycling_example.json")
    dt = 0.5
    kmin = int(ex["L_grid"] / dt)
    flags = np.ones(int(48 / dt) - kmin + 1, dtype=np.uint8)
    return ex, dt, kmin, flags


def test_root_recycling_worked_example():
    ex, dt, kmin, flags = _recycle_fixture()
    N = len(ex["roots"])
    T, hr, ac, gen, n = O.recycle_update(ex["roots"], [1] * N, [1] * N, [0] * N, ex["U"], kmin, flags, dt)
    assert n == len(ex["donors"])
    for i in range(N):
        if str(i) in ex["replacements"]:
            assert T[i] == ex["replacements"][str(i)] and ac[i] == 1 and gen[i] == 1
            assert T[i] < ex["U"] and T[i] >= ex["L_grid"]
        elif i in ex["inactive_kept"]:
            assert T[i] == ex["roots"][i] and ac[i] == 0 and gen[i] == 0
        else:
            assert T[i] == ex["roots"][i] and ac[i] == 1 and gen[i] == 0


def test_root_at_U_is_donor_only_after_strict_improvement():
    ex, dt, kmin, flags = _recycle_fixture()
    N = len(ex["roots"])
    T, hr, ac, gen, _ = O.recycle_update(ex["roots"], [1] * N, [1] * N, [0] * N, 32.0, kmin, flags, dt)
    # Same U again (no strict improvement): nothing changes.
    T2, hr2, ac2, gen2, n2 = O.recycle_update(T, hr, ac, gen, 32.0, kmin, flags, dt)
    assert n2 == 0 and np.array_equal(T2, T) and np.array_equal(ac2, ac)
    # Strict improvement to U = 30: the root at 32 is now a donor and is replaced
    # inside [14, 30) at the middle of the range (single donor), below first.
    T3, hr3, ac3, gen3, n3 = O.recycle_update(T, hr, ac, gen, 30.0, kmin, flags, dt)
    assert n3 == 1 and T3[2] == 22.0 and ac3[2] == 1 and gen3[2] == 1
    # A root exactly at the new U becomes inactive but is not replaced.
    T4, hr4, ac4, gen4, n4 = O.recycle_update(T3, hr3, ac3, gen3, 27.5, kmin, flags, dt)
    assert ac4[4] == 0 and T4[4] == 27.5 and gen4[4] == 1 and n4 == 0


def test_recycling_without_free_candidates_keeps_donor_inactive():
    ex, dt, kmin, flags = _recycle_fixture()
    N = len(ex["roots"])
    blocked = np.zeros_like(flags)
    T, hr, ac, gen, n = O.recycle_update(ex["roots"], [1] * N, [1] * N, [0] * N, 32.0, kmin, blocked, dt)
    assert n == 0
    assert list(ac) == [1, 1, 0, 0, 0] and list(T) == ex["roots"]


def test_recycling_skips_times_held_by_active_roots():
    # Donor target falls on a held grid time; the outward scan takes the next
    # lower free time first.
    dt, kmin = 1.0, 0
    flags = np.ones(20, dtype=np.uint8)
    # roots 5 (active), 15 (donor when U = 10); K_U = 10, m = 1 -> target 5 (held)
    T, hr, ac, gen, n = O.recycle_update([5.0, 15.0], [1, 1], [1, 1], [0, 0], 10.0, kmin, flags, dt)
    assert n == 1 and T[1] == 4.0
    flags[4] = 0   # 4 blocked -> next candidate above: 6
    T, hr, ac, gen, n = O.recycle_update([5.0, 15.0], [1, 1], [1, 1], [0, 0], 10.0, kmin, flags, dt)
    assert T[1] == 6.0
