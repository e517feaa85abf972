"""Write accepted_candidates.json: for each arm workload and seed, the index of
the first start/goal candidate whose start is clear (>= 2 cm) at t = 0 and whose
goal is clear (>= 2 cm) at some time on a 0.1 s grid of [0, H].

Acceptance is decided by the FP64 oracle only (a committed script that calls
only oracle/); the planner library never runs this.

    python -m workloads.select_candidates
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as WL  # noqa: E402

MARGIN = 0.02


def accept(prob, H):
    ok, clr = O.state_free(prob, prob.qs, 0.0)
    if not ok or clr < MARGIN:
        return False
    for t in np.arange(0.0, H + 1e-9, 0.1):
        ok, clr = O.state_free(prob, prob.qg, float(t))
        if ok and clr >= MARGIN:
            return True
    return False


def first_accepted(make, H):
    for c in range(WL.N_CANDIDATES):
        prob, _ = make(c)
        if accept(prob, H):
            return c
    return 0


def main():
    table = {"ur5e": {}, "arm7": {}, "mixed": {}}
    for seed in range(8):
        table["ur5e"][str(seed)] = first_accepted(lambda c: WL.ur5e(seed, candidate=c), 15.0)
        table["arm7"][str(seed)] = first_accepted(lambda c: WL.arm7(seed, candidate=c), 60.0)
    for idx in range(512):
        fam = idx % 3
        if fam == 0:
            continue
        rng = np.random.default_rng(4000 + idx)
        H = float(rng.uniform(10.0, 60.0))
        n_obs = int(rng.integers(4, 129))
        if fam == 1:
            mk = lambda c: WL.ur5e(seed=idx, n_obs=n_obs, H=H, candidate=c)  # noqa: E731
        else:
            mk = lambda c: WL.arm7(seed=idx, n_obs=n_obs, H=H, candidate=c)  # noqa: E731
        table["mixed"][str(idx)] = first_accepted(mk, H)
    table["c4"] = {}
    for i in range(WL.C4_TRAIN_TABLED):
        seed = WL.C4_TRAIN_BASE + i
        table["c4"][str(seed)] = first_accepted(lambda c: WL.arm7(seed, candidate=c), 60.0)
    for i in range(WL.C4_TEST_TABLED):
        seed = WL.C4_TEST_BASE + i
        table["c4"][str(seed)] = first_accepted(lambda c: WL.arm7(seed, candidate=c), 60.0)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "accepted_candidates.json")
    with open(path, "w") as f:
        json.dump(table, f, indent=0, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
