"""The persistent planner launch (STP_LAUNCH_PERSISTENT: one cooperative
kernel per plan, steps separated by team barriers) against the per-step
kernels (STP_LAUNCH_STEPS, the single-problem default), through the C ABI. Both run the same step bodies in
the same order, so every decision must be the same: tree structure (parents,
insertion iterations, tree ids), statistics, U history and path lengths are
equal. Values may differ in their last bits where the compiler contracted a
multiply-add differently in the two kernels, so coordinates, times, costs,
U and C agree to 64 ulps of the working precision (relative; ulp-level
differences can accumulate along a tree path of a few dozen steps). Checked in FP32
and FP64, for single problems and for a batch planned from the persistent
work queue. Both forms are also checked against the FP64 oracle elsewhere
(test_gpu_plan.py and test_gpu_follow.py run single problems with the
per-step kernels and batches from the persistent queue)."""
import dataclasses

import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


def _small_arm(variant=1, workers=64, iters=30):
    prob, prm = WL.ur5e(0, n_obs=4, candidate=0)
    prob.qg = prob.qs + np.array([0.6, -0.4, 0.5, 0.3, -0.2, 0.4])
    return prob, dataclasses.replace(prm, variant=variant, workers=workers, max_iters=iters,
                                     eta=0.3 if variant == 0 else prm.eta)


CASES = {
    "disc2d-interval": lambda: (WL.disc2d(0)[0], dataclasses.replace(WL.disc2d(0)[1], max_iters=120)),
    "disc2d-recycling": lambda: (WL.disc2d(1)[0], dataclasses.replace(WL.disc2d(1)[1], variant=1, max_iters=80,
                                                                       eta=0.05)),
    "ur5e-small-recycling": lambda: _small_arm(1),
    "ur5e-small-interval": lambda: _small_arm(0),
    "ur5e-timed": lambda: (WL.ur5e(0)[0], dataclasses.replace(WL.ur5e(0)[1], max_iters=32)),
    "arm7-interval": lambda: (WL.arm7(0)[0], dataclasses.replace(WL.arm7(0)[1], variant=0, workers=512,
                                                                  max_iters=6)),
    "ragged-workers": lambda: (WL.disc2d(2)[0], dataclasses.replace(WL.disc2d(2)[1], workers=1500, max_iters=4)),
}

KEYS = ("iterations", "first_solution_iter", "nodes", "edges_validated", "bridges_validated", "root_checks",
        "nn_evals", "nn_nodes", "bridge_evals", "bridge_nodes")


def _snapshot(P, prm, out):
    trees = [P.tree(a) for a in range(-1, prm.n_roots)]
    return dict(U=out.U, C=out.C, path=out.path.copy(), stats=tuple(out.stats[k] for k in KEYS),
                trees=[{k: v.copy() for k, v in t.items()} for t in trees], hist=P.history().copy(),
                status=out.status)


def _close(x, y, rtol):
    x, y = np.asarray(x, float), np.asarray(y, float)
    if x.shape != y.shape:
        return False
    same_inf = np.isinf(x) & np.isinf(y) & (np.sign(x) == np.sign(y))
    fin = np.isfinite(x) & np.isfinite(y)
    ok = np.zeros(x.shape, dtype=bool)
    ok[fin] = np.abs(x[fin] - y[fin]) <= rtol * np.maximum(np.abs(y[fin]), 1e-30)
    return bool(np.all(same_inf | ok))


def _identical(a, b, rtol):
    assert a["status"] == b["status"]
    assert a["stats"] == b["stats"], (a["stats"], b["stats"])
    assert _close(a["U"], b["U"], rtol) and _close(a["C"], b["C"], rtol), (a["U"], b["U"], a["C"], b["C"])
    assert a["path"].shape == b["path"].shape and _close(a["path"], b["path"], rtol)
    assert _close(a["hist"], b["hist"], rtol)
    for ta, tb in zip(a["trees"], b["trees"]):
        for k in ("parent", "iter", "tree"):
            assert np.array_equal(ta[k], tb[k]), k
        for k in ("x", "troot", "cost"):
            assert _close(ta[k], tb[k], rtol), (k, float(np.max(np.abs(ta[k] - tb[k]))))


def _rtol(precision):
    return 64 * (2.0 ** -52 if precision else 2.0 ** -23)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_persistent_equals_per_step_kernels(case, precision):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    snaps = []
    for mode in (stp.STP_LAUNCH_PERSISTENT, stp.STP_LAUNCH_STEPS):
        P = stp.problem_from(prob, prm, precision=precision, launch_mode=mode)
        out = P.plan()
        snaps.append(_snapshot(P, prm, out))
        if mode == stp.STP_LAUNCH_PERSISTENT:
            # A replay of the persistent plan gives the same result.
            _identical(snaps[0], _snapshot(P, prm, P.plan()), 0.0)
            prof = P.profile()
            assert all(v[0] > 0 for v in prof.values()), prof
        P.close()
    _identical(snaps[0], snaps[1], _rtol(precision))
    print(case, "fp%d" % (64 if precision else 32), snaps[0]["stats"])


@pytest.mark.parametrize("ctas", [1, 2, 16, 64])
def test_persistent_team_size_does_not_change_results(ctas):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES["ur5e-small-recycling"]()
    ref = None
    for c in (0, ctas):
        P = stp.problem_from(prob, prm, precision=0, launch_mode=stp.STP_LAUNCH_PERSISTENT, persist_ctas=c)
        snap = _snapshot(P, prm, P.plan())
        P.close()
        if ref is None:
            ref = snap
        else:
            _identical(ref, snap, 0.0)


def test_persistent_batch_equals_per_step_batch_and_single_runs():
    """A mixed batch from the persistent work queue (teams of CTAs taking
    problems from a device queue) equals the per-step batch and each
    problem's single persistent run."""
    from paper_2609_30533_gb300 import stp
    cases = [CASES[k]() for k in ("disc2d-interval", "disc2d-recycling", "ur5e-small-recycling",
                                  "ur5e-small-interval")]
    p, q = WL.arm7(1, variant=0)
    cases.append((p, dataclasses.replace(q, workers=128, max_iters=5)))
    p, q = WL.disc2d(1)
    p.qg = p.qs.copy()           # start == goal: resolved without iterations
    cases.append((p, q))
    cases = cases * 3            # more problems than a small team count: the queue hands out the rest
    results = {}
    for mode, team in ((stp.STP_LAUNCH_DEFAULT, 4), (stp.STP_LAUNCH_PERSISTENT, 16), (stp.STP_LAUNCH_STEPS, 0)):
        probs = [stp.problem_from(pb, pm, precision=0, iters_per_graph=8) for pb, pm in cases]
        B = stp.Batch(probs, nn_ctas=4, validate_ctas=4, launch_mode=mode, team_ctas=team)
        _, stats = B.plan()
        snap = []
        for P, (pb, pm), st in zip(probs, cases, stats):
            trees = [P.tree(a) for a in range(-1, pm.n_roots)] if st["iterations"] else []
            snap.append((tuple(st[k] for k in KEYS), st["U"], st["C"], trees, B.path(probs.index(P))))
        results[(mode, team)] = snap
        B.close()
        for P in probs:
            P.close()
    results[(0, 16)] = results.pop((2, 16))
    base = results[(1, 0)]
    rt = _rtol(0)
    for key in ((0, 4), (0, 16)):
        for a, b in zip(results[key], base):
            assert a[0] == b[0]
            assert _close(a[1], b[1], rt) and _close(a[2], b[2], rt)
            assert a[4].shape == b[4].shape and _close(a[4], b[4], rt)
            for ta, tb in zip(a[3], b[3]):
                for k in ("parent", "iter", "tree"):
                    assert np.array_equal(ta[k], tb[k]), k
                for k in ("x", "troot", "cost"):
                    assert _close(ta[k], tb[k], rt), k
        # The two persistent team sizes run the same kernel: identical.
    for a, b in zip(results[(0, 4)], results[(0, 16)]):
        assert a[0] == b[0] and np.array_equal(a[4], b[4])
    # Single persistent runs of the members agree with the batch.
    for (pb, pm), (st, U, Cc, trees, path) in zip(cases[:6], results[(0, 4)][:6]):
        P = stp.problem_from(pb, pm, precision=0, launch_mode=stp.STP_LAUNCH_PERSISTENT)
        out = P.plan()
        assert tuple(out.stats[k] for k in KEYS) == st
        assert out.path.shape == path.shape and _close(out.path, path, _rtol(0))
        P.close()
