"""Learned sampling branch on the GPU against the oracle: problem features,
FP64 trees node for node with a proposal installed, FP32 trees until the first
flagged decision, a batch of learned problems equal to single runs, and the
missing-proposal error."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as WL
from oracle import mlp as M
from test_gpu_plan import CASES, _compare_arena, _first_flag, _first_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


@pytest.mark.parametrize("make", [lambda: WL.disc2d(0), lambda: WL.ur5e(0), lambda: WL.arm7(0),
                                  lambda: WL.mixed(5)])
def test_features_match_oracle(make):
    from paper_2609_30533_gb300 import stp
    prob, prm = make()
    P = stp.problem_from(prob, prm, precision=0)
    x = P.features()
    ref = M.features(prob, prm.H)
    assert np.allclose(x, ref, rtol=1e-6, atol=1e-6)
    P.close()


LCASES = ["disc2d-interval", "ur5e-small-recycling", "ur5e-small-interval", "ur5e-recycling"]


def _run(case, precision):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES[case]()
    y = WL.random_proposal(prob, seed=11)
    ref = O.plan(prob, prm, proposal=y.astype(np.float64))
    P = stp.problem_from(prob, prm, precision=precision, learned=1)
    P.set_proposal(y)
    out = P.plan()
    return prob, prm, ref, P, out


@pytest.mark.parametrize("case", LCASES)
def test_fp64_learned_trees_match_oracle(case):
    from paper_2609_30533_gb300 import stp
    prob, prm, ref, P, out = _run(case, 1)
    assert out.status == (stp.STP_OK if ref.status == 0 else stp.STP_NO_SOLUTION)
    st = out.stats
    assert st["iterations"] == ref.iters and st["nodes"] == ref.inserted
    assert st["edges_validated"] == ref.ext_checked and st["bridges_validated"] == ref.bridge_checked
    _compare_arena(P.tree(-1), ref.fwd, 1e-9)
    for i in range(prm.n_roots):
        _compare_arena(P.tree(i), ref.seg[i], 1e-9)
    if ref.status == 0:
        assert abs(out.U - ref.U) < 1e-9
    # the learned branch changes the search
    plain = O.plan(prob, prm)
    assert plain.inserted != ref.inserted or not np.array_equal(plain.fwd.x, ref.fwd.x)
    P.close()


@pytest.mark.parametrize("case", LCASES)
def test_fp32_learned_trees_match_until_first_flag(case):
    prob, prm, ref, P, out = _run(case, 0)
    flag = _first_flag(ref)
    mism = _first_mismatch(P, ref, prm)
    print("%s learned: first flagged iteration %d, first FP32 mismatch %d of %d" % (case, flag, mism, ref.iters))
    assert mism >= flag
    P.close()


def test_batch_of_learned_problems_equals_single_runs():
    from paper_2609_30533_gb300 import stp
    probs, singles = [], []
    for i in range(6):
        prob, prm = WL.mixed(i)
        prm = dataclasses.replace(prm, workers=128, max_iters=24, problem_id=i)
        y = WL.random_proposal(prob, seed=i)
        a = stp.problem_from(prob, prm, precision=0, learned=1, iters_per_graph=8)
        a.set_proposal(y)
        sa = a.plan()
        singles.append((sa, a.tree(-1)["x"].copy()))
        a.close()
        b = stp.problem_from(prob, prm, precision=0, learned=1, iters_per_graph=8)
        b.set_proposal(y)
        probs.append(b)
    B = stp.Batch(probs, iters_per_graph=8)
    _, stats = B.plan()
    for i, (sa, fx) in enumerate(singles):
        for k in ("iterations", "first_solution_iter", "nodes", "edges_validated", "bridges_validated"):
            assert stats[i][k] == sa.stats[k], (i, k)
        assert np.array_equal(probs[i].tree(-1)["x"], fx)
    B.close()
    for p in probs:
        p.close()


def test_learned_without_proposal_is_rejected():
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.disc2d(0)
    P = stp.problem_from(prob, prm, precision=0, learned=1)
    with pytest.raises(stp.StpError) as e:
        P.plan()
    assert e.value.status == stp.STP_ERR_INVALID
    with pytest.raises(stp.StpError):
        P.set_proposal(np.full(160, np.nan, dtype=np.float32))
    P.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_path_targets_match_oracle_definition(precision):
    from paper_2609_30533_gb300 import stp
    prob, prm = CASES["ur5e-small-recycling"]()
    P = stp.problem_from(prob, prm, precision=precision)
    out = P.plan()
    assert out.status == stp.STP_OK
    t = P.targets()
    ref = M.path_targets(out.path, out.U, prm.H, prob.dof, prob.qlo, prob.qhi)
    assert np.allclose(t, ref, rtol=0, atol=2e-6 if precision == 0 else 1e-7)
    P.close()
    prob, prm = WL.disc2d(0)
    prob.qs = prob.way[0, 0, 1:3].copy()      # start in collision: no path
    P = stp.problem_from(prob, prm, precision=0)
    P.plan()
    assert P.targets() is None
    P.close()


def test_trained_network_gains_over_plain_sampling():
    """Train the proposal network on plain solutions of 7-DoF training problems
    (on the GPU, own kernels), then plan held-out problems with and without it
    at the same budget: the learned branch solves more problems and arrives
    earlier on average on the problems both arms solve."""
    from paper_2609_30533_gb300 import proposal as PR
    from paper_2609_30533_gb300 import stp

    def make(split, idxs, learned=0, seed=None):
        out = []
        for i in idxs:
            prob, prm = WL.arm7_c4(split, i)
            prm = dataclasses.replace(prm, variant=0, workers=256, max_iters=96,
                                      seed=prm.seed if seed is None else seed)
            out.append(stp.problem_from(prob, prm, precision=0, iters_per_graph=16, learned=learned))
        return out

    Xs, Ts = [], []
    for sd in (0, 1):
        for c in range(0, 1024, 512):
            probs = make("train", range(c, c + 512), seed=sd)
            o = PR.plan_batch(probs)
            x, t = PR.collect(probs, o)
            Xs.append(x)
            Ts.append(t)
            for P in probs:
                P.close()
    X, T = np.concatenate(Xs), np.concatenate(Ts)
    assert len(X) >= 60
    net = stp.Mlp(1024)
    net.set_params(PR.init_params(0))
    log = PR.train(net, X, T, 600, 128, 3e-4)
    assert log.best_val < log.val[0][1]
    outs = {}
    for flag in (0, 1):
        res = []
        for c in range(0, 512, 256):
            probs = make("test", range(c, c + 256), learned=flag)
            if flag:
                PR.install(net, probs)
            res.append(PR.plan_batch(probs))
            for P in probs:
                P.close()
        outs[flag] = (np.concatenate([r.solved for r in res]), np.concatenate([r.first_iter for r in res]),
                      np.concatenate([r.U for r in res]))
    net.close()
    (sp, ip, Up), (sl, il, Ul) = outs[0], outs[1]
    both = sp & sl
    print("solved plain %d learned %d, both %d; on the common solves: p50 first iteration plain %.1f learned %.1f, "
          "mean arrival plain %.3f learned %.3f s" % (sp.sum(), sl.sum(), both.sum(), np.median(ip[both]),
                                                       np.median(il[both]), Up[both].mean(), Ul[both].mean()))
    # The learned branch solves more held-out problems at the same budget and,
    # on the problems both arms solve, arrives earlier on average.
    assert sl.sum() > sp.sum()
    assert both.sum() >= 10
    assert Ul[both].mean() < Up[both].mean()
