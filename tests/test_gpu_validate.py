"""GPU collision kernel vs the FP64 oracle (through the C ABI).

Bar: FP64 device mode gives the oracle's verdicts, check counts and clearances
(to rounding); FP32 verdicts equal the FP64 ones except for edges whose FP64
clearance lies within 1e-5 m of zero, which are counted and reported. FP32 also
rounds the configuration box (float32(pi) > pi), so edges whose checked states
lie within 1e-6 of the box boundary are counted in the band as well.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

BAND = 1e-5
BOX_BAND = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_30533_gb300 import build as B
    B.build()


def _problem(name):
    if name == "disc2d":
        return WL.disc2d(0)
    if name == "ur5e":
        return WL.ur5e(0)
    if name == "arm7":
        return WL.arm7(0)
    raise KeyError(name)


def _edges(prob, prm, n, seed):
    if prob.arm:
        return WL.microbench_edges(prob, n, prm.eta, prm.H, seed=seed)
    rng = np.random.default_rng(seed)
    qa = rng.uniform(0, 1, (n, 2))
    qb = np.clip(qa + rng.uniform(-0.15, 0.15, (n, 2)), 0, 1)
    D = np.linalg.norm(qb - qa, axis=1)
    ta = rng.uniform(0, prm.H - 1, n)
    tb = ta + D / prob.vmax * rng.uniform(1.0, 3.0, n)
    return qa, ta, qb, tb


def _as(x, dt):
    return np.asarray(x, dtype=dt).astype(np.float64)


@pytest.mark.parametrize("name", ["disc2d", "ur5e", "arm7"])
def test_fp64_verdicts_counts_clearance_match_oracle(name):
    from paper_2609_30533_gb300 import stp
    prob, prm = _problem(name)
    n = 3000 if name != "arm7" else 1000
    qa, ta, qb, tb = _edges(prob, prm, n, 11)
    P = stp.problem_from(prob, prm, precision=1, max_iters=1)
    v, clr, nc = P.check_edges(qa, ta, qb, tb, clearance=True, n_checks=True)
    rv, rclr, rnc, rim = O.check_edges(prob, qa, ta, qb, tb, prm.res)
    assert np.array_equal(nc, rnc)
    tiny = np.abs(rclr) < 1e-9
    assert np.array_equal(v[~tiny], rv[~tiny])
    assert np.allclose(clr, rclr, rtol=0, atol=1e-9)
    v2, _, _ = P.check_edges(qa, ta, qb, tb)                       # early-exit path
    v3, _, _ = P.check_edges(qa, ta, qb, tb, early_exit=False)
    assert np.array_equal(v2, v) and np.array_equal(v3, v)
    assert 0.05 < v.mean() < 0.98, v.mean()                        # both outcomes exercised
    P.close()


@pytest.mark.parametrize("name", ["disc2d", "ur5e", "arm7"])
def test_fp32_verdicts_within_clearance_band(name):
    from paper_2609_30533_gb300 import stp
    prob, prm = _problem(name)
    n = 4000 if name != "arm7" else 1500
    qa, ta, qb, tb = _edges(prob, prm, n, 12)
    f = np.float32
    qa, ta, qb, tb = _as(qa, f), _as(ta, f), _as(qb, f), _as(tb, f)
    P = stp.problem_from(prob, prm, precision=0, max_iters=1)
    v, clr, nc = P.check_edges(qa, ta, qb, tb, clearance=True, n_checks=True)
    rv, rclr, rnc, rim, rbm = O.check_edges(prob, qa, ta, qb, tb, prm.res, bounds=True)
    # Counts are evaluated in double from the same FP32 endpoints on both sides.
    assert np.array_equal(nc, rnc)
    mism = v != rv
    banded = (np.abs(rclr) <= BAND) | (np.abs(rbm) <= BOX_BAND)
    assert not (mism & ~banded).any(), np.flatnonzero(mism & ~banded)[:10]
    print("%s: %d edges, %d in the 1e-5 m band, %d verdict flips inside it" %
          (name, n, int(banded.sum()), int(mism.sum())))
    assert np.allclose(clr, rclr, rtol=0, atol=BAND)
    print("  box-band edges: %d" % int((np.abs(rbm) <= BOX_BAND).sum()))
    v2, _, _ = P.check_edges(qa, ta, qb, tb)
    assert np.array_equal(v2, v)
    P.close()


def test_edge_cases_point_edges_and_small_batches():
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.ur5e(0)
    P = stp.problem_from(prob, prm, precision=1, max_iters=1)
    # n = 0 is a no-op; n = 1; zero-length edges (single point at s = 1).
    v, _, _ = P.check_edges(np.zeros((0, 6)), np.zeros(0), np.zeros((0, 6)), np.zeros(0))
    assert len(v) == 0
    q = prob.qs[None]
    v, clr, nc = P.check_edges(q, [0.0], q, [0.0], clearance=True, n_checks=True)
    ok, c0 = O.state_free(prob, prob.qs, 0.0)
    assert nc[0] == 1 and bool(v[0]) == ok and abs(clr[0] - c0) < 1e-9
    # Out of the joint box collides.
    qo = prob.qs.copy()
    qo[0] = 4.0
    v, _, _ = P.check_edges(qo[None], [0.0], qo[None], [0.0])
    assert v[0] == 0
    # Ragged batch sizes around warp / tile boundaries.
    qa, ta, qb, tb = WL.microbench_edges(prob, 97, prm.eta, prm.H, seed=3)
    for m in (1, 31, 33, 97):
        v, _, nc = P.check_edges(qa[:m], ta[:m], qb[:m], tb[:m], n_checks=True)
        rv, rclr, rnc, _ = O.check_edges(prob, qa[:m], ta[:m], qb[:m], tb[:m], prm.res)
        assert np.array_equal(nc, rnc) and np.array_equal(v[np.abs(rclr) > 1e-9], rv[np.abs(rclr) > 1e-9])
    P.close()


def test_full_size_microbench_sampled_against_oracle():
    """2^20 UR5e edges through the device-pointer path (the benchmark's launch
    configuration); 1500 sampled verdicts checked one by one by the oracle."""
    import torch
    from paper_2609_30533_gb300 import stp
    prob, prm = WL.ur5e(0)
    n = 1 << 20
    qa, ta, qb, tb = WL.microbench_edges(prob, n, prm.eta, prm.H, seed=0)
    dev = torch.device("cuda:0")
    tq = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in (qa, ta, qb, tb)]
    ver = torch.zeros(n, dtype=torch.uint8, device=dev)
    P = stp.problem_from(prob, prm, precision=0, max_iters=1)
    torch.cuda.synchronize()
    P.check_edges_device(tq[0].data_ptr(), tq[1].data_ptr(), tq[2].data_ptr(), tq[3].data_ptr(), n,
                         ver.data_ptr())
    torch.cuda.synchronize()
    v = ver.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = rng.choice(n, 1500, replace=False)
    f = np.float32
    rv, rclr, _, _, rbm = O.check_edges(prob, _as(qa[idx], f), _as(ta[idx], f), _as(qb[idx], f),
                                        _as(tb[idx], f), prm.res, bounds=True)
    bad = (v[idx] != rv) & (np.abs(rclr) > BAND) & (np.abs(rbm) > BOX_BAND)
    assert not bad.any()
    frac_free = v.mean()
    assert 0.2 < frac_free < 0.95, frac_free
    P.close()
