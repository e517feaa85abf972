"""Proposal network on the tensor cores against the FP64 oracle network:
an exact identity network (layout pin), forward outputs and every parameter
gradient element by element (each output slice and each tensor on its own)
within bfloat16 tolerances on ragged and maximum batch sizes, the first Adam
step, and a training run that lowers a held-out loss."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stp():
    from paper_2609_30533_gb300 import build as B
    B.build()
    from paper_2609_30533_gb300 import stp as S
    return S


def _targets(rng, X):
    """Smooth synthetic targets: tau and waypoints as functions of x."""
    B = X.shape[0]
    T = np.zeros((B, M.N_TGT))
    T[:, 0] = 1 / (1 + np.exp(-(X[:, 0] - X[:, 7])))
    dof = rng.choice([2, 6, 7], size=B)
    for i in range(M.N_WP):
        f = (i + 1) / 17
        T[:, 1 + 8 * i:1 + 8 * i + 7] = (1 - f) * X[:, 0:7] + f * X[:, 7:14]
        T[:, 1 + 8 * i + 7] = f * T[:, 0]
    for n in range(B):
        for i in range(M.N_WP):
            T[n, 1 + 8 * i + dof[n]:1 + 8 * i + 7] = 0.0
    T[:, -1] = dof
    return T


def _inputs(rng, B):
    X = np.zeros((B, M.IN))
    X[:, 0:26] = rng.uniform(-1, 1, size=(B, 26))
    return X


def test_identity_network_is_exact(stp):
    P = {k: np.zeros_like(v) for k, v in M.init_params(np.random.default_rng(0)).items()}
    P["W1"][0:32, 0:32] = np.eye(32)
    P["W1"][32:64, 0:32] = -np.eye(32)
    P["W2"][:] = np.eye(256)
    P["W3"][:] = np.eye(256)
    P["W4"][0:32, 0:32] = np.eye(32)
    P["W4"][0:32, 32:64] = -np.eye(32)
    net = stp.Mlp(512)
    net.set_params(stp.flatten_params(P))
    X = np.random.default_rng(1).normal(size=(300, 32))
    Y = net.forward(X)
    assert np.array_equal(Y[:, 0:32].astype(np.float64), M.bf16_round(X))
    assert np.all(Y[:, 32:] == 0)
    net.close()


def _rel_rows(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-12)


def _check_forward(Y, Ye, label):
    """Element-wise per output slice against the bf16 reference."""
    worst = {}
    for name, a, b in M.OUT_SLICES:
        ok, w = M.close_elementwise(Y[:, a:b], Ye[:, a:b], M.RTOL_FWD)
        worst[name] = round(w, 4)
        assert ok, (label, name, w)
    print(label, "worst |err|/tol per slice:", worst)


@pytest.mark.parametrize("B", [1, 128, 300])
def test_forward_matches_oracle(stp, B):
    rng = np.random.default_rng(10 + B)
    P = M.init_params(rng)
    for b in ("b1", "b2", "b3", "b4"):
        P[b] = rng.normal(scale=0.1, size=P[b].shape)
    P["b4"][M.OUT_USED:] = 0.0
    X = _inputs(rng, B)
    net = stp.Mlp(512)
    net.set_params(stp.flatten_params(P))
    Y = net.forward(X).astype(np.float64)
    Ye, _ = M.forward(P, X, bf16=True)
    _check_forward(Y, Ye, "B=%d" % B)
    # Against the unrounded FP64 network: the bfloat16 rounding itself (a few
    # ulps through four layers), per row.
    Y64, _ = M.forward(P, X, bf16=False)
    assert np.max(_rel_rows(Y, Y64[:, :160])) < 3e-2
    net.close()


def test_forward_at_maximum_batch_sampled(stp):
    rng = np.random.default_rng(7)
    P = M.init_params(rng)
    B = 65536
    X = _inputs(rng, B)
    net = stp.Mlp(B)
    net.set_params(stp.flatten_params(P))
    Y = net.forward(X).astype(np.float64)
    idx = np.r_[0, 1, 127, 128, rng.integers(0, B, size=250), B - 129, B - 1]
    Ye, _ = M.forward(P, X[idx], bf16=True)
    _check_forward(Y[idx], Ye, "B=65536 sampled")
    net.close()


# 37 and 300: one split of the weight-gradient products over a ragged batch;
# 20000: 314 K stages of 64 batch rows in 63 splits, and 314 work units of the
# resident-weight products (two or three per CTA).
@pytest.mark.parametrize("B", [37, 300, 20000])
def test_gradients_match_oracle(stp, B):
    rng = np.random.default_rng(20 + B)
    P = M.init_params(rng)
    X = _inputs(rng, B)
    T = _targets(rng, X)
    net = stp.Mlp(max(512, B))
    net.set_params(stp.flatten_params(P))
    loss, g = net.gradients(X, T)
    y, cache = M.forward(P, X, bf16=True)
    Ls, dy = M.loss(y, T)
    G = M.backward(P, cache, dy, bf16=True)
    assert abs(loss - Ls.mean()) <= M.RTOL_FWD * abs(Ls.mean())
    Gg = stp.unflatten_params(g)
    worst = {}
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        ref = G[k][:Gg[k].shape[0]]
        if k in ("W4", "b4"):
            # Output rows per slice: mixture logits, means, log-sds, waypoints.
            for name, a, b in M.OUT_SLICES[:4]:
                ok, w = M.close_elementwise(Gg[k][a:b], ref[a:b], M.RTOL_BWD)
                worst[k + "." + name] = round(w, 4)
                assert ok, (k, name, w)
        else:
            ok, w = M.close_elementwise(Gg[k], ref, M.RTOL_BWD)
            worst[k] = round(w, 4)
            assert ok, (k, w)
    print("B=%d worst |err|/tol per gradient:" % B, worst)
    net.close()


def test_first_adam_step_against_oracle(stp):
    rng = np.random.default_rng(3)
    P = M.init_params(rng)
    X = _inputs(rng, 256)
    T = _targets(rng, X)
    net = stp.Mlp(256)
    net.set_params(stp.flatten_params(P))
    lr = 1e-3
    net.train_step(X, T, lr)
    P1 = stp.unflatten_params(net.get_params())
    y, cache = M.forward(P, X, bf16=True)
    _, dy = M.loss(y, T)
    G = M.backward(P, cache, dy, bf16=True)
    Pe = {k: v.copy() for k, v in P.items()}
    M.adam_step(Pe, G, M.adam_init(Pe), 1, lr)
    for k in P1:
        g = G[k][:P1[k].shape[0]]
        sure = np.abs(g) > 0.05 * np.abs(g).max()      # sign of the step is unambiguous
        d_gpu = (P1[k] - np.float32(P[k][:P1[k].shape[0]]))[sure]
        d_ref = (Pe[k][:P1[k].shape[0]] - P[k][:P1[k].shape[0]])[sure]
        assert np.allclose(d_gpu, d_ref, rtol=0, atol=2e-4 * lr / 1e-3 + 1e-7), k
    net.close()


def test_training_lowers_heldout_loss(stp):
    rng = np.random.default_rng(4)
    P = M.init_params(rng)
    Xtr, Xte = _inputs(rng, 4096), _inputs(rng, 512)
    Ttr, Tte = _targets(rng, Xtr), _targets(rng, Xte)
    net = stp.Mlp(4096)
    net.set_params(stp.flatten_params(P))
    before = M.batch_loss(stp.unflatten_params(net.get_params()), Xte, Tte)
    for it in range(300):
        idx = rng.integers(0, 4096, size=1024)
        net.train_step(Xtr[idx], Ttr[idx], 1e-3)
    after = M.batch_loss(stp.unflatten_params(net.get_params()), Xte, Tte)
    assert after < 0.5 * before, (before, after)
    net.close()


def test_gradients_and_steps_are_reproducible(stp):
    """The backward pass runs on two streams (weight gradients beside the input
    gradients) and the forward products as dependent launches: two gradient
    evaluations of the same batch, and two networks trained identically,
    agree bit for bit (no order-dependent reductions, no races)."""
    rng = np.random.default_rng(77)
    B = 20000
    P = M.init_params(rng)
    X = _inputs(rng, B)
    T = _targets(rng, X)
    nets = [stp.Mlp(B), stp.Mlp(B)]
    for net in nets:
        net.set_params(stp.flatten_params(P))
    l0, g0 = nets[0].gradients(X, T)
    l1, g1 = nets[0].gradients(X, T)
    assert l0 == l1 and np.array_equal(g0, g1)
    for net in nets:
        for _ in range(3):
            net.train_step(X, T, 1e-3)
    p0, p1 = nets[0].get_params(), nets[1].get_params()
    assert np.array_equal(p0, p1)
    assert not np.array_equal(p0, stp.flatten_params(P))
    for net in nets:
        net.close()


def test_profiling_intervals(stp):
    """With profiling on, every training step yields one whole-step interval
    and the GEMM intervals inside it (forward chain, backward pass) take less
    device time than the whole step; turning profiling off records nothing."""
    rng = np.random.default_rng(5)
    B = 4096
    P = M.init_params(rng)
    X = _inputs(rng, B)
    T = _targets(rng, X)
    net = stp.Mlp(B)
    net.set_params(stp.flatten_params(P))
    net.train_step(X, T, 1e-3)
    assert net.profile_step() == (0.0, 0)
    net.set_profiling(True)
    for _ in range(3):
        net.train_step(X, T, 1e-3)
    gms, gfl, gby = net.profile()
    sms, n = net.profile_step()
    assert n == 3 and sms > 0 and 0 < gms < sms
    assert gfl > 0 and gby > 0
    assert net.profile_step() == (0.0, 0)     # read and cleared
    net.set_profiling(False)
    net.train_step(X, T, 1e-3)
    assert net.profile_step() == (0.0, 0) and net.profile()[0] == 0.0
    net.close()
