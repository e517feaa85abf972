"""Pins of the FP64 proposal-network reference (no GPU): finite differences,
the closed-form Gaussian NLL, softmax shift invariance, an identity network,
the first Adam step, bfloat16 rounding and the path targets."""
import math

import numpy as np
import pytest

from oracle import mlp as M
import workloads as WL


def _batch(rng, B=5):
    X = rng.normal(size=(B, M.IN))
    T = np.zeros((B, M.N_TGT))
    T[:, 0] = rng.uniform(0.1, 0.9, size=B)
    T[:, 1:-1] = rng.uniform(-1, 1, size=(B, M.N_WP * M.WP_DIM))
    T[:, -1] = rng.choice([2, 6, 7], size=B)
    return X, T


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    P = M.init_params(rng)
    # larger biases so that ReLUs are away from their kinks for the step used
    for b in ("b1", "b2", "b3"):
        P[b] = rng.normal(scale=0.3, size=P[b].shape)
    X, T = _batch(rng)
    y, cache = M.forward(P, X)
    _, dy = M.loss(y, T)
    G = M.backward(P, cache, dy)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b3", "W4", "b4"):
        A = P[name]
        idx = [tuple(rng.integers(0, s) for s in A.shape) for _ in range(6)]
        if name in ("W4", "b4"):
            idx = [(i[0] % M.OUT_USED,) + i[1:] for i in idx]
        for i in idx:
            old = A[i]
            A[i] = old + h
            lp = M.batch_loss(P, X, T)
            A[i] = old - h
            lm = M.batch_loss(P, X, T)
            A[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[name][i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, G[name][i])


def test_mixture_of_identical_components_is_one_gaussian():
    rng = np.random.default_rng(2)
    B = 4
    y = np.zeros((B, M.OUT))
    mu, s = rng.uniform(0.2, 0.8, size=B), rng.uniform(-3, 0, size=B)
    y[:, 0:8] = rng.normal(size=(B, 1))            # equal logits per row
    y[:, 8:16] = mu[:, None]
    y[:, 16:24] = s[:, None]
    T = np.zeros((B, M.N_TGT))
    T[:, 0] = rng.uniform(0, 1, size=B)
    T[:, -1] = 7
    T[:, 1:-1] = y[:, 24:152]                       # waypoint term zero
    L, dy = M.loss(y, T)
    z = (T[:, 0] - mu) / np.exp(s)
    assert np.allclose(L, 0.5 * z * z + s + 0.5 * math.log(2 * math.pi), rtol=0, atol=1e-12)
    # d/dmu of the Gaussian NLL is -z/sigma, d/ds is 1 - z^2 (batch mean: / B)
    assert np.allclose(dy[:, 8:16].sum(axis=1) * B, -z / np.exp(s), atol=1e-12)
    assert np.allclose(dy[:, 16:24].sum(axis=1) * B, 1 - z * z, atol=1e-12)
    assert np.allclose(dy[:, 0:8], 0.0, atol=1e-15)


def test_logit_shift_invariance():
    rng = np.random.default_rng(3)
    y = rng.normal(size=(3, M.OUT))
    T = _batch(rng, 3)[1]
    L0, dy = M.loss(y, T)
    y2 = y.copy()
    y2[:, 0:8] += 5.0
    L1, _ = M.loss(y2, T)
    assert np.allclose(L0, L1, atol=1e-12)
    assert np.allclose(dy[:, 0:8].sum(axis=1), 0.0, atol=1e-15)


def test_identity_network():
    """W1 = [I; -I], W2 = W3 = I, W4 = [I, -I]: y = relu(x) - relu(-x) = x."""
    P = {k: np.zeros_like(v) for k, v in M.init_params(np.random.default_rng(0)).items()}
    P["W1"][0:32, 0:32] = np.eye(32)
    P["W1"][32:64, 0:32] = -np.eye(32)
    P["W2"][:] = np.eye(256)
    P["W3"][:] = np.eye(256)
    P["W4"][0:32, 0:32] = np.eye(32)
    P["W4"][0:32, 32:64] = -np.eye(32)
    X = np.random.default_rng(4).normal(size=(6, 32))
    y, _ = M.forward(P, X)
    assert np.array_equal(y[:, 0:32], X)
    assert np.array_equal(y[:, 32:], np.zeros((6, M.OUT - 32)))


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(5)
    P = M.init_params(rng)
    G = {k: rng.normal(size=v.shape) for k, v in P.items()}
    G["W4"][M.OUT_USED:] = 0.0
    G["b4"][M.OUT_USED:] = 0.0
    P0 = {k: v.copy() for k, v in P.items()}
    st = M.adam_init(P)
    M.adam_step(P, G, st, 1, lr=1e-3)
    for k in P:
        assert np.allclose(P[k] - P0[k], -1e-3 * G[k] / (np.abs(G[k]) + 1e-8), rtol=1e-12, atol=1e-15)


def test_bf16_round():
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -2.5, 3.0e38])
    r = M.bf16_round(x)
    assert list(r[:5]) == [1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -2.5]
    assert abs(r[5] - 3.0e38) / 3.0e38 < 2.0 ** -8


def test_path_targets_on_a_straight_path():
    lo, hi = -np.pi * np.ones(6), np.pi * np.ones(6)
    qs, qg = np.full(6, -1.0), np.full(6, 2.0)
    U, H = 8.0, 16.0
    path = np.array([np.r_[qs, 0.0], np.r_[0.5 * (qs + qg), 4.0], np.r_[qg, U]])
    T = M.path_targets(path, U, H, 6, lo, hi)
    assert T[0] == 0.5 and T[-1] == 6
    for i in range(16):
        f = (i + 1) / 17
        o = 1 + 8 * i
        # a constant-speed straight path has zero offsets from the line
        assert np.allclose(T[o:o + 6], 0.0, atol=1e-15)
        assert T[o + 6] == 0.0
        assert abs(T[o + 7] - f * U / H) < 1e-15
    # a detour through a middle state q_m at t = 4: offsets of the piecewise path
    qm = np.array([1.0, 0.0, 0.5, -0.5, 2.0, 0.3])
    path = np.array([np.r_[qs, 0.0], np.r_[qm, 4.0], np.r_[qg, U]])
    T = M.path_targets(path, U, H, 6, lo, hi)
    for i in range(16):
        f = (i + 1) / 17
        t = f * U
        q = qs + (t / 4.0) * (qm - qs) if t <= 4.0 else qm + ((t - 4.0) / 4.0) * (qg - qm)
        assert np.allclose(T[1 + 8 * i:7 + 8 * i], (q - (qs + f * (qg - qs))) / np.pi, atol=1e-14)


def test_features_of_a_hand_made_problem():
    prob, prm = WL.ur5e(0)
    x = M.features(prob, prm.H)
    assert np.allclose(x[0:6], prob.qs / np.pi) and np.allclose(x[7:13], prob.qg / np.pi)
    assert x[6] == 0 and x[13] == 0 and list(x[14:17]) == [0, 1, 0]
    way = np.asarray(prob.way)
    assert np.allclose(x[17:20], way[:, 0, 1:4].mean(axis=0))
    v = (way[:, -1, 1:4] - way[:, 0, 1:4]) / (way[:, -1, 0] - way[:, 0, 0])[:, None]
    assert np.allclose(x[20:23], v.mean(axis=0)) and x[23] == pytest.approx(0.06)
    assert x[24] == prm.H / 60
    assert x[25] == pytest.approx(np.linalg.norm(prob.qg - prob.qs) / prob.vmax / prm.H)
    assert np.all(x[26:] == 0)
