"""Pins of the oracle's learned sampling branch (no GPU): the learned coin is
the integer threshold on the slot-12 Philox word, learned q_r stay inside the
clipped window around the drawn waypoint with the uniform window's moments,
mixture goal times follow the mixture (moments of a single component and the
component weights of two), and waypoints map onto the joint box."""
import ctypes as C

import numpy as np

import oracle

SEED, PID = 12345, 3


def _y(mu=0.5, logsd=-3.0, logits=None, wp=None):
    y = np.zeros(160)
    y[0:8] = -50.0 if logits is None else logits
    if logits is None:
        y[0] = 50.0
    y[8:16] = mu
    y[16:24] = logsd
    if wp is not None:
        y[24:152] = wp
    return y


def _philox_word(k, w, slot):
    ctr = (C.c_uint * 4)(slot // 4, w, k, PID)
    key = (C.c_uint * 2)(SEED & 0xFFFFFFFF, SEED >> 32)
    out = (C.c_uint * 4)()
    oracle.lib().orc_philox4x32_10(ctr, key, out)
    return out[slot % 4]


def test_learned_coin_is_the_slot12_threshold():
    lo, hi = -np.ones(6), np.ones(6)
    n, hits = 4000, 0
    for w in range(n):
        f, _, _, _ = oracle.learned_sample(_y(), lo, hi, 10.0, SEED, PID, 7, w)
        assert f == ((_philox_word(7, w, 12) >> 8) < 15099495)
        hits += f
    p = hits / n
    assert abs(p - 0.9) < 4 * np.sqrt(0.09 / n)


def test_learned_q_window_and_moments():
    lo, hi = np.array([-np.pi] * 7), np.array([np.pi] * 7)
    wp = np.zeros(128)
    rng = np.random.default_rng(0)
    wp[:] = rng.uniform(-0.7, 0.7, size=128)
    wp.reshape(16, 8)[3, 0] = 0.99        # waypoint 3 near the upper joint limit: clipped window
    y = _y(wp=wp)
    half = 0.1 * (hi - lo)
    devs = []
    for w in range(3000):
        f, i, q, _ = oracle.learned_sample(y, lo, hi, 10.0, SEED, PID, 1, w)
        if not f:
            assert np.all((q >= lo) & (q <= hi))
            continue
        c = lo + (np.clip(wp.reshape(16, 8)[i, :7], -1, 1) + 1) * 0.5 * (hi - lo)
        assert np.all(q >= np.maximum(c - half, lo) - 1e-12) and np.all(q <= np.minimum(c + half, hi) + 1e-12)
        if i != 3:
            devs.append((q - c) / half)
    d = np.array(devs)
    assert abs(d.mean()) < 0.03 and abs(d.var() - 1 / 3) < 0.02    # U(-1, 1): mean 0, variance 1/3


def test_single_component_goal_time_moments():
    H, mu, lsd = 20.0, 0.4, -2.5
    lo, hi = -np.ones(2), np.ones(2)
    T = []
    for w in range(20000):
        f, _, _, t = oracle.learned_sample(_y(mu, lsd), lo, hi, H, SEED, PID, 2, w)
        if f:
            T.append(t)
    T = np.array(T)
    sd = np.exp(lsd) * H
    assert abs(T.mean() - mu * H) < 4 * sd / np.sqrt(len(T))
    assert abs(T.std() / sd - 1) < 0.03
    assert abs(np.mean(np.abs(T - mu * H) < sd) - 0.6827) < 0.02


def test_two_equal_components():
    H = 10.0
    logits = np.full(8, -50.0)
    logits[2] = logits[5] = 0.0
    y = _y(logits=logits)
    y[8 + 2], y[8 + 5] = 0.2, 0.8
    y[16:24] = -6.0
    lo, hi = -np.ones(2), np.ones(2)
    T = np.array([t for f, _, _, t in (oracle.learned_sample(y, lo, hi, H, SEED, PID, 3, w) for w in range(6000))
                  if f])
    near2 = np.abs(T - 2.0) < 0.1
    near8 = np.abs(T - 8.0) < 0.1
    assert np.all(near2 | near8)
    assert abs(near2.mean() - 0.5) < 4 * np.sqrt(0.25 / len(T))


def test_waypoint_denormalisation_clips_to_the_box():
    lo, hi = np.array([0.0, -2.0]), np.array([1.0, 2.0])
    wp = np.zeros(128)
    wp.reshape(16, 8)[:, 0] = 5.0          # beyond +1: upper bound
    wp.reshape(16, 8)[:, 1] = -1.0         # lower bound
    for w in range(400):
        f, i, q, _ = oracle.learned_sample(_y(wp=wp), lo, hi, 5.0, SEED, PID, 4, w)
        if f:
            assert 1.0 - 0.1 * 1.0 - 1e-12 <= q[0] <= 1.0
            assert -2.0 <= q[1] <= -2.0 + 0.1 * 4.0 + 1e-12


def test_zero_offsets_put_waypoints_on_the_straight_line():
    lo, hi = np.array([-np.pi] * 6), np.array([np.pi] * 6)
    qs, qg = np.full(6, -1.0), np.array([2.0, 0.5, -0.3, 1.0, 0.0, 2.5])
    half = 0.1 * (hi - lo)
    seen = set()
    for w in range(2000):
        f, i, q, _ = oracle.learned_sample(_y(), lo, hi, 10.0, SEED, PID, 5, w, qs=qs, qg=qg)
        if not f:
            continue
        c = qs + (i + 1) / 17 * (qg - qs)
        assert np.all(np.abs(q - c) <= half + 1e-12)
        seen.add(i)
    assert seen == set(range(16))
