"""The synthetic input recipe (stand-ins for the paper's suites): every
generator produces the stated shapes, sizes and value ranges, reproducibly."""
import math

import numpy as np
import pytest

import workloads as WL


def _legs(way):
    """Per-leg speeds and time steps of [M][K][4] waypoint paths."""
    dt = np.diff(way[:, :, 0], axis=1)
    dx = np.linalg.norm(np.diff(way[:, :, 1:4], axis=1), axis=2)
    return dx / dt, dt


def test_disc2d_recipe():
    prob, prm = WL.disc2d(0)
    assert prob.dof == 2 and not prob.arm and prob.vmax == 0.5
    assert np.array_equal(prob.qs, [0.05, 0.05]) and np.array_equal(prob.qg, [0.95, 0.95])
    assert prob.way.shape == (8, 2, 4) and np.all(prob.obs_r == 0.05)
    p0 = prob.way[:, 0, 1:3]
    assert np.all((p0 >= 0) & (p0 <= 1))
    assert np.all(np.linalg.norm(p0 - prob.qs, axis=1) >= 0.1)
    assert np.all(np.linalg.norm(p0 - prob.qg, axis=1) >= 0.1)
    vel = (prob.way[:, 1, 1:3] - p0) / prm.H
    assert np.all(np.abs(vel) <= 0.1 + 1e-12)
    assert (prm.variant, prm.n_roots, prm.workers, prm.max_iters) == (0, 4, 64, 2000)
    assert (prm.eta, prm.res, prm.dt, prm.H) == (0.1, 0.01, 0.02, 20.0)


def test_ur5e_recipe():
    prob, prm = WL.ur5e(0)
    assert prob.dof == 6 and prob.arm and abs(prob.vmax - math.pi / 2) < 1e-15
    assert np.allclose(prob.dh[:, 2], [0.1625, 0, 0, 0.1333, 0.0997, 0.0996])
    assert np.allclose(prob.dh[:, 0], [0, -0.425, -0.3922, 0, 0, 0])
    assert np.allclose(prob.dh[:, 1], [math.pi / 2, 0, 0, math.pi / 2, -math.pi / 2, 0])
    assert prob.spheres.shape == (32, 5) and np.all(prob.spheres[:, 4] == 0.05)
    assert prob.way.shape == (16, 4, 4) and np.all(prob.obs_r == 0.06)
    assert np.all(np.abs(prob.way[:, :, 1:4]) <= 0.6 + 1e-12)
    speed, dt = _legs(prob.way)
    assert np.all(dt > 0) and np.all(speed <= 0.5 + 1e-9)
    assert np.allclose(prob.way[:, 0, 0], 0.0) and np.allclose(prob.way[:, -1, 0], 15.0)
    assert np.all(np.abs(prob.qs) <= math.pi) and np.all(np.abs(prob.qg) <= math.pi)
    assert (prm.variant, prm.n_roots, prm.workers, prm.eta, prm.H) == (1, 8, 1024, 0.5, 15.0)


def test_arm7_recipe():
    prob, prm = WL.arm7(0)
    assert prob.dof == 7 and prob.arm
    assert np.all((prob.dh[:, 2] >= 0.1) & (prob.dh[:, 2] <= 0.4)) and np.all(prob.dh[:, 0] == 0)
    assert np.allclose(prob.dh[:, 1], [math.pi / 2 * (1 if j % 2 == 0 else -1) for j in range(7)])
    assert prob.spheres.shape == (48, 5) and np.all(prob.spheres[:, 4] == 0.04)
    assert prob.way.shape == (64, 8, 4)
    assert np.all((prob.obs_r >= 0.04) & (prob.obs_r <= 0.1))
    speed, dt = _legs(prob.way)
    assert np.all(dt > 0) and np.all(speed <= 0.5 + 1e-9)
    assert (prm.n_roots, prm.workers, prm.H) == (16, 4096, 60.0)


def test_sphere_layout_covers_every_link_on_its_polyline():
    for dh, S in ((WL.UR5E_DH, 32), (WL.arm7_dh(np.random.default_rng(0)), 48)):
        sp = WL.sphere_layout(dh, S, 0.05)
        assert len(sp) == S
        frames = sp[:, 0].astype(int)
        assert set(frames) == set(range(1, len(dh) + 1))
        for row in sp:
            a, alpha, d, _ = dh[int(row[0]) - 1]
            c = row[1:4]
            # on the d-segment (x = -a) or on the a-segment (y = z = 0)
            on_d = abs(c[0] + a) < 1e-12
            on_a = abs(c[1]) < 1e-12 and abs(c[2]) < 1e-12
            assert on_d or on_a


@pytest.mark.parametrize("i", range(9))
def test_mixed_recipe(i):
    prob, prm = WL.mixed(i)
    fam = i % 3
    assert prob.dof == (2, 6, 7)[fam]
    assert 10.0 <= prm.H <= 60.0
    M = len(prob.obs_r)
    assert (4 <= M <= 32) if fam == 0 else (4 <= M <= 128)
    assert prm.problem_id == i


def test_microbench_edges_are_eta_steps_at_max_speed():
    prob, prm = WL.ur5e(0)
    qa, ta, qb, tb = WL.microbench_edges(prob, 4096, prm.eta, prm.H, seed=0)
    D = np.linalg.norm(qb - qa, axis=1)
    assert np.allclose(D, prm.eta, atol=1e-12)
    assert np.all((qb >= prob.qlo) & (qb <= prob.qhi)) and np.all((qa >= prob.qlo) & (qa <= prob.qhi))
    assert np.allclose(tb - ta, D / prob.vmax) and np.all(ta >= 0) and np.all(tb <= prm.H + 1e-12)


def test_generators_are_reproducible():
    a, _ = WL.arm7(3)
    b, _ = WL.arm7(3)
    assert np.array_equal(a.way, b.way) and np.array_equal(a.qs, b.qs) and np.array_equal(a.dh, b.dh)
