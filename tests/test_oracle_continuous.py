"""Pins of the oracle's closed-form (continuous) edge validation for point
robots: hand cases whose closest approach is known exactly, a crossing that
the discrete check misses between its samples, agreement with a brute-force
fine grid, and the ordering continuous clearance <= discrete clearance."""
import numpy as np
import pytest

import oracle as O
import workloads as WL


def _problem(way, obs_r, r_robot=0.05, lo=(-2.0, -2.0), hi=(2.0, 2.0), vmax=2.0):
    return WL.Problem(dof=2, arm=False, dh=None, qlo=np.array(lo), qhi=np.array(hi),
                      spheres=np.array([[0, 0.0, 0.0, 0.0, r_robot]]), vmax=vmax,
                      obs_r=np.asarray(obs_r, float), way=np.asarray(way, float),
                      qs=np.zeros(2), qg=np.zeros(2))


def test_static_disc_closest_approach():
    # robot along x from (-1, 0) to (1, 0) over [0, 2]; disc at (0, 0.3), r 0.1
    way = np.array([[[0.0, 0.0, 0.3, 0.0]]])
    P = _problem(way, [0.1])
    v, clr = O.check_edges_continuous(P, [[-1.0, 0.0]], [0.0], [[1.0, 0.0]], [2.0])
    assert v[0] == 1 and abs(clr[0] - 0.15) < 1e-15
    way[0, 0, 2] = 0.12
    P = _problem(way, [0.1])
    v, clr = O.check_edges_continuous(P, [[-1.0, 0.0]], [0.0], [[1.0, 0.0]], [2.0])
    assert v[0] == 0 and abs(clr[0] + 0.03) < 1e-15


def test_touching_is_free_and_box_ends_checked():
    way = np.array([[[0.0, 0.0, 0.375, 0.0]]])         # clearance exactly 0 (binary fractions)
    P = _problem(way, [0.25], r_robot=0.125)
    v, clr = O.check_edges_continuous(P, [[-1.0, 0.0]], [0.0], [[1.0, 0.0]], [2.0])
    assert v[0] == 1 and abs(clr[0]) < 1e-15
    P = _problem(np.array([[[0.0, 5.0, 5.0, 0.0]]]), [0.1], hi=(0.5, 2.0))
    v, _ = O.check_edges_continuous(P, [[-1.0, 0.0]], [0.0], [[1.0, 0.0]], [2.0])
    assert v[0] == 0                                    # leaves the box at its end


def test_crossing_between_discrete_samples():
    """Robot x(t) = -1 + t on [0, 2]; obstacle on y from (0.25, -1) at t = 0.25
    to (0.25, 1) at t = 2.25 (held before): both are at (0.25, 0) at t = 1.25,
    between the discrete samples t = 1.0 and 1.5 of res = 0.5."""
    way = np.array([[[0.25, 0.25, -1.0, 0.0], [2.25, 0.25, 1.0, 0.0]]])
    P = _problem(way, [0.05], r_robot=0.05, vmax=1.0)
    v, clr = O.check_edges_continuous(P, [[-1.0, 0.0]], [0.0], [[1.0, 0.0]], [2.0])
    assert v[0] == 0 and abs(clr[0] + 0.1) < 1e-12
    vd, cd, nc, _ = O.check_edges(P, np.array([[-1.0, 0.0]]), np.array([0.0]), np.array([[1.0, 0.0]]),
                                  np.array([2.0]), 0.5)
    assert nc[0] == 4 and vd[0] == 1 and cd[0] > 0.0


def _random_case(seed, n=300):
    rng = np.random.default_rng(seed)
    K, M = 4, 6
    way = np.zeros((M, K, 4))
    for m in range(M):
        way[m, :, 0] = np.sort(rng.uniform(0, 10, size=K))
        way[m, :, 1:3] = rng.uniform(-1, 1, size=(K, 2))
    P = _problem(way, rng.uniform(0.05, 0.2, size=M), r_robot=0.03)
    qa = rng.uniform(-1, 1, size=(n, 2))
    step = rng.normal(size=(n, 2))
    step *= (rng.uniform(0.05, 0.6, size=n) / np.linalg.norm(step, axis=1))[:, None]
    qb = qa + step
    ta = rng.uniform(0, 9, size=n)
    tb = ta + np.linalg.norm(step, axis=1) / 2.0 * rng.uniform(1.0, 3.0, size=n)
    return P, qa, ta, qb, tb


@pytest.mark.parametrize("seed", [0, 1])
def test_agrees_with_a_fine_grid(seed):
    P, qa, ta, qb, tb = _random_case(seed)
    v, clr = O.check_edges_continuous(P, qa, ta, qb, tb)
    vf, cf, _, _ = O.check_edges(P, qa, ta, qb, tb, 1e-4)
    assert np.all(clr <= cf + 1e-12)          # the exact minimum is below every sample
    assert np.all(cf - clr < 2e-4)            # and within the fine grid's spacing
    near = np.abs(clr) < 2e-4
    assert np.array_equal(v[~near], vf[~near])


@pytest.mark.parametrize("seed", [2, 3])
def test_continuous_is_never_less_strict_than_discrete(seed):
    P, qa, ta, qb, tb = _random_case(seed)
    v, clr = O.check_edges_continuous(P, qa, ta, qb, tb)
    vd, cd, _, _ = O.check_edges(P, qa, ta, qb, tb, 0.01)
    assert np.all(clr <= cd + 1e-12)
    assert not np.any((v == 1) & (vd == 0))
