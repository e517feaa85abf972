"""Oracle pins for forward kinematics, obstacle motion and collision checks.

Pinned against values fixed by geometry, not by the oracle's own formulas:
  * UR5e zero pose: with the published standard DH table the flange sits at
    (a2 + a3, -(d4 + d6), d1 - d5) (derived by hand from the frame chain);
  * a planar two-link arm has the textbook closed form
    x = a1 cos q1 + a2 cos(q1+q2), y = a1 sin q1 + a2 sin(q1+q2);
  * any FK pose is a rigid transform and preserves DH link offsets;
  * obstacles interpolate linearly between waypoints and hold outside them
    (Sec. "Simulation Protocol"; holding is a reading);
  * a point/sphere moving linearly against a linearly moving sphere has
    squared distance quadratic in t, minimised in closed form;
  * a one-link arm sweeping an arc vs a static sphere: closest approach in
    closed form.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as WL


def _point_problem(discs, radius=0.0, dof=2, qlo=-10.0, qhi=10.0, vmax=1.0):
    """discs: list of (r, waypoints [(t, x, y, z)...])."""
    K = max(len(w) for _, w in discs)
    way = np.zeros((len(discs), K, 4))
    for m, (_, w) in enumerate(discs):
        w = list(w) + [w[-1]] * (K - len(w))
        way[m] = np.array(w, dtype=float)
        for k in range(len(discs[m][1]), K):   # pad with increasing times
            way[m, k, 0] = way[m, k - 1, 0] + 1.0
    return WL.Problem(dof=dof, arm=False, dh=None, qlo=np.full(dof, qlo), qhi=np.full(dof, qhi),
                      spheres=np.array([[0, 0, 0, 0, radius]]), vmax=vmax,
                      obs_r=np.array([r for r, _ in discs], dtype=float), way=way,
                      qs=np.zeros(dof), qg=np.ones(dof))


def _arm_problem(dh, spheres, obstacles=((0.05, [(0, 5, 5, 5)]),)):
    dof = len(dh)
    K = max(len(w) for _, w in obstacles)
    way = np.zeros((len(obstacles), K, 4))
    for m, (_, w) in enumerate(obstacles):
        way[m, :len(w)] = np.array(w, dtype=float)
        for k in range(len(w), K):
            way[m, k] = way[m, k - 1]
            way[m, k, 0] = way[m, k - 1, 0] + 1.0
    return WL.Problem(dof=dof, arm=True, dh=np.array(dh, dtype=float), qlo=np.full(dof, -10.0),
                      qhi=np.full(dof, 10.0), spheres=np.array(spheres, dtype=float), vmax=1.0,
                      obs_r=np.array([r for r, _ in obstacles], dtype=float), way=way,
                      qs=np.zeros(dof), qg=np.zeros(dof))


def test_ur5e_zero_pose_flange():
    prob, _ = WL.ur5e(0, candidate=0)
    _, org, rot = O.fk(prob, np.zeros(6))
    d1, a2, a3, d4, d5, d6 = 0.1625, -0.425, -0.3922, 0.1333, 0.0997, 0.0996
    assert np.allclose(org[-1], [a2 + a3, -(d4 + d6), d1 - d5], atol=1e-12)
    # Flange axes at zero pose: x along base x, y along base -z... z along -y.
    assert np.allclose(rot[-1] @ np.array([0, 0, 1.0]), [0, -1, 0], atol=1e-12)
    assert np.allclose(org[0], 0) and np.allclose(rot[0], np.eye(3))


@pytest.mark.parametrize("q", [(0.3, -1.1), (2.5, 0.7), (-3.0, 3.0)])
def test_planar_two_link_closed_form(q):
    a1, a2 = 0.7, 0.45
    dh = [[a1, 0, 0, 0], [a2, 0, 0, 0]]
    prob = _arm_problem(dh, [[2, 0, 0, 0, 0.1], [1, 0, 0, 0, 0.1], [2, -a2 / 2, 0, 0, 0.1]])
    cen, org, _ = O.fk(prob, np.array(q))
    q1, q2 = q
    tip = [a1 * math.cos(q1) + a2 * math.cos(q1 + q2), a1 * math.sin(q1) + a2 * math.sin(q1 + q2), 0]
    elbow = [a1 * math.cos(q1), a1 * math.sin(q1), 0]
    assert np.allclose(org[2], tip, atol=1e-12)
    assert np.allclose(cen[0], tip, atol=1e-12)
    assert np.allclose(cen[1], elbow, atol=1e-12)
    mid = (np.array(elbow) + np.array(tip)) / 2
    assert np.allclose(cen[2], mid, atol=1e-12)


def test_fk_rigid_and_link_offsets():
    prob, _ = WL.arm7(0, candidate=0)
    rng = np.random.default_rng(7)
    for _ in range(20):
        q = rng.uniform(-math.pi, math.pi, 7)
        _, org, rot = O.fk(prob, q)
        for R in rot:
            assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
            assert abs(np.linalg.det(R) - 1) < 1e-12
        for j in range(7):
            a, _, d, _ = prob.dh[j]
            assert abs(np.linalg.norm(org[j + 1] - org[j]) - math.hypot(a, d)) < 1e-12


def test_sphere_centres_follow_their_frame():
    prob, _ = WL.ur5e(0, candidate=0)
    q = np.array([0.4, -1.0, 0.9, 0.2, -0.5, 1.7])
    cen, org, rot = O.fk(prob, q)
    for s, sp in enumerate(prob.spheres):
        j = int(sp[0])
        assert np.allclose(cen[s], rot[j] @ sp[1:4] + org[j], atol=1e-12)


def test_obstacle_interpolation_and_hold():
    w = [(1.0, 0, 0, 0), (3.0, 2, 4, -2), (4.0, 2, 4, 6)]
    prob = _point_problem([(0.1, w)])
    assert np.allclose(O.obstacle_position(prob, 0, 0.0), [0, 0, 0])      # hold first
    assert np.allclose(O.obstacle_position(prob, 0, 2.0), [1, 2, -1])     # midway leg 1
    assert np.allclose(O.obstacle_position(prob, 0, 3.0), [2, 4, -2])     # waypoint
    assert np.allclose(O.obstacle_position(prob, 0, 3.25), [2, 4, 0])     # quarter of leg 2
    assert np.allclose(O.obstacle_position(prob, 0, 9.0), [2, 4, 6])      # hold last


def test_point_clearance_closed_form():
    prob = _point_problem([(0.25, [(0, 1.0, 2.0, 0.0)])], radius=0.05)
    free, clr = O.state_free(prob, np.array([1.3, 2.4]), 0.0)
    assert free and abs(clr - (0.5 - 0.3)) < 1e-12
    free, clr = O.state_free(prob, np.array([1.0, 2.29]), 0.0)
    assert (not free) and abs(clr - (0.29 - 0.3)) < 1e-12
    # Touching is free (strict inequality); exactly representable values.
    touch = _point_problem([(0.25, [(0, 0.0, 0.0, 0.0)])], radius=0.25)
    free, clr = O.state_free(touch, np.array([0.5, 0.0]), 0.0)
    assert free and clr == 0.0
    free, clr = O.state_free(touch, np.array([0.4375, 0.0]), 0.0)
    assert (not free) and clr == -0.0625
    # Out of the configuration box collides.
    free, _ = O.state_free(prob, np.array([11.0, 0.0]), 0.0)
    assert not free


def _quadratic_min_clearance(p0, v, t0, t1, rsum):
    """min over t in [t0,t1] of |p0 + v t| - rsum for relative motion p(t)."""
    vv = float(v @ v)
    ts = t0 if vv == 0 else min(max(-float(p0 @ v) / vv, t0), t1)
    return float(np.linalg.norm(p0 + v * ts)) - rsum


def test_edge_check_matches_moving_sphere_quadratic():
    rng = np.random.default_rng(3)
    agree = 0
    for trial in range(200):
        o0 = rng.uniform(-1, 1, 2)
        ov = rng.uniform(-0.5, 0.5, 2)
        r_o, r_p = 0.2, 0.05
        prob = _point_problem([(r_o, [(0.0, *o0, 0.0), (10.0, *(o0 + 10 * ov), 0.0)])], radius=r_p, vmax=1.0)
        qa = rng.uniform(-1, 1, 2)
        qb = qa + rng.uniform(-0.6, 0.6, 2)
        ta = rng.uniform(0, 5)
        tb = ta + max(np.linalg.norm(qb - qa), 0.1) * rng.uniform(1.0, 2.0)
        # Relative position robot - obstacle as a function of absolute time t.
        vq = (qb - qa) / (tb - ta)
        p0 = (qa - vq * ta) - o0     # at t = 0
        vrel = vq - ov
        exact = _quadratic_min_clearance(p0, vrel, ta, tb, r_o + r_p)
        res = 0.001
        v, clr, nc, _ = O.check_edges(prob, qa[None], np.array([ta]), qb[None], np.array([tb]), res)
        # Discrete points are a subset of the segment: clearance >= exact min,
        # and within the sampling error bound (speed * step / 2) of it.
        speed = float(np.linalg.norm(vrel)) * (tb - ta)
        assert clr[0] >= exact - 1e-12
        assert clr[0] - exact <= speed / nc[0] + 1e-12
        if abs(exact) > speed / nc[0] + 1e-9:
            assert bool(v[0]) == (exact >= 0), (trial, exact, clr[0])
            agree += 1
    assert agree > 150


def test_edge_check_arc_of_one_link_arm():
    # One revolute link of length L about z; a sphere at the tip sweeps an arc.
    L, r_tip, r_o = 0.8, 0.05, 0.1
    for ang_obs, expect_free in [(0.5, False), (1.5, True), (-0.2, True)]:
        o = [L * math.cos(ang_obs), L * math.sin(ang_obs), 0.0]
        prob = _arm_problem([[L, 0, 0, 0]], [[1, 0, 0, 0, r_tip]], obstacles=((r_o, [(0, *o)]),))
        qa, qb = np.array([0.0]), np.array([1.0])   # sweep angles 0..1 rad
        v, clr, nc, _ = O.check_edges(prob, qa[None], np.array([0.0]), qb[None], np.array([1.0]), 0.001)
        # Closest approach on the arc: the obstacle angle clamped to the swept range.
        near = min(max(ang_obs, 0.0), 1.0)
        if near == 0.0:          # the start state itself is not among the check points
            near = 0.001
        tip = np.array([L * math.cos(near), L * math.sin(near), 0.0])
        exact = float(np.linalg.norm(tip - np.array(o))) - r_tip - r_o
        assert bool(v[0]) == expect_free
        assert abs(clr[0] - exact) < 1e-3


def test_check_count_and_points():
    # Exactly representable: D = 5 (3-4-5), dt = 3.
    prob = _point_problem([(0.01, [(0, 50, 50, 0)])], vmax=2.0)
    _, _, nc, im = O.check_edges(prob, np.array([[0.0, 0.0]]), np.array([1.0]), np.array([[3.0, 4.0]]),
                                 np.array([4.0]), 0.25)
    assert nc[0] == 24 and abs(im[0] - 1e-3) < 1e-12   # v*dt = 6 dominates D = 5
    prob1 = _point_problem([(0.01, [(0, 50, 50, 0)])], vmax=1.0)
    _, _, nc, _ = O.check_edges(prob1, np.array([[0.0, 0.0]]), np.array([1.0]), np.array([[3.0, 4.0]]),
                                np.array([4.0]), 0.25)
    assert nc[0] == 20                            # D = 5 dominates v*dt = 3
    _, _, nc, im = O.check_edges(prob1, np.array([[0.0, 0.0]]), np.array([1.0]), np.array([[3.0, 4.0]]),
                                 np.array([4.0]), 0.3)
    assert nc[0] == 17 and abs(im[0] - (1 - (5 / 0.3 - 1e-3 - 16))) < 1e-12
    # Within 1e-3 of a step above a multiple of res, the count does not grow.
    _, _, nc, _ = O.check_edges(prob1, np.array([[0.0, 0.0]]), np.array([1.0]), np.array([[3.0, 4.0002]]),
                                np.array([4.0]), 0.25)
    assert nc[0] == 20
    # A zero-length edge in q and t still takes one point.
    _, _, nc, _ = O.check_edges(prob, np.array([[1.0, 1.0]]), np.array([2.0]), np.array([[1.0, 1.0]]),
                                np.array([2.0]), 0.01)
    assert nc[0] == 1
