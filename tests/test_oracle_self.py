"""Pins of the oracle's self-collision (arms, optional): a planar three-link
arm whose poses put non-adjacent link spheres on top of each other (closed-form
positions), the exclusion of same / adjacent frames and of pairs already
overlapping at the zero configuration, and the UR5e at rest."""
import math

import numpy as np

import oracle as O
import workloads as WL


def _planar(a=(1.0, 1.0, 1.0), r=0.3, self_collision=True):
    dh = np.zeros((3, 4))
    dh[:, 0] = a                                  # a_j; alpha = d = theta0 = 0
    spheres = np.array([[f, 0.0, 0.0, 0.0, r] for f in range(4)])
    return WL.Problem(dof=3, arm=True, dh=dh, qlo=np.full(3, -4.0), qhi=np.full(3, 4.0), spheres=spheres,
                      vmax=1.0, obs_r=np.zeros(0), way=np.zeros((0, 1, 4)), qs=np.zeros(3), qg=np.zeros(3),
                      self_collision=self_collision)


def test_folded_planar_arm_collides_with_itself():
    P = _planar()
    ok, clr = O.state_free(P, np.zeros(3), 0.0)
    assert ok and abs(clr - (2.0 - 0.6)) < 1e-12            # nearest non-adjacent pair: frames 0-2, 1-3
    # q = (0, pi, 0): frame 2 returns to the base
    ok, clr = O.state_free(P, np.array([0.0, math.pi, 0.0]), 0.0)
    assert not ok and abs(clr + 0.6) < 1e-12
    # q = (0, 2pi/3, 2pi/3): an equilateral triangle, frame 3 back at the base
    ok, clr = O.state_free(P, np.array([0.0, 2 * math.pi / 3, 2 * math.pi / 3]), 0.0)
    assert not ok and abs(clr + 0.6) < 1e-12
    # the same poses without self-collision checking are free (no obstacles)
    P0 = _planar(self_collision=False)
    assert O.state_free(P0, np.array([0.0, math.pi, 0.0]), 0.0)[0]


def test_pair_list_excludes_adjacent_frames_and_rest_contacts():
    assert O.self_pairs(_planar()).tolist() == [[0, 2], [0, 3], [1, 3]]
    # a zero-length second link puts frame 2 on frame 1: frames 0 and 2 overlap
    # at rest (distance 0.5 < 0.6), so that pair is ignored
    assert O.self_pairs(_planar(a=(0.5, 0.0, 1.0))).tolist() == [[0, 3], [1, 3]]


def test_ur5e_rest_pose_is_free():
    prob, _ = WL.ur5e(0, n_obs=0)
    prob.self_collision = True
    assert len(O.self_pairs(prob)) > 100
    assert O.state_free(prob, np.zeros(6), 0.0)[0]
