"""Host-side logic of the learned-proposal experiment (no GPU): the
final-trajectory-cost accounting of collided episodes, the guidance path
planned around the static boxes, and its lookahead point."""
import math

import numpy as np

from paper_2605_29663_gb300 import learned as L


def test_collided_robot_pays_its_own_remaining_steps():
    cost = np.array([100.0, 200.0, 300.0, 400.0])
    collided = np.array([True, False, True, False])
    t_coll = np.array([30, 250, 240, 250])
    dist = np.array([5.0, 0.2, 1.5, 7.0])
    out = L.collided_remainder(cost, collided, t_coll, dist, 250, 2.0)
    # robot 0: 2 * 5 m * 220 steps; robot 2: 2 * 1.5 m * 10 steps; the others unchanged
    np.testing.assert_allclose(out, [100.0 + 2200.0, 200.0, 300.0 + 30.0, 400.0])


def test_collision_at_the_last_step_adds_nothing():
    out = L.collided_remainder(np.array([50.0]), np.array([True]), np.array([250]), np.array([3.0]), 250, 1.0)
    assert out[0] == 50.0


def test_plan_path_keeps_the_margin_around_a_box():
    box = (4.0, 0.0, 1.0, 1.0)            # centre, width, height
    path = L.plan_path([box], (0.0, 0.0), (8.0, 0.0), (-4.0, -9.0), (12.0, 9.0))
    assert np.allclose(path[0], (0.0, 0.0)) and np.allclose(path[-1], (8.0, 0.0))
    inner = path[1:-1]
    dx = np.maximum(np.abs(inner[:, 0] - box[0]) - box[2] / 2, 0.0)
    dy = np.maximum(np.abs(inner[:, 1] - box[1]) - box[3] / 2, 0.0)
    assert np.hypot(dx, dy).min() > L.INFLATE        # every cell centre on the path is outside the blocked band
    steps = np.hypot(*np.diff(inner, axis=0).T)
    assert steps.max() <= L.GRID * math.sqrt(2) + 1e-9   # 8-connected grid moves


def test_plan_path_without_obstacles_is_straight():
    path = L.plan_path([], (0.0, 0.0), (6.0, 0.0), (-4.0, -9.0), (10.0, 9.0))
    assert np.abs(path[:, 1]).max() <= L.GRID / 2 + 1e-9


def test_lookahead_point_along_the_path():
    path = np.array([(0.0, 0.0), (2.0, 0.0), (2.0, 5.0)])
    # 3 m along the path from vertex 0: 2 m on the first segment, 1 m up the second
    np.testing.assert_allclose(L.lookahead_point(path, (0.1, 0.0)), (2.0, 1.0))
    # near the end the last point is returned
    np.testing.assert_allclose(L.lookahead_point(path, (2.0, 4.9)), (2.0, 5.0))
