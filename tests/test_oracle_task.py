"""Pins of the oracle's task logic (Sec. III-C, III-D, III-E): collisions,
the differentiable reward R_ctrl, the sparse reward R_goal, termination and
reset, on hand-computed tiny cases."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth


def _scene(p, spheres=(), boxes=(), targets=None, pool=None):
    sp = np.array(spheres, float).reshape(-1, 4)
    bx = np.array(boxes, float).reshape(-1, 6)
    NM = p["n_env"] * p["n_agent"]
    D = synth.STATE_DIM[p["model"]]
    return dict(spheres=sp, sph_off=np.array([0, len(sp)], np.int32), boxes=bx,
                box_off=np.array([0, len(bx)], np.int32),
                env_map=np.zeros(p["n_env"], np.int32),
                targets=np.zeros((NM, 3)) if targets is None else np.array(targets, float),
                pool=np.zeros((p["pool_size"], NM, D)) if pool is None else np.array(pool, float))


def _hover_pm(pos, g=9.81):
    s = np.zeros(12)
    s[0:3] = pos
    s[8] = g
    return s


def test_reward_position_task_by_hand():
    # hover in place: R_ctrl = -|p - p*|^2 - 0.01 |a|^2
    p = synth.params(n_env=1, horizon=1, cam=None)
    o = oracle.Oracle(p, _scene(p, targets=[[1.0, 2.0, 2.0]]))
    act = np.array([[[0.0, 0.0, 0.981]]])
    rec = o.rollout(_hover_pm([0, 0, 0])[None], act)
    assert rec["r_ctrl"][0, 0] == pytest.approx(-(1 + 4 + 4) - 0.01 * 0.981 ** 2, abs=1e-12)
    assert rec["r_goal"][0, 0] == 0
    assert rec["done"][0, 0] == 0


def test_reward_avoid_task_by_hand():
    # |e| = 3 (norm, not squared); sphere SDF 0.5 < d_safe = 1: -10 * 0.5^2
    p = synth.params(n_env=1, horizon=1, cam=None, pos_sq=0, w_obs=10.0, d_safe=1.0)
    o = oracle.Oracle(p, _scene(p, spheres=[(2.0, 0, 0, 1.5)], targets=[[0, 3, 0]]))
    act = np.array([[[0.0, 0.0, 0.981]]])
    rec = o.rollout(_hover_pm([0, 0, 0])[None], act)
    assert rec["r_ctrl"][0, 0] == pytest.approx(-3.0 - 10 * 0.25 - 0.01 * 0.981 ** 2, abs=1e-12)
    assert rec["sdf_id"][0, 0] == 0


def test_box_obstacle_term_by_hand():
    p = synth.params(n_env=1, horizon=1, cam=None, pos_sq=0, w_obs=2.0, d_safe=1.0, w_act=0.0)
    o = oracle.Oracle(p, _scene(p, spheres=[(50, 0, 0, 1)], boxes=[(0.6, -1, -1, 2, 1, 1)],
                                targets=[[0, 0, 0]]))
    rec = o.rollout(_hover_pm([0, 0, 0])[None], np.array([[[0, 0, 0.981]]]))
    # SDF to the box face x = 0.6 is 0.6: -2 * (1 - 0.6)^2
    assert rec["r_ctrl"][0, 0] == pytest.approx(-2 * 0.16, abs=1e-12)
    assert rec["sdf_id"][0, 0] == 1


def test_collision_sets_done_goal_and_resets_from_pool():
    p = synth.params(n_env=1, horizon=3, cam=None, terminate=1, pool_size=2, r_quad=0.2)
    pool = np.stack([_hover_pm([5, 5, 5])[None], _hover_pm([-5, -5, -5])[None]])
    o = oracle.Oracle(p, _scene(p, spheres=[(0.5, 0, 0, 0.4)], targets=[[9, 9, 9]], pool=pool))
    act = np.tile(np.array([0, 0, 0.981]), (3, 1, 1))
    rec = o.rollout(_hover_pm([0, 0, 0])[None], act)
    # SDF 0.1 < r_quad: collision at step 0, reset to pool[0]
    assert rec["done"][0, 0] == 1 and rec["r_goal"][0, 0] == -1
    np.testing.assert_allclose(rec["states"][1, 0], pool[0, 0])
    assert rec["done"][1, 0] == 0
    assert rec["pool_k"][0] == 1


def test_success_reward():
    p = synth.params(n_env=1, horizon=1, cam=None, success_radius=0.5)
    o = oracle.Oracle(p, _scene(p, targets=[[0.3, 0, 0]]))
    rec = o.rollout(_hover_pm([0, 0, 0])[None], np.array([[[0, 0, 0.981]]]))
    assert rec["r_goal"][0, 0] == 1


def test_bounds_collision():
    p = synth.params(n_env=1, horizon=1, cam=None, terminate=1, bound_lo=(-9, -9, 0.0),
                     bound_hi=(9, 9, 10.0))
    o = oracle.Oracle(p, _scene(p))
    s = _hover_pm([0, 0, 0.0001])
    s[5] = -1.0  # falling through the floor within one step (dt v = -0.01)
    rec = o.rollout(s[None], np.array([[[0, 0, 0.981]]]))
    assert rec["done"][0, 0] == 1


def test_swarm_pair_terms_and_env_reset():
    # 3 agents; agents 0 and 1 are 0.3 apart (< d_agent = 0.4): both collide,
    # the env resets as a whole; pair penalty -w (0.4 - 0.3)^2 on both
    p = synth.params(n_env=1, n_agent=3, horizon=1, cam=None, terminate=1, w_agent=10.0,
                     d_agent=0.4, w_pos=0.0, w_act=0.0)
    s0 = np.stack([_hover_pm([0, 0, 0]), _hover_pm([0.3, 0, 0]), _hover_pm([5, 0, 0])])
    pool = np.stack([np.stack([_hover_pm([k, 10, 0]) for k in range(3)])] * 4)
    o = oracle.Oracle(p, _scene(p, targets=np.zeros((3, 3)), pool=pool))
    rec = o.rollout(s0, np.tile(np.array([0, 0, 0.981]), (1, 3, 1)))
    np.testing.assert_allclose(rec["r_ctrl"][0], [-10 * 0.01, -10 * 0.01, 0.0], atol=1e-12)
    np.testing.assert_array_equal(rec["r_goal"][0], [-1, -1, 0])
    np.testing.assert_array_equal(rec["done"][0], [1, 1, 1])
    np.testing.assert_allclose(rec["states"][1], pool[0])


def test_no_termination_when_disabled():
    p = synth.params(n_env=1, horizon=1, cam=None, terminate=0)
    o = oracle.Oracle(p, _scene(p, spheres=[(0.1, 0, 0, 0.5)]))
    rec = o.rollout(_hover_pm([0, 0, 0])[None], np.array([[[0, 0, 0.981]]]))
    assert rec["done"][0, 0] == 0 and rec["r_goal"][0, 0] == -1


def test_depth_is_observation_of_next_state():
    # output t renders s_{t+1}: the agent moves 1 cm toward a wall in one step
    p = synth.params(model="rigid", n_env=1, horizon=1, cam=(2, 2, 90.0, 10.0))
    o = oracle.Oracle(p, _scene(p, boxes=[(5, -100, -100, 6, 100, 100)]))
    s = np.zeros(13)
    s[3] = 1.0
    s[7] = 1.0  # v_x = 1 m/s
    rec = o.rollout(s[None], np.zeros((1, 1, 4)))
    np.testing.assert_allclose(rec["depth"][0, 0], 5.0 - p["dt"] * 1.0, atol=1e-12)
