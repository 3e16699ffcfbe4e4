"""Pins of the oracle's dynamics (Sec. III-A, Eq. 1 and Eq. 3) to closed forms.

Each case fixes the explicit-Euler step of the paper's continuous equations by
a result that follows from the mathematics alone (fixed points, exact Euler
recurrences, conservation laws, known rotations), so that a dropped term, a
wrong sign or a transposed index in the oracle fails here.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def pm_params(**kw):
    return synth.params(model="pm", **kw)


def rb_params(**kw):
    return synth.params(model="rigid", **kw)


def pm_state(p=(0, 0, 0), v=(0, 0, 0), a=(0, 0, 0), e=(0, 0, 0)):
    return np.array(list(p) + list(v) + list(a) + list(e), dtype=float)


def rb_state(p=(0, 0, 0), q=(1, 0, 0, 0), v=(0, 0, 0), w=(0, 0, 0)):
    return np.array(list(p) + list(q) + list(v) + list(w), dtype=float)


# ---------------------------------------------------------------- point mass
def test_pm_hover_is_fixed_point():
    # Eq. 3: a = u = -g (thrust acceleration cancels gravity), v = 0
    p = pm_params()
    g = p["gravity"]
    s = pm_state(p=(1, 2, 3), a=(0, 0, g))
    act = np.array([0.0, 0.0, g / p["act_scale"]])
    for _ in range(50):
        s = oracle.pm_step(p, s, act)
    np.testing.assert_allclose(s[:3], [1, 2, 3], atol=1e-12)
    np.testing.assert_allclose(s[3:6], 0, atol=1e-12)
    np.testing.assert_allclose(s[6:9], [0, 0, g], atol=1e-12)


def test_pm_freefall_golden():
    gold = json.load(open(os.path.join(GOLD, "freefall_pointmass.json")))
    p = pm_params(dt=gold["dt"], gravity=gold["gravity"], ema_alpha=gold["ema_alpha"])
    s = pm_state()
    for n in range(len(gold["z"])):
        assert s[2] == pytest.approx(gold["z"][n], abs=1e-12)
        assert s[5] == pytest.approx(gold["vz"][n], abs=1e-12)
        assert s[11] == pytest.approx(gold["ez"][n], abs=1e-12)
        np.testing.assert_allclose(s[6:9], 0, atol=0)
        s = oracle.pm_step(p, s, np.zeros(3))


def test_pm_freefall_closed_form_with_initial_velocity():
    p = pm_params(dt=0.02)
    dt, g = p["dt"], np.array([0, 0, -p["gravity"]])
    p0, v0 = np.array([0.5, -1.0, 2.0]), np.array([1.0, -2.0, 3.0])
    s = pm_state(p=p0, v=v0)
    for n in range(1, 40):
        s = oracle.pm_step(p, s, np.zeros(3))
        np.testing.assert_allclose(s[3:6], v0 + n * dt * g, atol=1e-12)
        np.testing.assert_allclose(s[0:3], p0 + n * dt * v0 + 0.5 * n * (n - 1) * dt * dt * g, atol=1e-11)


def test_pm_command_lag_closed_form():
    # a_{n} = u (1 - (1 - lambda dt)^n) for constant u from a_0 = 0
    p = pm_params(lam=10.0, dt=0.01)
    act = np.array([0.3, -0.7, 1.0])
    u = p["act_scale"] * act
    s = pm_state()
    for n in range(1, 60):
        s = oracle.pm_step(p, s, act)
        np.testing.assert_allclose(s[6:9], u * (1 - (1 - p["lam"] * p["dt"]) ** n), atol=1e-12)


def test_pm_lag_converges_to_continuous_solution():
    # Euler error of a(t) = u (1 - exp(-lambda t)) at t = 0.5 s shrinks linearly in dt
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        p = pm_params(lam=10.0, dt=dt)
        act = np.array([0.5, 0, 0])
        s = pm_state()
        for _ in range(int(round(0.5 / dt))):
            s = oracle.pm_step(p, s, act)
        errs.append(abs(s[6] - 5.0 * (1 - math.exp(-10.0 * 0.5))))
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.05)


def test_pm_action_clip():
    p = pm_params()
    s1 = oracle.pm_step(p, pm_state(), np.array([3.0, -5.0, 0.5]))
    s2 = oracle.pm_step(p, pm_state(), np.array([1.0, -1.0, 0.5]))
    np.testing.assert_array_equal(s1, s2)


def test_pm_drag_decay():
    # hover thrust, drag d: v_n = (1 - dt d)^n v_0
    p = pm_params(drag=0.4)
    g = p["gravity"]
    v0 = np.array([2.0, -1.0, 0.5])
    s = pm_state(v=v0, a=(0, 0, g))
    act = np.array([0, 0, g / p["act_scale"]])
    for n in range(1, 30):
        s = oracle.pm_step(p, s, act)
        np.testing.assert_allclose(s[3:6], (1 - p["dt"] * 0.4) ** n * v0, atol=1e-12)


def test_pm_per_env_drag_and_lag_override():
    p = pm_params()
    s = pm_state(v=(1, 0, 0))
    a = oracle.pm_step(p, s, np.array([1.0, 0, 0]), drag=0.5, lam=4.0)
    assert a[3] == pytest.approx(1 + p["dt"] * (0 - 0.5 * 1))
    assert a[6] == pytest.approx(p["dt"] * 4.0 * p["act_scale"])


# ---------------------------------------------------------------- rigid body
def test_rb_hover_is_fixed_point():
    # Eq. 1: level attitude, thrust m g (action 0), zero rates
    p = rb_params()
    s = rb_state(p=(1, -2, 3))
    s0 = s.copy()
    for _ in range(100):
        s = oracle.rb_step(p, s, np.zeros(4))
    np.testing.assert_allclose(s, s0, atol=1e-14)


def test_rb_freefall_matches_point_mass_closed_form():
    p = rb_params(dt=0.005)
    dt, g = p["dt"], np.array([0, 0, -p["gravity"]])
    v0 = np.array([0.3, 0.2, -0.1])
    s = rb_state(v=v0)
    for n in range(1, 50):
        s = oracle.rb_step(p, s, np.array([-1.0, 0, 0, 0]))  # thrust m g (1 - 1) = 0
        np.testing.assert_allclose(s[7:10], v0 + n * dt * g, atol=1e-12)
        np.testing.assert_allclose(s[0:3], n * dt * v0 + 0.5 * n * (n - 1) * dt * dt * g, atol=1e-12)


def test_rb_tilted_thrust_direction():
    # q = rotation about x by theta: z_B = (0, -sin, cos); thrust m g gives
    # v' = dt g (0, -sin, cos - 1) from rest
    p = rb_params()
    th = 0.3
    s = rb_state(q=(math.cos(th / 2), math.sin(th / 2), 0, 0))
    s1 = oracle.rb_step(p, s, np.zeros(4))
    g, dt = p["gravity"], p["dt"]
    np.testing.assert_allclose(s1[7:10], dt * g * np.array([0, -math.sin(th), math.cos(th) - 1]), atol=1e-14)


def test_rb_quaternion_stays_unit():
    p = rb_params()
    rng = np.random.default_rng(0)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    s = rb_state(q=q, w=rng.standard_normal(3))
    for _ in range(200):
        s = oracle.rb_step(p, s, rng.uniform(-1, 1, 4))
        assert abs(np.linalg.norm(s[3:7]) - 1) < 1e-14


def test_rb_constant_body_rate_closed_form():
    # omega = omega_c is a fixed point of the rate loop; then each Euler step
    # right-multiplies q by (1, dt/2 omega) (renormalised), i.e. a rotation
    # about the body axis omega by 2 atan(dt |omega| / 2).
    p = rb_params()
    rs = np.array(p["rate_scale"])
    act = np.array([0.0, 0.4, -0.3, 0.8])
    w = rs * act[1:]
    q0 = np.array([math.cos(0.2), 0.0, math.sin(0.2), 0.0])
    s = rb_state(q=q0, w=w)
    th = 2 * math.atan(0.5 * p["dt"] * np.linalg.norm(w))
    ax = w / np.linalg.norm(w)

    def qmul(a, b):
        return np.array([a[0] * b[0] - a[1:] @ b[1:],
                         *(a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:]))])

    for n in range(1, 80):
        s = oracle.rb_step(p, s, act)
        ang = n * th
        qn = qmul(q0, np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)]))
        np.testing.assert_allclose(s[3:7], qn, atol=1e-12)
        np.testing.assert_allclose(s[10:13], w, atol=1e-12)


def test_rb_yaw_rate_rotates_heading():
    # body yaw rate: the body x axis turns counter-clockwise about world z
    p = rb_params()
    act = np.array([0.0, 0.0, 0.0, 1.0])
    wz = p["rate_scale"][2]
    s = rb_state(w=(0, 0, wz))
    n = 100
    for _ in range(n):
        s = oracle.rb_step(p, s, act)
    R = oracle.quat_to_rot(s[3:7])
    ang = n * 2 * math.atan(0.5 * p["dt"] * wz)
    np.testing.assert_allclose(R[:, 0], [math.cos(ang), math.sin(ang), 0], atol=1e-12)


def test_rb_gyroscopic_feedforward_cancels():
    # Eq. 1's -omega x J omega and the controller's +omega x J omega cancel:
    # with zero rate gain every body rate is held, although omega x J omega is
    # not zero for J = diag(.01, .01, .02) (a sign slip would make omega drift)
    p = rb_params(k_rate=(0.0, 0.0, 0.0))
    w0 = np.array([0.7, -0.4, 2.5])
    J = np.array(p["inertia"])
    assert np.linalg.norm(np.cross(w0, J * w0)) > 1e-3
    s = rb_state(w=w0)
    for _ in range(100):
        s = oracle.rb_step(p, s, np.zeros(4))
        np.testing.assert_allclose(s[10:13], w0, atol=1e-13)


def test_rb_rate_loop_first_order():
    # omega' = omega + dt K (omega_c - omega) (the gyroscopic feed-forward cancels)
    p = rb_params()
    K, rs, dt = np.array(p["k_rate"]), np.array(p["rate_scale"]), p["dt"]
    act = np.array([0.0, 0.5, -0.25, 1.0])
    wc = rs * act[1:]
    s = rb_state()
    for n in range(1, 40):
        s = oracle.rb_step(p, s, act)
        np.testing.assert_allclose(s[10:13], wc * (1 - (1 - dt * K) ** n), atol=1e-12)


def test_rb_isotropic_drag_decay():
    # D = d I: R D R^T v = d v for any attitude
    p = rb_params(drag_body=(0.5, 0.5, 0.5))
    v0 = np.array([1.0, 2.0, -0.5])
    th = 0.4
    s = rb_state(q=(math.cos(th / 2), 0, 0, math.sin(th / 2)), v=v0)  # yawed, level
    for n in range(1, 30):
        s = oracle.rb_step(p, s, np.zeros(4))
        np.testing.assert_allclose(s[7:10], (1 - p["dt"] * 0.5) ** n * v0, atol=1e-12)


def test_rb_anisotropic_drag_acts_in_body_frame():
    # D = diag(d, 0, 0) with the body yawed by 90 deg: body x = world y, so
    # only the world-y velocity decays
    p = rb_params(drag_body=(0.8, 0.0, 0.0))
    s = rb_state(q=(math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)), v=(1.0, 1.0, 0.0))
    s1 = oracle.rb_step(p, s, np.zeros(4))
    np.testing.assert_allclose(s1[7:10], [1.0, 1.0 - p["dt"] * 0.8, 0.0], atol=1e-14)


def test_quat_to_rot_rotations():
    th = 0.7
    R = oracle.quat_to_rot([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    np.testing.assert_allclose(R @ [1, 0, 0], [math.cos(th), math.sin(th), 0], atol=1e-15)
    R = oracle.quat_to_rot([math.cos(th / 2), math.sin(th / 2), 0, 0])
    np.testing.assert_allclose(R @ [0, 1, 0], [0, math.cos(th), math.sin(th)], atol=1e-15)
    rng = np.random.default_rng(1)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    R = oracle.quat_to_rot(q)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert np.linalg.det(R) == pytest.approx(1.0)
