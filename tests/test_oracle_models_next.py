"""Pins of the oracle's discrete point mass (Eq. 4) and simplified
quadrotor (Eq. 2): closed forms the schemes reach exactly, invariants, and
central differences of the adjoint on tiny instances with sensors and
obstacles."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth

G = 9.81


def _pmd(**kw):
    return synth.params(model="pm_disc", **kw)


def _simple(**kw):
    return synth.params(model="simple", **kw)


# ------------------------------------------------------------- Eq. 4
def test_pmd_free_fall_is_exact():
    """Zero thrust: p_n = p0 + v0 n dt + g (n dt)^2 / 2 exactly (the scheme
    integrates a constant acceleration without error)."""
    p = _pmd(dt=0.01)
    s = np.zeros(12)
    s[0:3] = [1.0, -2.0, 3.0]
    s[3:6] = [0.5, 0.25, 2.0]
    for n in range(1, 101):
        s = oracle.pmd_step(p, s, np.zeros(3))
        t = n * 0.01
        np.testing.assert_allclose(s[0:3], [1.0 + 0.5 * t, -2.0 + 0.25 * t, 3.0 + 2.0 * t - 0.5 * G * t * t],
                                   rtol=0, atol=1e-12)
        np.testing.assert_allclose(s[3:6], [0.5, 0.25, 2.0 - G * t], rtol=0, atol=1e-12)


def test_pmd_hover_is_a_fixed_point():
    p = _pmd()
    s = np.zeros(12)
    s[0:3] = [0.3, 0.2, 1.0]
    s[6:9] = [0.0, 0.0, G]
    cmd = np.array([0.0, 0.0, G / p["act_scale"]])
    for _ in range(50):
        s = oracle.pmd_step(p, s, cmd)
    np.testing.assert_allclose(s[0:3], [0.3, 0.2, 1.0], atol=1e-12)
    np.testing.assert_allclose(s[3:6], 0.0, atol=1e-12)


def test_pmd_velocity_takes_the_half_step_average():
    """A command change from u0 to u1 moves v by (u0 + u1)/2 + g over one step,
    p by u0 / 2 dt^2 (the new command enters p one step later)."""
    p = _pmd(dt=0.02)
    s = np.zeros(12)
    s[6:9] = [1.0, -2.0, 5.0]
    a = np.array([0.3, 0.1, -0.4])
    o = oracle.pmd_step(p, s, a)
    u1 = p["act_scale"] * a
    g = np.array([0.0, 0.0, -G])
    np.testing.assert_allclose(o[3:6], 0.5 * (s[6:9] + u1) * 0.02 + g * 0.02, atol=1e-14)
    np.testing.assert_allclose(o[0:3], 0.5 * (s[6:9] + g) * 0.02 ** 2, atol=1e-14)
    np.testing.assert_allclose(o[6:9], u1, atol=1e-15)
    np.testing.assert_allclose(o[9:12], p["ema_alpha"] * o[3:6], atol=1e-15)


def test_pmd_constant_command_is_exact():
    p = _pmd(dt=0.01)
    a = np.array([0.2, -0.5, 0.9])
    u = p["act_scale"] * a
    w = u + np.array([0.0, 0.0, -G])
    s = np.zeros(12)
    s[6:9] = u
    for n in range(1, 60):
        s = oracle.pmd_step(p, s, a)
        t = n * 0.01
        np.testing.assert_allclose(s[0:3], 0.5 * w * t * t, atol=1e-12)


# ------------------------------------------------------------- Eq. 2
def _rest_simple():
    s = np.zeros(15)
    s[6] = s[10] = s[14] = 1.0
    return s


def test_simple_hover_is_a_fixed_point():
    p = _simple()
    s = _rest_simple()
    s[0:3] = [1.0, 2.0, 3.0]
    for _ in range(40):
        s = oracle.simple_step(p, s, np.zeros(4))
    np.testing.assert_allclose(s, np.r_[1.0, 2.0, 3.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], atol=1e-13)


def test_simple_free_fall():
    p = _simple(dt=0.01)
    s = _rest_simple()
    for n in range(1, 31):
        s = oracle.simple_step(p, s, np.array([-1.0, 0, 0, 0]))
    t = 30 * 0.01
    # explicit Euler: v_n = g n dt, p_n = g dt^2 n (n - 1) / 2
    np.testing.assert_allclose(s[5], -G * t, atol=1e-12)
    np.testing.assert_allclose(s[2], -G * 0.01 ** 2 * 30 * 29 / 2, atol=1e-12)


def test_simple_yaw_rate_closed_form():
    """Constant yaw rate w: Euler + Gram-Schmidt rotate by exactly
    atan(w dt) per step about z."""
    p = _simple(dt=0.01)
    w = 1.2  # rad/s, within rate_scale z = 1.5
    a = np.array([0.0, 0.0, 0.0, w / p["rate_scale"][2]])
    s = _rest_simple()
    for n in range(1, 81):
        s = oracle.simple_step(p, s, a)
        th = n * math.atan(w * 0.01)
        Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
        np.testing.assert_allclose(s[6:15].reshape(3, 3), Rz, atol=1e-12)


def test_simple_rotation_stays_orthonormal_and_thrust_follows_z_body():
    p = _simple(dt=0.005)
    rng = np.random.default_rng(3)
    s = _rest_simple()
    for _ in range(200):
        a = rng.uniform(-1, 1, 4)
        o = oracle.simple_step(p, s, a)
        R = s[6:15].reshape(3, 3)
        c = G * (1 + a[0])
        np.testing.assert_allclose(o[3:6], s[3:6] + 0.005 * (c * R[:, 2] + [0, 0, -G]), atol=1e-12)
        Rn = o[6:15].reshape(3, 3)
        np.testing.assert_allclose(Rn @ Rn.T, np.eye(3), atol=1e-13)
        assert np.linalg.det(Rn) > 0.999999
        s = o


# ------------------------------------------------------------- adjoints
def _fd(p, s0, seed, min_hits=5):
    inp = synth.make_inputs(p, seed=seed)
    o = oracle.Oracle(p, inp)
    act = inp["actions"]
    rec = o.rollout(s0, act)
    assert ((rec["amb_cam"] & 3) == 0).all() and (rec["amb_step"] == 0).all()
    assert (rec["hit_cam"] >= 0).sum() >= min_hits
    cot = synth.cotangents(p, seed=seed + 1)
    gsT = np.random.default_rng(seed + 2).standard_normal((o.NM, o.D))
    ga, gs0 = o.backward(rec, cot["g_r"], cot.get("g_depth"), None, gsT)
    L = lambda s, a: o.loss(s, a, cot["g_r"], cot.get("g_depth"), None, gsT)
    skipped = 0
    for x, g, f in ((act, ga, lambda a: L(s0, a)), (s0, gs0, lambda s: L(s, act))):
        scale = np.abs(g).max()
        for idx in np.ndindex(x.shape):
            d = []
            for h in (1e-6, 2e-6):
                xp, xm = x.copy(), x.copy()
                xp[idx] += h
                xm[idx] -= h
                d.append((f(xp) - f(xm)) / (2 * h))
            if abs(d[0] - d[1]) > 1e-6 * max(abs(d[0]), scale):
                skipped += 1
                continue
            assert abs(g[idx] - d[0]) <= 1e-6 * max(abs(d[0]), scale), (idx, g[idx], d[0])
    assert skipped <= 2


def test_pmd_adjoint_matches_central_differences():
    p = _pmd(n_env=2, horizon=6, cam=(4, 3, 90.0, 10.0), map_counts=[(3, 2)], obst_lo=(2, -3, -3),
             obst_hi=(7, 3, 3), init_lo=(-1, -1, -1), init_hi=(1, 1, 1), w_obs=5.0, d_safe=4.0)
    inp = synth.make_inputs(p, seed=5)
    s0 = inp["s0"].copy()
    s0[:, 3:6] = [1.0, 0.2, 0.1]
    s0[:, 6:9] = [0.5, 0.3, 9.81]
    s0[:, 9:12] = [1.0, 0.1, 0.0]
    _fd(p, s0, seed=5, min_hits=10)


def test_simple_adjoint_matches_central_differences():
    p = _simple(n_env=2, horizon=6, dt=0.02, cam=(4, 3, 90.0, 10.0), map_counts=[(3, 2)],
                obst_lo=(2, -3, -3), obst_hi=(7, 3, 3), init_lo=(-1, -1, -1), init_hi=(1, 1, 1),
                w_obs=5.0, d_safe=4.0, pos_sq=0)
    inp = synth.make_inputs(p, seed=6)
    s0 = inp["s0"].copy()
    s0[:, 3:6] = [1.0, 0.3, 0.2]
    _fd(p, s0, seed=6, min_hits=10)
