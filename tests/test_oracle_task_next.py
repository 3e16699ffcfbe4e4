"""Pins of the oracle's racing task (Sec. III-C: gates passed in a predefined
order, the progress reward of the racing task) and of the IMU readout
(Sec. III-B: specific force and angular rate in the body frame, optional
white noise and bias random walk), on hand-computed cases, plus finite
differences of the adjoint through both."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth


def _scene(p, gates=(), spheres=(), pool=None):
    NM = p["n_env"] * p["n_agent"]
    D = synth.STATE_DIM[p["model"]]
    gt = np.array(gates, float).reshape(-1, 7)
    sp = np.array(spheres, float).reshape(-1, 4)
    z = lambda k: np.zeros((0, k))
    off = lambda n: np.array([0, n], np.int32)
    return dict(spheres=sp, sph_off=off(len(sp)), boxes=z(6), box_off=off(0), cylinders=z(5),
                cyl_off=off(0), gates=gt, gate_off=off(len(gt)),
                env_map=np.zeros(p["n_env"], np.int32), targets=np.zeros((NM, 3)),
                pool=np.zeros((p["pool_size"], NM, D)) if pool is None else np.array(pool, float))


def _simple(pos, vel):
    s = np.zeros(15)
    s[0:3], s[3:6] = pos, vel
    s[6] = s[10] = s[14] = 1.0
    return s


# ------------------------------------------------------------------ racing
def test_racing_pass_reward_and_progress_by_hand():
    # simplified quadrotor hovering (a0 = 0), flying at 10 m/s along +x through
    # a gate at the origin facing +x: positions -0.45, -0.35, ..., crossing
    # x = 0 during step 5; before it every step gains 0.1 m of progress
    p = synth.params(model="simple", n_env=1, horizon=8, cam=None, task="racing", w_pos=2.0,
                     w_act=0.0, gravity=9.81)
    sc = _scene(p, gates=[(0, 0, 0, 0, 1, 0.2, 0.1), (5, 5, 0, 0, 1, 0.2, 0.1)])
    o = oracle.Oracle(p, sc)
    rec = o.rollout(_simple([-0.55, 0, 0], [10, 0, 0])[None], np.zeros((8, 1, 4)))
    np.testing.assert_array_equal(rec["r_goal"][:, 0], [0, 0, 0, 0, 0, 1, 0, 0])
    np.testing.assert_array_equal(rec["gate_tape"][:, 0], [0, 0, 0, 0, 0, 0, 1, 1])
    assert rec["gate_k"][0] == 1
    np.testing.assert_allclose(rec["r_ctrl"][:5, 0], 2.0 * 0.1, atol=1e-12)
    # step 5 moves from x = -0.05 to 0.05: |p_t - g| - |p_{t+1} - g| = 0
    assert rec["r_ctrl"][5, 0] == pytest.approx(0.0, abs=1e-12)
    # step 6 targets gate 1 at (5, 5, 0)
    d0, d1 = math.hypot(5 - 0.05, 5), math.hypot(5 - 0.15, 5)
    assert rec["r_ctrl"][6, 0] == pytest.approx(2.0 * (d0 - d1), abs=1e-12)
    assert (rec["amb_step"] == 0).all()


def test_racing_wrong_direction_outside_and_wraparound():
    p = synth.params(model="simple", n_env=1, horizon=8, cam=None, task="racing", w_act=0.0)
    act = np.zeros((8, 1, 4))
    # backwards through the opening: no pass
    o = oracle.Oracle(p, _scene(p, gates=[(0, 0, 0, math.pi, 1, 0.2, 0.1)]))
    rec = o.rollout(_simple([-0.55, 0, 0], [10, 0, 0])[None], act)
    assert (rec["r_goal"] == 0).all() and rec["gate_k"][0] == 0
    # beside the gate (outside the frame): no pass
    o = oracle.Oracle(p, _scene(p, gates=[(0, 0, 0, 0, 1, 0.2, 0.1)]))
    rec = o.rollout(_simple([-0.55, 3, 0], [10, 0, 0])[None], act)
    assert (rec["r_goal"] == 0).all()
    # two gates in a row, then back to gate 0 (cyclic order)
    o = oracle.Oracle(p, _scene(p, gates=[(0, 0, 0, 0, 1, 0.2, 0.1), (0.3, 0, 0, 0, 1, 0.2, 0.1)]))
    rec = o.rollout(_simple([-0.55, 0, 0], [10, 0, 0])[None], act)
    np.testing.assert_array_equal(rec["r_goal"][:, 0], [0, 0, 0, 0, 0, 1, 0, 0])
    rec = o.rollout(_simple([-0.55, 0, 0], [10, 0, 0])[None], act, gate_k=[1])
    assert (rec["r_goal"][:, 0] == 0).all()  # gate 0 is passed while gate 1 is targeted
    rec = o.rollout(_simple([-0.25, 0, 0], [10, 0, 0])[None], act, gate_k=[1])
    np.testing.assert_array_equal(rec["r_goal"][:, 0], [0, 0, 0, 0, 0, 1, 0, 0])
    assert rec["gate_k"][0] == 0


def test_racing_collision_with_frame_resets_to_first_gate():
    p = synth.params(model="simple", n_env=1, horizon=6, cam=None, task="racing", terminate=1,
                     pool_size=1, r_quad=0.2)
    pool = _simple([-3, 0, 0], [0, 0, 0])[None, None]
    o = oracle.Oracle(p, _scene(p, gates=[(0, 0, 0, 0, 1, 0.2, 0.1), (5, 0, 0, 0, 1, 0.2, 0.1)],
                                pool=pool))
    # targeting gate 1, flying along the top bar's height into gate 0's frame:
    # the collision resets the environment and the course restarts at gate 0
    rec = o.rollout(_simple([-0.55, 0, 1.1], [10, 0, 0])[None], np.zeros((6, 1, 4)), gate_k=[1])
    t = int(np.argmax(rec["done"][:, 0]))
    assert rec["done"][t, 0] == 1 and rec["r_goal"][t, 0] == -1
    assert rec["gate_tape"][t, 0] == 1 and rec["gate_tape"][t + 1, 0] == 0


# --------------------------------------------------------------------- IMU
def _imu_one(p, s, a):
    o = oracle.Oracle(p, _scene(p))
    rec = o.rollout(np.array(s, float)[None], np.array(a, float)[None, None])
    return rec["imu"][0, 0], rec


def test_imu_rigid_hover_free_fall_and_drag_frame():
    p = synth.params(model="rigid", n_env=1, horizon=1, cam=None, drag_body=(0.3, 0.5, 0.7))
    s = np.zeros(13)
    s[3] = 1.0
    imu, _ = _imu_one(p, s, [0, 0, 0, 0])
    np.testing.assert_allclose(imu, [0, 0, 9.81, 0, 0, 0], atol=1e-12)      # hover
    imu, _ = _imu_one(p, s, [-1, 0, 0, 0])
    # free fall: no thrust; after one step v_z = -g dt, so only drag remains
    np.testing.assert_allclose(imu, [0, 0, 0.7 * 9.81 * 0.01, 0, 0, 0], atol=1e-12)
    # yawed 90 deg, moving along world +x: body velocity (0, -1, 0), so the
    # drag part of the specific force is (0, +D_y, 0) (a wrong transpose gives -D_y)
    c = math.cos(math.pi / 4)
    s = np.zeros(13)
    s[3:7] = [c, 0, 0, c]
    s[7:10] = [1, 0, 0]
    s[10:13] = [0.2, -0.1, 0.3]
    imu, rec = _imu_one(p, s, [0, 0, 0, 0])
    s1 = rec["spre"][0, 0]
    R1 = oracle.quat_to_rot(s1[3:7])
    np.testing.assert_allclose(imu[:3], [0, 0, 9.81] - np.array([0.3, 0.5, 0.7]) * (R1.T @ s1[7:10]),
                               atol=1e-12)
    assert imu[1] == pytest.approx(0.5, abs=0.05)
    np.testing.assert_allclose(imu[3:], s1[10:13], atol=1e-15)


def test_imu_point_mass_specific_force_and_rate():
    # hover thrust a = (0, 0, g), heading EMA along +y: x_B = +y, y_B = -x
    p = synth.params(n_env=1, horizon=1, cam=None, drag=0.4)
    s = np.zeros(12)
    s[3:6] = [1, 0, 0]
    s[6:9] = [0, 0, 9.81]
    s[9:12] = [0, 1, 0]
    imu, rec = _imu_one(p, s, [0, 0, 0.981])
    s1 = rec["spre"][0, 0]
    # f = R^T (a - d v) with R from the new state's attitude
    _, R1, _ = oracle.pose(p, s1)
    np.testing.assert_allclose(imu[:3], R1.T @ (s1[6:9] - 0.4 * s1[3:6]), atol=1e-12)
    assert imu[1] == pytest.approx(0.4, abs=0.01) and imu[0] == pytest.approx(0.0, abs=0.05)
    # the angular rate is the attitude change over the step, in the body frame:
    # compare with the rotation vector of R0^T R1 (agrees to O(theta^3))
    rng = np.random.default_rng(0)
    for _ in range(10):
        s = np.zeros(12)
        s[3:6] = rng.uniform(-3, 3, 3)
        s[6:9] = [0, 0, 9.81] + rng.uniform(-3, 3, 3)
        s[9:12] = rng.uniform(-2, 2, 3)
        imu, rec = _imu_one(p, s, rng.uniform(-1, 1, 3))
        _, R0, _ = oracle.pose(p, s)
        _, R1, _ = oracle.pose(p, rec["spre"][0, 0])
        A = R0.T @ R1
        th = math.acos(min(1.0, (np.trace(A) - 1) / 2))
        axis = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
        rv = axis * (th / (2 * math.sin(th))) if th > 1e-12 else axis / 2
        np.testing.assert_allclose(imu[3:] * p["dt"], rv, rtol=th ** 2, atol=1e-14)
        assert th > 1e-4


def test_imu_discrete_and_simplified():
    p = synth.params(model="pm_disc", n_env=1, horizon=1, cam=None)
    s = np.zeros(12)
    s[6:9] = [0, 0, 9.81]
    s[9:12] = [1, 0, 0]
    imu, _ = _imu_one(p, s, [0.1, -0.2, 0.981])
    np.testing.assert_allclose(np.linalg.norm(imu[:3]), 10 * np.linalg.norm([0.1, -0.2, 0.981]),
                               rtol=1e-12)  # |R^T u| = |u|, the command in force
    p = synth.params(model="simple", n_env=1, horizon=1, cam=None)
    imu, _ = _imu_one(p, _simple([0, 0, 0], [1, 2, 3]), [0.5, 0.2, -0.4, 1.5])
    np.testing.assert_allclose(imu, [0, 0, 9.81 * 1.5, 0.6, -1.2, 1.5], atol=1e-12)


def test_imu_noise_and_bias_walk():
    p = synth.params(model="rigid", n_env=2, horizon=5, cam=None, imu_noise=(0.1, 0.01),
                     imu_walk=(0.2, 0.02))
    inp = synth.make_inputs(p, seed=3)
    o = oracle.Oracle(p, inp)
    clean = o.rollout(inp["s0"], inp["actions"])["imu"]
    z = np.random.default_rng(9).standard_normal((5, 2, 12))
    b0 = np.random.default_rng(10).standard_normal((2, 6))
    rec = o.rollout(inp["s0"], inp["actions"], imu_noise=z, imu_bias=b0)
    sig = np.array([0.1] * 3 + [0.01] * 3)
    walk = np.array([0.2] * 3 + [0.02] * 3) * math.sqrt(p["dt"])
    b = b0.copy()
    for t in range(5):
        np.testing.assert_allclose(rec["imu"][t], clean[t] + b + sig * z[t, :, :6], atol=1e-12)
        b = b + walk * z[t, :, 6:]
    np.testing.assert_allclose(rec["imu_bias"], b, atol=1e-12)


def test_imu_after_reset_reads_the_new_state_at_rest():
    p = synth.params(n_env=1, horizon=2, cam=None, terminate=1, pool_size=1,
                     bound_lo=(-1, -1, -1), bound_hi=(1, 1, 1))
    pool = np.zeros((1, 1, 12))
    pool[0, 0, 8] = 9.81
    pool[0, 0, 9] = 1.0
    o = oracle.Oracle(p, _scene(p, pool=pool))
    s = pool[0, 0].copy()
    s[0] = 0.999
    s[3] = 5.0
    rec = o.rollout(s[None], np.zeros((2, 1, 3)))
    assert rec["done"][0, 0] == 1
    np.testing.assert_allclose(rec["imu"][0, 0], [0, 0, 9.81, 0, 0, 0], atol=1e-12)


# ------------------------------------------------------------ adjoint (FD)
def _fd(o, s0, act, g_r, g_imu, gate_k=None, eps=1e-6):
    rec = o.rollout(s0, act, gate_k=gate_k)
    assert (rec["amb_step"] == 0).all()
    ga, gs0 = o.backward(rec, g_r, g_imu=g_imu)

    def L(s, a):
        return o.loss(s, a, g_r, g_imu=g_imu, gate_k=gate_k)

    for x, g, f in ((act, ga, lambda a: L(s0, a)), (s0, gs0, lambda s: L(s, act))):
        scale = np.abs(g).max()
        bad = 0
        for idx in np.ndindex(x.shape):
            xp, xm = x.copy(), x.copy()
            xp[idx] += eps
            xm[idx] -= eps
            d1 = (f(xp) - f(xm)) / (2 * eps)
            xp[idx] += eps
            xm[idx] -= eps
            d2 = (f(xp) - f(xm)) / (4 * eps)
            if abs(d1 - d2) > 1e-6 * max(abs(d1), scale):
                bad += 1
                continue
            assert abs(g[idx] - d1) <= 1e-6 * max(abs(d1), scale), (idx, g[idx], d1)
        assert bad <= 2
    return rec


@pytest.mark.parametrize("model", ["pm", "rigid", "pm_disc", "simple"])
def test_imu_adjoint_matches_central_differences(model):
    p = synth.params(model=model, n_env=2, horizon=4, cam=None, dt=0.01, drag=0.3,
                     drag_body=(0.3, 0.4, 0.2))
    inp = synth.make_inputs(p, seed=4)
    o = oracle.Oracle(p, inp)
    s0 = inp["s0"].copy()
    if model in ("pm", "pm_disc"):
        s0[:, 3:6] = [1.0, 0.2, 0.1]
        s0[:, 6:9] = [0.5, 0.3, 9.81]
        s0[:, 9:12] = [1.0, 0.4, 0.0]
    elif model == "rigid":
        q = np.array([0.95, 0.1, -0.2, 0.2])
        s0[:, 3:7] = q / np.linalg.norm(q)
        s0[:, 7:10] = [0.5, -0.3, 0.2]
        s0[:, 10:13] = [0.3, -0.5, 0.8]
    rng = np.random.default_rng(5)
    act = rng.uniform(-0.9, 0.9, inp["actions"].shape)
    g_r = rng.standard_normal((4, 2))
    g_imu = rng.standard_normal((4, 2, 6))
    _fd(o, s0, act, g_r, g_imu)


def test_racing_adjoint_matches_central_differences():
    p = synth.params(model="rigid", n_env=2, horizon=6, cam=(4, 3, 90.0, 10.0), dt=0.01,
                     task="racing", w_obs=2.0, d_safe=3.0, map_counts=[(1, 0, 0, 3)],
                     obst_lo=(-3, -3, -1), obst_hi=(3, 3, 1), race_radius=2.0,
                     init_lo=(-0.5, -0.5, -0.5), init_hi=(0.5, 0.5, 0.5))
    for seed in range(40, 80):
        inp = synth.make_inputs(p, seed=seed)
        o = oracle.Oracle(p, inp)
        s0 = inp["s0"].copy()
        s0[:, 7:10] = [2.0, 0.5, 0.0]
        rec = o.rollout(s0, inp["actions"])
        if (rec["amb_step"] != 0).any() or (rec["amb_cam"] & 3).any():
            continue
        rng = np.random.default_rng(seed)
        _fd(o, s0, inp["actions"], rng.standard_normal((6, 2)), rng.standard_normal((6, 2, 6)))
        return
    pytest.fail("no screened racing instance")
