"""Pins of the oracle's hand-written adjoint (Eq. 5, reverse mode through
dynamics, attitude, ray casting, rewards and resets) by central finite
differences of the oracle's own forward map, in FP64, on tiny instances.

Instances are screened: the rollout must report no ambiguous ray or step, and
each finite difference must agree at two step sizes (no branch crossed).
"""
import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth

EPS = 1e-6


def _fd_check(p, s0, seed=5, rtol=1e-6, min_depth_hits=1):
    inp = synth.make_inputs(p, seed=seed)
    o = oracle.Oracle(p, inp)
    act = inp["actions"]
    rec = o.rollout(s0, act)
    # no decision within reach of the finite-difference step (bits 0, 1);
    # FP32 conditioning flags (bits 2, 3) do not concern an FP64 check
    assert ((rec["amb_cam"] & 3) == 0).all() and ((rec["amb_lid"] & 3) == 0).all()
    assert (rec["amb_step"] == 0).all()
    if p["cam"] is not None:
        assert (rec["hit_cam"] >= 0).sum() >= min_depth_hits
    cot = synth.cotangents(p, seed=seed + 1)
    gsT = np.random.default_rng(seed + 2).standard_normal((o.NM, o.D))
    ga, gs0 = o.backward(rec, cot["g_r"], cot.get("g_depth"), cot.get("g_lidar"), gsT)

    def L(s, a):
        return o.loss(s, a, cot["g_r"], cot.get("g_depth"), cot.get("g_lidar"), gsT)

    def fd(x, f, idx, h):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        return (f(xp) - f(xm)) / (2 * h)

    skipped = 0
    for x, g, f in ((act, ga, lambda a: L(s0, a)), (s0, gs0, lambda s: L(s, act))):
        scale = np.abs(g).max()
        for idx in np.ndindex(x.shape):
            d1, d2 = fd(x, f, idx, EPS), fd(x, f, idx, 2 * EPS)
            if abs(d1 - d2) > 1e-6 * max(abs(d1), scale):
                skipped += 1
                continue
            assert abs(g[idx] - d1) <= rtol * max(abs(d1), scale), (idx, g[idx], d1)
    assert skipped <= 2
    return rec


def _pm_s0(inp, NM):
    s0 = inp["s0"].copy()
    s0[:, 3:6] = [1.0, 0.2, 0.1]
    s0[:, 6:9] = [0.5, 0.3, 9.81]
    s0[:, 9:12] = [1.0, 0.1, 0.0]
    return s0


def test_adjoint_pointmass_depth_spheres_boxes():
    p = synth.params(n_env=2, horizon=6, cam=(4, 3, 90.0, 10.0), map_counts=[(3, 2)],
                     obst_lo=(2, -3, -3), obst_hi=(7, 3, 3), init_lo=(-1, -1, -1),
                     init_hi=(1, 1, 1), drag=0.2, w_obs=5.0, d_safe=4.0)
    inp = synth.make_inputs(p, seed=5)
    _fd_check(p, _pm_s0(inp, 2), min_depth_hits=10)


def test_adjoint_pointmass_swarm_pairs():
    p = synth.params(n_env=2, n_agent=3, horizon=5, cam=(4, 3, 90.0, 10.0), map_counts=[(2, 1)],
                     obst_lo=(2, -3, -3), obst_hi=(7, 3, 3), init_lo=(-1, -1, -1),
                     init_hi=(1, 1, 1), w_agent=10.0, d_agent=3.0, w_obs=5.0, d_safe=4.0)
    inp = synth.make_inputs(p, seed=11)
    _fd_check(p, _pm_s0(inp, 6), seed=11, min_depth_hits=5)


def test_adjoint_pointmass_domain_randomised():
    p = synth.params(n_env=2, horizon=5, cam=(4, 3, 90.0, 10.0), map_counts=[(2, 1)],
                     obst_lo=(2, -3, -3), obst_hi=(7, 3, 3), init_lo=(-1, -1, -1),
                     init_hi=(1, 1, 1), drag_range=(0.1, 0.5), lam_range=(5.0, 15.0))
    inp = synth.make_inputs(p, seed=5)
    _fd_check(p, _pm_s0(inp, 2))


def test_adjoint_rigid_depth_lidar():
    p = synth.params(model="rigid", n_env=2, horizon=6, dt=0.005, cam=(4, 3, 90.0, 10.0),
                     lidar=(2, 8, -15.0, 15.0, 10.0), map_counts=[(3, 2)],
                     obst_lo=(-6, -6, -2), obst_hi=(6, 6, 2), init_lo=(-1, -1, -1),
                     init_hi=(1, 1, 1), drag_body=(0.3, 0.3, 0.1), pos_sq=0, w_obs=5.0,
                     d_safe=4.0)
    inp = synth.make_inputs(p, seed=7)
    s0 = inp["s0"].copy()
    q = np.array([0.95, 0.1, -0.2, 0.2])
    s0[:, 3:7] = q / np.linalg.norm(q)
    s0[:, 7:10] = [0.5, -0.3, 0.2]
    s0[:, 10:13] = [0.3, -0.5, 0.8]
    _fd_check(p, s0, seed=7, min_depth_hits=5)


def test_adjoint_with_resets():
    # collisions terminate and reset mid-rollout; no cotangent crosses a reset
    p = synth.params(n_env=2, horizon=8, cam=(4, 3, 90.0, 10.0), map_counts=[(3, 2)],
                     obst_lo=(0.3, -1.0, -1.0), obst_hi=(1.2, 1.0, 1.0), sph_radius=(0.3, 0.5),
                     box_half=(0.2, 0.4), init_lo=(-1, -1, -1), init_hi=(1, 1, 1),
                     terminate=1, pool_size=3)
    for seed in range(20, 60):
        inp = synth.make_inputs(p, seed=seed)
        o = oracle.Oracle(p, inp)
        s0 = _pm_s0(inp, 2)
        rec = o.rollout(s0, inp["actions"])
        if rec["done"].sum() == 0 or rec["done"][-1].any():
            continue
        if (rec["amb_cam"] & 3).any() or (rec["amb_step"] != 0).any():
            continue
        _fd_check(p, s0, seed=seed)
        return
    pytest.fail("no screened instance with a reset")


def test_adjoint_cylinders_and_gates():
    # depth and LiDAR hits on cylinder sides / caps and gate bars, and the
    # obstacle reward through their signed distances
    p = synth.params(model="rigid", n_env=2, horizon=5, dt=0.005, cam=(8, 6, 90.0, 12.0),
                     lidar=(3, 24, -20.0, 20.0, 12.0), map_counts=[(1, 1, 4, 4)],
                     obst_lo=(-6, -6, -2), obst_hi=(6, 6, 2), init_lo=(-1, -1, -1),
                     init_hi=(1, 1, 1), race_radius=4.0, gate_half=(0.8, 1.2), gate_border=0.4,
                     pos_sq=0, w_obs=5.0, d_safe=6.0)
    for seed in range(30, 90):
        inp = synth.make_inputs(p, seed=seed)
        o = oracle.Oracle(p, inp)
        s0 = inp["s0"].copy()
        q = np.array([0.97, 0.05, -0.1, 0.2])
        s0[:, 3:7] = q / np.linalg.norm(q)
        s0[:, 7:10] = [0.5, -0.3, 0.2]
        rec = o.rollout(s0, inp["actions"])
        if (rec["amb_cam"] & 3).any() or (rec["amb_lid"] & 3).any() or (rec["amb_step"] != 0).any():
            continue
        hits = np.concatenate([rec["hit_cam"].ravel(), rec["hit_lid"].ravel()])
        if (hits >= 2).sum() < 10 or ((hits >= 2) & (hits < 6)).sum() < 3 or (hits >= 6).sum() < 3:
            continue
        if not ((rec["sdf_id"] >= 2).any()):
            continue
        _fd_check(p, s0, seed=seed, min_depth_hits=5)
        return
    pytest.fail("no screened instance hitting cylinders and gates")
