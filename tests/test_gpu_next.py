"""GPU parity of the racing task (Sec. III-C: gates in order, progress
reward) and of the IMU readout (Sec. III-B) against the FP64 oracle: full
rollouts (rewards, gate passes, gate indices, readings with noise and bias
walk) and their BPTT gradients, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.binding import Simulator
from parity_util import (DRIFT, GRAD_RTOL, compare_grads, compare_rollout, dev, grad_spread, host,
                         masked_cotangents)

pytestmark = pytest.mark.gpu

IMU_TOL = 2e-3  # full rollout, FP32 drift: |imu - imu*| <= IMU_TOL max(|imu*|, 1)


def _racing():
    p = synth.params(model="rigid", n_env=40, horizon=12, dt=0.01, cam=(12, 8, 90.0, 12.0), task="racing",
                     map_counts=[(6, 3, 4, 5)], n_maps=4, obst_lo=(-6, -6, -2), obst_hi=(6, 6, 2),
                     race_radius=4.0, gate_half=(0.8, 1.0), w_obs=2.0, d_safe=1.0, pos_sq=0, terminate=1,
                     ckpt_every=4)
    inp = synth.make_inputs(p, seed=2)
    # every agent starts behind its map's first gate, facing and flying through it
    rng = np.random.default_rng(7)
    s0 = inp["s0"].copy()
    for e in range(p["n_env"]):
        g = inp["gates"][inp["gate_off"][inp["env_map"][e]]]
        n = np.array([math.cos(g[3]), math.sin(g[3]), 0.0])
        l = np.array([-n[1], n[0], 0.0])
        s0[e, 0:3] = g[:3] - 0.2 * n + rng.uniform(-0.4, 0.4) * l + [0, 0, rng.uniform(-0.4, 0.4)]
        s0[e, 3:7] = [math.cos(g[3] / 2), 0.0, 0.0, math.sin(g[3] / 2)]
        s0[e, 7:10] = 4.0 * n
    inp["s0"] = s0.astype(np.float32).astype(np.float64)
    inp["actions"] = inp["actions"] * 0.3
    return p, inp


def test_racing_rollout_and_gradient():
    torch.cuda.init()
    p, inp = _racing()
    orc = oracle.Oracle(p, inp)
    rec = orc.rollout(inp["s0"], inp["actions"])
    assert (rec["r_goal"] == 1).sum() >= p["n_env"] // 2, "the instance should pass gates"
    sim = Simulator(p, inp)
    sim.reset(dev(inp["s0"]))
    act = dev(inp["actions"])
    out = sim.rollout(act)
    sT = sim.get_state()
    k = host(sim.gate_index()).astype(np.int32)
    torch.cuda.synchronize()
    assert sim.status() == 0
    bad = compare_rollout(p, rec, out, sT)
    keep = ~bad
    np.testing.assert_array_equal(k[keep], rec["gate_k"][keep])
    # gradient of the progress reward (plus obstacle and action terms)
    g_r, g_d, _ = masked_cotangents(p, rec)
    g_sT = np.random.default_rng(3).standard_normal((orc.NM, orc.D)).astype(np.float32).astype(np.float64)
    ga_o, gs_o = orc.backward(rec, g_r, g_d, None, g_sT)
    sa, ss = grad_spread(orc, p, inp, rec, g_r, g_d, None, g_sT)
    sim.reset(dev(inp["s0"]))
    sim.rollout(act)
    ga, gs0 = sim.backward(dev(g_r), dev(g_d), None, dev(g_sT))
    torch.cuda.synchronize()
    wa, ia = compare_grads(p, host(ga), ga_o, bad, "g_a", spread=sa)
    ws, is_ = compare_grads(p, host(gs0), gs_o, bad, "g_s0", spread=ss)
    print("racing: worst rel g_a %.2e g_s0 %.2e; ill-conditioned %d, %d of %d" % (wa, ws, ia, is_, p["n_env"]))
    assert ia <= p["n_env"] // 2


def test_racing_gate_index_round_trip_and_step_backward_refused():
    p, inp = _racing()
    sim = Simulator(p, inp)
    k = torch.tensor([(i % 5) for i in range(p["n_env"])], dtype=torch.int32, device="cuda")
    sim.set_gate_index(k)
    assert (sim.gate_index() == k).all()
    sim.reset(dev(inp["s0"]))
    assert (sim.gate_index() == 0).all()
    with pytest.raises(Exception):
        sim.set_gate_index(torch.full((p["n_env"],), 5, dtype=torch.int32, device="cuda"))


def _imu_case(model):
    p = synth.params(model=model, n_env=24, horizon=8, dt=0.01, cam=None, map_counts=[(4, 2, 2, 1)], n_maps=2,
                     obst_lo=(-6, -6, -6), obst_hi=(6, 6, 6), drag=0.3, drag_body=(0.3, 0.4, 0.2),
                     imu_noise=(0.05, 0.01), imu_walk=(0.1, 0.02), w_obs=1.0, ckpt_every=4)
    inp = synth.make_inputs(p, seed=5)
    s0 = inp["s0"].copy()
    rng = np.random.default_rng(8)
    if model in ("pm", "pm_disc"):
        s0[:, 3:6] = rng.uniform(-2, 2, (p["n_env"], 3))
        s0[:, 6:9] = [0.0, 0.0, 9.81] + rng.uniform(-2, 2, (p["n_env"], 3))
        s0[:, 9:12] = rng.uniform(-2, 2, (p["n_env"], 3))
    elif model == "rigid":
        q = rng.standard_normal((p["n_env"], 4)) * 0.2 + [1, 0, 0, 0]
        s0[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
        s0[:, 7:13] = rng.uniform(-1, 1, (p["n_env"], 6))
    inp["s0"] = s0.astype(np.float32).astype(np.float64)
    noise = rng.standard_normal((p["horizon"], p["n_env"], 12)).astype(np.float32).astype(np.float64)
    return p, inp, noise


@pytest.mark.parametrize("model", ["pm", "rigid", "pm_disc", "simple"])
def test_imu_readout_and_gradient(model):
    torch.cuda.init()
    p, inp, noise = _imu_case(model)
    orc = oracle.Oracle(p, inp)
    rec = orc.rollout(inp["s0"], inp["actions"], imu_noise=noise)
    sim = Simulator(p, inp)
    sim.reset(dev(inp["s0"]))
    act = dev(inp["actions"])
    out = sim.rollout(act, imu_noise=dev(noise))
    torch.cuda.synchronize()
    assert sim.status() == 0
    bad = compare_rollout(p, rec, out, sim.get_state())
    keep = np.repeat(~bad, p["n_agent"])
    amb = ((rec["amb_step"] & 4) != 0)
    imu, imu_o = host(out["imu"]), rec["imu"]
    d = np.abs(imu - imu_o)[:, keep]
    ok = (d <= IMU_TOL * np.maximum(np.abs(imu_o[:, keep]), 1.0)) | amb[:, keep, None]
    assert ok.all(), (d.max(), np.argwhere(~ok)[:5])
    # adjoint with a cotangent on the readout (the noise is additive)
    g_r, _, _ = masked_cotangents(p, rec)
    g_imu = np.random.default_rng(4).standard_normal((p["horizon"], orc.NM, 6)) * ((rec["amb_step"] & 6) == 0)[..., None]
    g_imu = g_imu.astype(np.float32).astype(np.float64)
    ga_o, gs_o = orc.backward(rec, g_r, g_imu=g_imu)
    sa, ss = grad_spread(orc, p, inp, rec, g_r, g_imu=g_imu)
    sim.reset(dev(inp["s0"]))
    sim.rollout(act)
    ga, gs0 = sim.backward(dev(g_r), g_imu=dev(g_imu))
    torch.cuda.synchronize()
    wa, ia = compare_grads(p, host(ga), ga_o, bad, "g_a", spread=sa)
    ws, is_ = compare_grads(p, host(gs0), gs_o, bad, "g_s0", spread=ss)
    print("imu %s: worst rel g_a %.2e g_s0 %.2e; ill-conditioned %d, %d of %d" % (model, wa, ws, ia, is_, p["n_env"]))
    assert ia <= p["n_env"] // 2
