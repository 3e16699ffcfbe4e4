"""Closed-loop policy on the GPU (through the C ABI) against the FP64
oracle with bf16 rounding: the policy's forward and backward passes, and
the closed-loop policy gradient through the simulator's step adjoint.

Tolerances: as for the surrogate network, both sides round the same
operands to bf16; where an fp32 pre-activation sits within fp32 summation
error of a bf16 rounding boundary the two round to neighbouring values, a
change of at most 2^-8 |w h| per flipped activation; so every pre-tanh
output within 2^-5 of its absolute sum, the median within 1e-5.  Gradients:
relative norm error per parameter tensor, median elementwise error against
the tensor's largest entry."""
import numpy as np
import pytest
import torch

import oracle
from oracle import policy as PO
from oracle.surrogate import bf16_round
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.policy import ClosedLoop, Policy

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _tiny(n_env=16, horizon=4, **kw):
    p = synth.preset("rigid_65536env_256obst_depth_lidar", n_env=n_env, horizon=horizon, cam=(6, 4, 90.0, 10.0),
                     lidar=(2, 8, -15.0, 15.0, 10.0), map_counts=[(3, 2)], obst_lo=(2.0, -3.0, -1.0),
                     obst_hi=(7.0, 3.0, 3.0), init_lo=(-1.0, -1.0, 0.5), init_hi=(1.0, 1.0, 1.5),
                     bound_lo=(-np.inf,) * 3, bound_hi=(np.inf,) * 3, terminate=0, w_obs=5.0, d_safe=4.0)
    p.update(kw)
    return p


def _inputs(rng, n, Rc, Rl):
    s = np.zeros((n, 13))
    s[:, 0:3] = rng.uniform(-5, 5, (n, 3))
    q = rng.standard_normal((n, 4))
    s[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    s[:, 7:13] = rng.standard_normal((n, 6))
    tg = rng.uniform(-5, 5, (n, 3))
    dep = rng.uniform(0, 20, (n, Rc))
    lid = rng.uniform(0, 20, (n, Rl))
    f32 = lambda a: a.astype(np.float32)
    return f32(s), f32(tg), f32(dep), f32(lid)


@pytest.mark.parametrize("n,Rc,Rl", [(1, 24, 16), (200, 3072, 0), (130, 40, 5760)])
def test_policy_forward_and_backward_match_oracle(n, Rc, Rl):
    rng = np.random.default_rng(n + Rc)
    p = dict(cam=(Rc, 1, 90.0, 20.0) if Rc else None, lidar=(1, Rl, -15.0, 15.0, 20.0) if Rl else None)
    pol = Policy(n, Rc, 20.0, Rl, 20.0)
    flat = synth.policy_init(dict(p), seed=n, scale=2.0)
    pol.set_params(flat)
    P = PO.split(p, flat)
    s, tg, dep, lid = _inputs(rng, n, Rc, Rl)
    a = host(pol.act(dev(s), dev(tg), dev(dep) if Rc else None, dev(lid) if Rl else None))
    f = PO.forward(P, PO.features(p, s, tg, dep, lid))
    S = np.abs(f["h"]) @ np.abs(bf16_round(P["W2"])).T + np.abs(P["b2"])
    e = np.abs(np.arctanh(np.clip(a, -1 + 1e-7, 1 - 1e-7)) - f["u"]) / S
    sat = np.abs(f["y"]) > 0.999  # tanh saturated: u is not resolvable from a
    assert (e[~sat] <= 2.0 ** -5).all() and np.median(e[~sat]) <= 1e-5, (e.max(), np.median(e))
    # backward
    ga = rng.standard_normal((n, 4)).astype(np.float32)
    g_s = rng.standard_normal((n, 13)).astype(np.float32)
    gs_dev = dev(g_s)
    g_dep = torch.empty(n, Rc, device="cuda") if Rc else None
    g_lid = torch.empty(n, Rl, device="cuda") if Rl else None
    pol.backward(dev(ga), gs_dev, g_dep, g_lid)
    grads = PO.split(p, pol.grads())
    assert pol.status() == 0
    go, g_obs = PO.backward(P, f, ga)
    for k in go:
        rel = np.linalg.norm(grads[k] - go[k]) / max(np.linalg.norm(go[k]), 1e-30)
        assert rel <= 1e-2, (k, rel)
        assert np.median(np.abs(grads[k] - go[k])) <= 1e-4 * np.abs(go[k]).max(), k
    gs_o = g_s + PO.state_feature_vjp(g_obs[:, :16])
    np.testing.assert_allclose(host(gs_dev), gs_o, rtol=0, atol=2e-2 * np.abs(gs_o - g_s).max() + 1e-6)
    if Rc:
        ref = g_obs[:, 16:16 + Rc] / 20.0
        assert np.linalg.norm(host(g_dep) - ref) <= 1e-2 * np.linalg.norm(ref)
    if Rl:
        ref = g_obs[:, 16 + Rc:] / 20.0
        assert np.linalg.norm(host(g_lid) - ref) <= 1e-2 * np.linalg.norm(ref)


def test_closed_loop_gradient_matches_oracle():
    p = _tiny()
    inp = synth.make_inputs(p, seed=7)
    flat = synth.policy_init(p, seed=8)
    g_r = synth.cotangents(p, seed=9)["g_r"]
    cl = ClosedLoop(p, inp)
    cl.pol.set_params(flat)
    L, g, rec = cl.gradient(dev(inp["s0"]), dev(g_r), store_hits=True)
    L2, g2, _ = cl.gradient(dev(inp["s0"]), dev(g_r), store_hits=False)
    assert L2 == L and np.array_equal(g, g2)
    Lo, go, reco = PO.closed_loop(oracle.Oracle(p, inp), PO.split(p, flat), inp["s0"], g_r)
    print("closed loop: loss %.6f vs %.6f, max |da| %.2e" % (L, Lo, np.abs(host(rec["actions"]) - reco["actions"]).max()))
    assert abs(L - Lo) <= 1e-3 * abs(Lo)
    gg = PO.split(p, g)
    for k in go:
        rel = np.linalg.norm(gg[k] - go[k]) / np.linalg.norm(go[k])
        print(k, rel)
        assert rel <= 3e-2, (k, rel)


def test_closed_loop_full_width_observation():
    """The full-scale observation (16 + 64x48 depth + 16x360 LiDAR = 8848
    features) at 512 agents over 3 steps: gradient finite and the loop's
    recomputed forward reproduces the recorded actions."""
    p = synth.preset("rigid_65536env_256obst_depth_lidar", n_env=512, horizon=3)
    inp = synth.make_inputs(p, seed=3)
    cl = ClosedLoop(p, inp)
    cl.pol.set_params(synth.policy_init(p, seed=4))
    g_r = dev(synth.cotangents(p, seed=5)["g_r"])
    L, g, rec = cl.gradient(dev(inp["s0"]), g_r)
    assert np.isfinite(L) and np.isfinite(g).all() and np.abs(g).max() > 0
    assert cl.pol.status() == 0 and cl.sim.status() == 0
    L2, g2, rec2 = cl.gradient(dev(inp["s0"]), g_r)
    assert L2 == L and np.array_equal(g, g2)  # deterministic
    # kept hits (observations rebuilt from them) vs re-rendering: bit for bit
    L3, g3, _ = cl.gradient(dev(inp["s0"]), g_r, store_hits=not cl.stored_hits)
    assert L3 == L and np.array_equal(g, g3)


def test_closed_loop_checkpointed_segments_match_stored_states():
    """Checkpoints every K steps (state and reset counters) and the replay of
    each segment in the backward pass give the stored-trajectory gradient bit
    for bit, for K dividing T or not, with collisions that reset agents."""
    p = _tiny(n_env=64, horizon=7, terminate=1, bound_lo=(-np.inf, -np.inf, 0.7),
              bound_hi=(np.inf, np.inf, 1.3))
    inp = synth.make_inputs(p, seed=21)
    cl = ClosedLoop(p, inp)
    cl.pol.set_params(synth.policy_init(p, seed=22))
    g_r = dev(synth.cotangents(p, seed=23)["g_r"])
    s0 = dev(inp["s0"])
    L0, g0, rec0 = cl.gradient(s0, g_r, ckpt_every=0, store_hits=True)
    assert int(rec0["done"].sum()) > 0  # resets happen inside segments
    for K in (1, 2, 3, 4):
        L, g, rec = cl.gradient(s0, g_r, ckpt_every=K)
        assert L == L0 and np.array_equal(g, g0), K
        assert torch.equal(rec["done"], rec0["done"])
    assert cl.sim.status() == 0 and cl.pol.status() == 0
