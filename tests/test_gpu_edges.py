"""Edge cases and host-visible failure reporting on the GPU: empty maps, an
origin inside an obstacle, a single environment and step, non-finite
actions (status word, no hang), call-order errors."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.binding import SimError, Simulator
from parity_util import (DEPTH_TOL, Pair, compare_grads, compare_rollout, dev, grad_spread, host,
                         masked_cotangents)

pytestmark = pytest.mark.gpu


def _scene(p, spheres=(), boxes=()):
    sp = np.array(spheres, float).reshape(-1, 4)
    bx = np.array(boxes, float).reshape(-1, 6)
    NM = p["n_env"] * p["n_agent"]
    D = synth.STATE_DIM[p["model"]]
    rng = np.random.default_rng(0)
    return dict(spheres=sp, sph_off=np.array([0, len(sp)], np.int32), boxes=bx,
                box_off=np.array([0, len(bx)], np.int32), env_map=np.zeros(p["n_env"], np.int32),
                targets=rng.uniform(-3, 3, (NM, 3)), pool=np.zeros((max(p["pool_size"], 1), NM, D)),
                s0=None, actions=None)


def test_empty_scene_reads_max_range():
    p = synth.params(n_env=5, horizon=4, map_counts=[(0, 0)])
    pr = Pair(p, seed=2)
    pr.run_oracle()
    out = pr.run_gpu()
    assert torch.all(out["depth"] == p["cam"][3])
    compare_rollout(p, pr.rec, out, pr.sT)


def test_origin_inside_obstacle_depth_zero_and_no_gradient():
    p = synth.params(model="rigid", n_env=2, horizon=2, cam=(8, 6, 90.0, 10.0), pos_sq=1)
    inp = _scene(p, spheres=[(0.0, 0.0, 0.0, 2.0)], boxes=[(5, -1, -1, 6, 1, 1)])
    s0 = np.zeros((2, 13))
    s0[:, 3] = 1.0
    s0[1, 0] = 4.0  # agent 1 outside the sphere, facing the box
    inp["s0"] = s0
    inp["actions"] = np.zeros((2, 2, 4))
    pr = Pair(p, inp=inp)
    rec = pr.run_oracle()
    out = pr.run_gpu()
    d = host(out["depth"])
    assert np.all(d[:, 0] == 0.0)
    assert np.all(np.abs(d[:, 1] - rec["depth"][:, 1]) <= DEPTH_TOL)
    g_d = np.random.default_rng(4).standard_normal((2, 2, 48))
    pr.sim.reset(dev(s0))
    pr.sim.rollout(pr.act)
    ga, gs = pr.sim.backward(dev(np.zeros((2, 2))), dev(g_d))
    ga_o, gs_o = pr.orc.backward(rec, np.zeros((2, 2)), g_d)
    np.testing.assert_allclose(host(gs)[0], 0.0, atol=0)
    compare_grads(p, host(ga), ga_o, np.zeros(2, bool), "g_a")


def test_single_env_single_step():
    p = synth.params(n_env=1, horizon=1, map_counts=[(3, 2)], w_obs=2.0, d_safe=3.0)
    pr = Pair(p, seed=5)
    rec = pr.run_oracle()
    out = pr.run_gpu()
    bad = compare_rollout(p, rec, out, pr.sT)
    g_r, g_d, _ = masked_cotangents(p, rec)
    ga, gs = pr.sim.backward(dev(g_r), dev(g_d))
    ga_o, gs_o = pr.orc.backward(rec, g_r, g_d)
    compare_grads(p, host(ga), ga_o, bad, "g_a")


def test_nonfinite_state_sets_status_and_returns():
    p = synth.params(n_env=4, horizon=3)
    inp = synth.make_inputs(p, seed=1)
    sim = Simulator(p, inp)
    s0 = dev(inp["s0"])
    s0[2, 4] = float("nan")
    sim.reset(s0)
    sim.rollout(dev(inp["actions"]))
    assert sim.status() & 1
    # the handle stays usable and the status word was cleared
    sim.reset(dev(inp["s0"]))
    sim.rollout(dev(inp["actions"]))
    assert sim.status() == 0


def test_call_order_errors():
    p = synth.params(n_env=2, horizon=2, terminate=1)
    inp = synth.make_inputs(p, seed=1)
    sim = Simulator(p, inp)
    with pytest.raises(SimError) as e:
        sim.backward(dev(np.zeros((2, 2))))
    assert e.value.code == -5


def test_map_too_large_for_shared_memory_is_rejected():
    p = synth.params(n_env=1, horizon=1, map_counts=[(20000, 0)])
    inp = synth.make_inputs(p, seed=1)
    with pytest.raises(SimError) as e:
        Simulator(p, inp)
    assert e.value.code == -3


def test_uneven_maps_long_horizon_ckpt():
    # T not a multiple of K, some empty maps, swarm of 5
    p = synth.params(n_env=23, n_agent=5, horizon=11, n_maps=3,
                     map_counts=[(0, 0), (9, 0), (0, 7)], w_obs=4.0, w_agent=3.0, d_agent=1.2,
                     terminate=1, ckpt_every=4)
    pr = Pair(p, seed=9)
    rec = pr.run_oracle()
    out = pr.run_gpu()
    bad = compare_rollout(p, rec, out, pr.sT)
    g_r, g_d, _ = masked_cotangents(p, rec)
    ga, gs = pr.sim.backward(dev(g_r), dev(g_d))
    ga_o, gs_o = pr.orc.backward(rec, g_r, g_d)
    sa, ss = grad_spread(pr.orc, p, pr.inp, rec, g_r, g_d)
    compare_grads(p, host(ga), ga_o, bad, "g_a", spread=sa)
    compare_grads(p, host(gs), gs_o, bad, "g_s0", spread=ss)


def test_foreign_hit_ids_stay_in_bounds():
    """Hit buffers that do not belong to the state (arbitrary int16 ids):
    the images rebuilt from them read the maximum range for ids outside the
    map, 0 for -2, and stay finite; the step adjoint gathering them ignores
    ids outside the map and reports no error."""
    p = synth.params(model="rigid", n_env=12, horizon=3, cam=(12, 8, 90.0, 10.0), lidar=(4, 32, -15.0, 15.0, 10.0),
                     map_counts=[(6, 3, 2, 2), (4, 2, 0, 0)], n_maps=2, obst_lo=(-6, -6, -3), obst_hi=(6, 6, 3))
    inp = synth.make_inputs(p, seed=4)
    sim = Simulator(p, inp)
    sim.reset(dev(inp["s0"]))
    rng = np.random.default_rng(9)
    hits = tuple(torch.as_tensor(rng.integers(-32768, 32768, (sim.NM, R)), dtype=torch.int16, device="cuda")
                 for R in (sim.Rc, sim.Rl))
    depth, lidar = sim.render_from_hits(hits)
    torch.cuda.synchronize()
    counts = np.diff(inp["sph_off"]) + np.diff(inp["box_off"]) + np.diff(inp["cyl_off"]) + np.diff(inp["gate_off"])
    n_of_agent = counts[inp["env_map"]].repeat(p["n_agent"])[:, None]
    for img, h, rng_max in ((depth, hits[0], p["cam"][3]), (lidar, hits[1], p["lidar"][4])):
        v, ids = host(img), host(h).astype(np.int64)
        assert np.isfinite(v).all() and (v <= rng_max).all()
        assert (v[(ids < -2) | (ids == -1) | (ids >= n_of_agent)] == np.float32(rng_max)).all()
        assert (v[ids == -2] == 0).all()
    a = dev(inp["actions"][0])
    s_t = sim.get_state().clone()
    o = sim.step(a)
    g = torch.ones(sim.NM, device="cuda")
    ga, gs = sim.step_backward(s_t, a, o["done"], torch.zeros(sim.NM, sim.D, device="cuda"), g,
                               torch.ones(sim.NM, sim.Rc, device="cuda"), torch.ones(sim.NM, sim.Rl, device="cuda"),
                               hits=hits)
    torch.cuda.synchronize()
    assert sim.status() in (0, 1)  # a foreign hit may give a non-finite gradient (flagged), never a fault


def test_bounded_wait_that_runs_out_is_reported_and_the_handle_recovers():
    """The first wait of every render CTA (for its map's bulk copy) limited
    to one non-blocking poll runs out before the copy lands: the kernels set
    SIM_STATUS_TIMEOUT, wait (bounded) for the copy in flight and stop, no
    hang and no fault; with the limit lifted the same handle reproduces the
    reference rollout and adjoint bit for bit."""
    p = synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=64, horizon=4)
    inp = synth.make_inputs(p, seed=3)
    sim = Simulator(p, inp)
    s0, act = dev(inp["s0"]), dev(inp["actions"])
    g_r = dev(synth.cotangents(p, seed=4)["g_r"])

    def run():
        sim.reset(s0)
        o = sim.rollout(act)
        ga, gs = sim.backward(g_r)
        torch.cuda.synchronize()
        return {k: (None if v is None else v.clone()) for k, v in o.items()}, ga.clone(), gs.clone()

    ref = run()
    assert sim.status() == 0
    sim.set_wait_limit(1)
    run()
    assert sim.status() & 2  # SIM_STATUS_TIMEOUT
    sim.set_wait_limit(0)
    again = run()
    assert sim.status() == 0
    for k in ("r_ctrl", "r_goal", "done", "depth"):
        assert torch.equal(ref[0][k], again[0][k]), k
    assert torch.equal(ref[1], again[1]) and torch.equal(ref[2], again[2])
    with pytest.raises(SimError):
        sim.set_wait_limit(-1)
    sim.close()
