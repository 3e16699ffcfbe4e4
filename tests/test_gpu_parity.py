"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, at sizes the oracle finishes in seconds that still
span several CTAs, warps and ragged ray chunks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.autograd import DiffSimRollout, DiffSimStep
from paper_2509_10247_b300.binding import Simulator
from parity_util import (DEPTH_TOL, STATE_TF, TF_FLAGS, VALUE_FLAGS, Pair, compare_grads, compare_grads_strict,
                         compare_rollout, dev, grad_spread, host, masked_cotangents, teacher_forced_chain)

pytestmark = pytest.mark.gpu

# small cases with the structure of the paper's workloads
WORKLOADS = {
    "pm_64env": lambda: synth.preset("pointmass_64env_depth16x9_10sph"),
    "rigid_depth": lambda: synth.preset("rigid_4096env_depth64x48_40sph20box", n_env=24, horizon=12),
    "swarm_maps": lambda: synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=48, horizon=12),
    "rigid_lidar": lambda: synth.preset("rigid_65536env_256obst_depth_lidar", n_env=6, horizon=6,
                                        ckpt_every=4),
    "pm_discrete": lambda: synth.params(model="pm_disc", n_env=40, horizon=10, cam=(16, 9, 90.0, 10.0),
                                        map_counts=[(30, 15)], n_maps=5, obst_lo=(-6, -6, -6), obst_hi=(6, 6, 6),
                                        w_obs=5.0, terminate=1, ckpt_every=4),
    "simple_quad": lambda: synth.params(model="simple", n_env=40, horizon=10, cam=(12, 8, 90.0, 10.0),
                                        lidar=(4, 32, -15.0, 15.0, 10.0), map_counts=[(30, 15)], n_maps=5,
                                        obst_lo=(-6, -6, -6), obst_hi=(6, 6, 6), w_obs=5.0, pos_sq=0,
                                        terminate=1, ckpt_every=4),
    "cyl_gate": lambda: synth.params(model="rigid", n_env=40, horizon=10, dt=0.01, cam=(16, 9, 90.0, 12.0),
                                     lidar=(4, 48, -15.0, 15.0, 12.0),
                                     map_counts=[(10, 5, 8, 4), (0, 0, 6, 6), (5, 0, 0, 3)], n_maps=3,
                                     obst_lo=(-6, -6, -3), obst_hi=(6, 6, 3), race_radius=4.0, w_obs=5.0,
                                     pos_sq=0, terminate=1, ckpt_every=4),
    "ragged": lambda: synth.params(n_env=37, n_agent=3, horizon=7, cam=(7, 5, 75.0, 9.0),
                                   map_counts=[(5, 3), (0, 4), (6, 0), (0, 0)], n_maps=4,
                                   w_obs=3.0, w_agent=2.0, d_agent=1.5, terminate=1, ckpt_every=3),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def pair(request):
    torch.cuda.init()
    p = WORKLOADS[request.param]()
    pr = Pair(p, seed=0)
    pr.run_oracle()
    pr.run_gpu()
    pr.name = request.param
    return pr


def test_rollout_parity(pair):
    compare_rollout(pair.p, pair.rec, pair.out, pair.sT)


def test_teacher_forced_steps(pair):
    """oracle state s_t (rounded to FP32) -> one GPU step vs one oracle step."""
    p, rec = pair.p, pair.rec
    T = rec["r_ctrl"].shape[0]
    sim = pair.sim
    o1 = pair.orc.with_horizon(1)
    M = p["n_agent"]
    for t in sorted(set([0, 1, T // 2, T - 1])):
        s32 = rec["states"][t].astype(np.float32).astype(np.float64)
        a = pair.inp["actions"][t:t + 1]
        # reset counters the oracle reached by step t; the GPU's restart at 0,
        # so envs that reset at this step with a non-zero counter are skipped
        pk = np.zeros(p["n_env"], np.int32)
        if t > 0:
            pk = rec["done"][:t].reshape(t, p["n_env"], M)[:, :, 0].sum(axis=0).astype(np.int32)
        ro = o1.rollout(s32, a, pool_k=pk)
        sim.reset(dev(s32))
        o = sim.step(dev(a[0]))
        s = host(sim.get_state())
        so = ro["states"][1]
        skip_env = (ro["done"][0].reshape(p["n_env"], M)[:, 0] != 0) & (pk != 0)
        skip = np.repeat(skip_env, M) | ((ro["amb_step"][0] & 1) != 0)
        ok = np.abs(s - so) <= STATE_TF * np.maximum(np.abs(so), 1.0)
        assert ok[~skip].all(), (t, np.abs(s - so)[~skip].max())
        np.testing.assert_array_equal(host(o["done"]).astype(np.uint8)[~skip], ro["done"][0][~skip])
        for key, ak in (("depth", "amb_cam"), ("lidar", "amb_lid")):
            if o[key] is None:
                continue
            d = np.abs(host(o[key]) - ro[key][0])
            m = ((ro[ak][0] & VALUE_FLAGS) == 0) & ~skip[:, None]
            assert (d[m] <= DEPTH_TOL).all(), (key, d[m].max())


def test_render_parity(pair):
    rec = pair.rec
    T = rec["r_ctrl"].shape[0]
    s32 = rec["states"][T // 2].astype(np.float32).astype(np.float64)
    pair.sim.reset(dev(s32))
    dep, lid = pair.sim.render()
    od, ol, _, _, ac, al = pair.orc.render(s32)
    if dep is not None:
        m = (ac & VALUE_FLAGS) == 0
        assert (np.abs(host(dep) - od)[m] <= DEPTH_TOL).all()
    if lid is not None:
        m = (al & VALUE_FLAGS) == 0
        assert (np.abs(host(lid) - ol)[m] <= DEPTH_TOL).all()


def test_backward_parity(pair):
    """Full-horizon BPTT gradient vs the oracle's, conditioning-aware."""
    p, rec = pair.p, pair.rec
    bad = compare_rollout(p, rec, pair.out, pair.sT, check_depth=False)
    g_r, g_d, g_l = masked_cotangents(p, rec)
    g_sT = np.random.default_rng(3).standard_normal((pair.orc.NM, pair.orc.D)).astype(np.float32).astype(np.float64)
    ga_o, gs_o = pair.orc.backward(rec, g_r, g_d, g_l, g_sT)
    sa, ss = grad_spread(pair.orc, p, pair.inp, rec, g_r, g_d, g_l, g_sT)
    pair.sim.reset(dev(pair.inp["s0"]))
    pair.sim.rollout(pair.act)
    ga, gs0 = pair.sim.backward(dev(g_r), None if g_d is None else dev(g_d),
                                None if g_l is None else dev(g_l), dev(g_sT))
    torch.cuda.synchronize()
    wa, ia = compare_grads(p, host(ga), ga_o, bad, "g_a", spread=sa)
    ws, is_ = compare_grads(p, host(gs0), gs_o, bad, "g_s0", spread=ss)
    print("%s: worst rel g_a %.2e g_s0 %.2e within the 1e-3 bar; on the widened bar %d, %d of %d"
          % (pair.name, wa, ws, ia, is_, p["n_env"]))


def test_trajectory_teacher_forced_adjoint(pair):
    """Eq. 5 over the whole horizon without FP32 trajectory drift: the GPU's
    step adjoint chained from t = T-1 down to 0 at the oracle's own states
    (rounded to FP32), carrying its own state cotangent, against the oracle's
    BPTT gradient.  Every environment at the plain 1e-3 bar, no carve-out."""
    p, rec = pair.p, pair.rec
    if p.get("task", "reach") != "reach":
        pytest.skip("step adjoint: reaching task only")
    rep = {}
    g_r, g_d, g_l = masked_cotangents(p, rec, seed=12, ray_flags=TF_FLAGS, report=rep)
    g_sT = np.random.default_rng(13).standard_normal((pair.orc.NM, pair.orc.D)).astype(np.float32).astype(np.float64)
    ga_o, gs_o = pair.orc.backward(rec, g_r, g_d, g_l, g_sT)
    ga, gs = teacher_forced_chain(pair.sim, p, rec, pair.act, np.arange(pair.sim.NM), g_r, g_d, g_l, g_sT)
    assert pair.sim.status() == 0
    ra = compare_grads_strict(p, ga, ga_o, "g_a")
    rs = compare_grads_strict(p, gs, gs_o, "g_s0")
    print("%s teacher-forced chain: worst rel g_a %.2e g_s0 %.2e over all %d envs; %.2e of ray cotangents masked"
          % (pair.name, ra.max(), rs.max(), p["n_env"], rep["masked"]))


def test_teacher_forced_adjoint(pair):
    """One step's vector-Jacobian product from the oracle's state s_t (rounded
    to FP32), with the same cotangents on both sides: the adjoint math
    without trajectory drift, at the strict 1e-3 bar."""
    p, rec = pair.p, pair.rec
    T, M, NM, D = rec["r_ctrl"].shape[0], p["n_agent"], pair.orc.NM, pair.orc.D
    o1 = pair.orc.with_horizon(1)
    rng = np.random.default_rng(11)
    for t in sorted(set([0, 1, T // 2, T - 1])):
        s32 = rec["states"][t].astype(np.float32).astype(np.float64)
        a = pair.inp["actions"][t:t + 1]
        pk = np.zeros(p["n_env"], np.int32)
        if t > 0:
            pk = rec["done"][:t].reshape(t, p["n_env"], M)[:, :, 0].sum(axis=0).astype(np.int32)
        r1 = o1.rollout(s32, a, pool_k=pk)
        g_r, g_d, g_l = masked_cotangents(dict(p, horizon=1), r1, seed=20 + t)
        g_sn = rng.standard_normal((NM, D)).astype(np.float32).astype(np.float64)
        ga_o, gs_o = o1.backward(r1, g_r, g_d, g_l, g_sn)
        # conditioning of this step's VJP: perturb s_t by ~2 FP32 ulps
        sa = np.zeros(p["n_env"]); ss = np.zeros(p["n_env"])
        for k in range(2):
            s2 = s32 * (1 + 1.2e-7 * rng.standard_normal(s32.shape))
            r2 = o1.rollout(s2, a, pool_k=pk)
            ga2, gs2 = o1.backward(r2, g_r, g_d, g_l, g_sn)
            for e in range(p["n_env"]):
                sl = slice(e * M, (e + 1) * M)
                if (r2["done"][:, sl] != r1["done"][:, sl]).any():
                    sa[e] = ss[e] = np.inf
                    continue
                sa[e] = max(sa[e], np.linalg.norm(ga2[:, sl] - ga_o[:, sl]) / max(np.linalg.norm(ga_o[:, sl]), 1e-4))
                ss[e] = max(ss[e], np.linalg.norm(gs2[sl] - gs_o[sl]) / max(np.linalg.norm(gs_o[sl]), 1e-4))
        ga, gs = pair.sim.step_backward(dev(s32), dev(a[0]), dev(r1["done"][0], torch.uint8), dev(g_sn),
                                        dev(g_r[0]), None if g_d is None else dev(g_d[0]),
                                        None if g_l is None else dev(g_l[0]))
        torch.cuda.synchronize()
        bad = (r1["amb_step"][0] & 1).reshape(p["n_env"], M).any(axis=1)
        _, ia = compare_grads(p, host(ga)[None], ga_o, bad, "g_a step %d" % t, spread=sa)
        _, is_ = compare_grads(p, host(gs), gs_o, bad, "g_s step %d" % t, spread=ss)
        assert ia <= max(1, p["n_env"] // 10) and is_ <= max(1, p["n_env"] // 10)



def test_step_backward_with_recorded_hits_matches_recast(pair):
    """sim_render_taped of the state a step produces records each ray's hit;
    the step adjoint gathering those hits equals the re-casting one bit for
    bit (both sensors, and a cotangent on one sensor only)."""
    p = pair.p
    if p["cam"] is None and p["lidar"] is None:
        pytest.skip("no sensor")
    if p.get("task", "reach") != "reach":
        pytest.skip("step adjoint: reaching task only")
    sim = Simulator(p, pair.inp)
    sim.reset(dev(pair.inp["s0"]))
    o = sim.step(pair.act[0])
    o = sim.step(pair.act[1])  # a state away from the initial one
    s_t = sim.get_state().clone()
    o = sim.step(pair.act[2])
    hits = sim.hit_buffers()
    depth, lidar = sim.render(hits=hits)
    if depth is not None:
        assert torch.equal(depth, o["depth"])
        assert int(hits[0].min()) >= -2 and int(hits[0].max()) < 32767
    if lidar is not None:
        assert torch.equal(lidar, o["lidar"])
    g = torch.Generator(device="cuda").manual_seed(5)
    rn = lambda *s: torch.randn(*s, device="cuda", generator=g)
    g_sn, g_r = rn(sim.NM, sim.D), rn(sim.NM)
    g_d = rn(sim.NM, sim.Rc) if sim.Rc else None
    g_l = rn(sim.NM, sim.Rl) if sim.Rl else None
    a2 = pair.act[2]
    cases = [(g_d, g_l, hits)]
    if sim.Rc and sim.Rl:
        cases.append((None, g_l, (None, hits[1])))
        cases.append((g_d, None, (hits[0], None)))
    for gd, gl, hh in cases:
        ga0, gs0 = sim.step_backward(s_t, a2, o["done"], g_sn, g_r, gd, gl)
        ga1, gs1 = sim.step_backward(s_t, a2, o["done"], g_sn, g_r, gd, gl, hits=hh)
        torch.cuda.synchronize()
        assert torch.equal(ga0, ga1) and torch.equal(gs0, gs1)
    assert sim.status() == 0
    if sim.Rc and sim.Rl:
        with pytest.raises(RuntimeError):  # a cotangent without its sensor's hits
            sim.step_backward(s_t, a2, o["done"], g_sn, g_r, g_d, g_l, hits=(None, hits[1]))


def test_render_from_hits_matches_render(pair):
    """sim_render_hits rebuilds a state's depth / LiDAR from the hit ids that
    sim_step_ex or sim_render_taped recorded for it, equal to a full render
    bit for bit (every primitive kind, misses, clamps, origins inside)."""
    p = pair.p
    if p["cam"] is None and p["lidar"] is None:
        pytest.skip("no sensor")
    sim = Simulator(p, pair.inp)
    sim.reset(dev(pair.inp["s0"]))
    for t in range(3):
        hits = sim.hit_buffers()
        o = sim.step(pair.act[t], hits=hits)
        depth, lidar = sim.render_from_hits(hits)
        for got, ref in ((depth, o["depth"]), (lidar, o["lidar"])):
            if ref is not None:
                assert torch.equal(got, ref), t
        d2, l2 = sim.render()
        for got, ref in ((d2, o["depth"]), (l2, o["lidar"])):
            if ref is not None:
                assert torch.equal(got, ref), t
        h2 = sim.hit_buffers()
        sim.render(hits=h2)
        for a, b in zip(hits, h2):
            if a is not None:
                assert torch.equal(a, b)
    torch.cuda.synchronize()
    assert sim.status() == 0

def test_culling_is_result_preserving(pair):
    p = pair.p
    if p["cam"] is None and p["lidar"] is None:
        pytest.skip("no sensor")
    outs = {}
    for mode in (0, 1, 2):
        s2 = Simulator(p, pair.inp, cull=mode)
        s2.reset(dev(pair.inp["s0"]))
        outs[mode] = s2.rollout(pair.act)
    for mode in (1, 2):
        for k in ("depth", "lidar"):
            if pair.out[k] is not None:
                assert torch.equal(outs[0][k], outs[mode][k]), (mode, k)
        assert torch.equal(outs[0]["r_ctrl"], outs[mode]["r_ctrl"])
    for k in ("depth", "lidar"):
        if pair.out[k] is not None:
            assert torch.equal(pair.out[k], outs[0][k]), k


def test_steps_equal_rollout(pair):
    """T launches of the one-step kernel reproduce the persistent rollout bitwise."""
    p = pair.p
    sim = pair.sim
    sim.reset(dev(pair.inp["s0"]))
    for t in range(p["horizon"]):
        o = sim.step(pair.act[t])
        assert torch.equal(o["r_ctrl"], pair.out["r_ctrl"][t])
        assert torch.equal(o["done"], pair.out["done"][t])
        if o["depth"] is not None:
            assert torch.equal(o["depth"], pair.out["depth"][t])
    assert torch.equal(sim.get_state(), pair.sT)


def test_launch_shape_variants_agree(pair):
    """Rays per thread, warps per CTA, culling mode and thread- or
    warp-per-ray casting change only the work split: outputs and adjoint
    gradients agree bit for bit."""
    p = pair.p
    if p["cam"] is None:
        pytest.skip("no camera")
    cot = synth.cotangents(p, seed=9)
    g_r = dev(cot["g_r"])
    g_d = dev(cot["g_depth"])
    g_l = dev(cot["g_lidar"]) if "g_lidar" in cot else None
    ref = None
    for ex in (dict(), dict(rays_per_thread=1), dict(rays_per_thread=3, warps_per_cta=4),
               dict(rays_per_thread=8, cull=2), dict(rays_per_thread=2, cull=1, tape_hits=0),
               dict(cast_mode=1), dict(cast_mode=1, cull=2, rays_per_thread=4), dict(cast_mode=1, cull=0)):
        s2 = Simulator(p, pair.inp, **ex)
        s2.reset(dev(pair.inp["s0"]))
        o2 = s2.rollout(pair.act)
        ga, gs = s2.backward(g_r, g_d, g_l)
        assert torch.equal(pair.out["depth"], o2["depth"]), ex
        if pair.out["lidar"] is not None:
            assert torch.equal(pair.out["lidar"], o2["lidar"]), ex
        if ref is None:
            ref = (ga, gs)
        else:
            assert torch.equal(ref[0], ga) and torch.equal(ref[1], gs), ex


def test_checkpoint_and_tape_variants_agree(pair):
    """Gradients do not depend on the checkpoint interval or on taping hits."""
    p = pair.p
    g_r = dev(synth.cotangents(p, seed=4)["g_r"])
    cot = synth.cotangents(p, seed=4)
    g_d = dev(cot["g_depth"]) if "g_depth" in cot else None
    g_l = dev(cot["g_lidar"]) if "g_lidar" in cot else None
    ref = None
    for ex in (dict(ckpt_every=1, tape_hits=1), dict(ckpt_every=p["horizon"], tape_hits=0),
               dict(ckpt_every=5, tape_hits=0), dict(ckpt_every=3, tape_hits=1)):
        s2 = Simulator(p, pair.inp, **ex)
        s2.reset(dev(pair.inp["s0"]))
        s2.rollout(pair.act)
        ga, gs = s2.backward(g_r, g_d, g_l)
        if ref is None:
            ref = (ga, gs)
        else:
            assert torch.equal(ref[0], ga), ex
            assert torch.equal(ref[1], gs), ex


def test_determinism(pair):
    p = pair.p
    outs = []
    for _ in range(2):
        pair.sim.reset(dev(pair.inp["s0"]))
        o = pair.sim.rollout(pair.act)
        ga, gs = pair.sim.backward(dev(synth.cotangents(p, seed=2)["g_r"]))
        outs.append((o["r_ctrl"].clone(), ga.clone(), gs.clone()))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_autograd_rollout_matches_backward(pair):
    p = pair.p
    act = pair.act.clone().requires_grad_(True)
    s0 = dev(pair.inp["s0"]).requires_grad_(True)
    r, depth, lidar, sT = DiffSimRollout.apply(pair.sim, act, s0)
    cot = synth.cotangents(p, seed=6)
    loss = (r * dev(cot["g_r"])).sum()
    if depth.numel():
        loss = loss + (depth * dev(cot["g_depth"])).sum()
    loss.backward()
    pair.sim.reset(dev(pair.inp["s0"]))
    pair.sim.rollout(pair.act)
    ga, gs = pair.sim.backward(dev(cot["g_r"]), dev(cot["g_depth"]) if depth.numel() else None)
    assert torch.equal(act.grad, ga)
    assert torch.equal(s0.grad, gs)


def test_step_adjoint_chain_matches_rollout_adjoint(pair):
    """Closed-loop form: DiffSimStep over T steps gives the rollout's gradient."""
    p = pair.p
    pair.sim.reset(dev(pair.inp["s0"]))  # zero the reset counters, as the rollout does
    s = dev(pair.inp["s0"]).requires_grad_(True)
    acts = [pair.act[t].clone().requires_grad_(True) for t in range(p["horizon"])]
    cot = synth.cotangents(p, seed=8)
    loss = 0.0
    x = s
    for t in range(p["horizon"]):
        x, r, depth, lidar, done = DiffSimStep.apply(pair.sim, x, acts[t])
        loss = loss + (r * dev(cot["g_r"][t])).sum()
        if depth.numel():
            loss = loss + (depth * dev(cot["g_depth"][t])).sum()
    loss.backward()
    pair.sim.reset(dev(pair.inp["s0"]))
    pair.sim.rollout(pair.act)
    ga, gs = pair.sim.backward(dev(cot["g_r"]), dev(cot["g_depth"]) if p["cam"] else None)
    g_chain = torch.stack([a.grad for a in acts])
    # resets replay from the pool in both; pool counters differ only after a
    # reset, whose cotangent is cut in both forms
    scale = ga.abs().max().item()
    assert (g_chain - ga).abs().max().item() <= 1e-5 * max(scale, 1.0)
    assert (s.grad - gs).abs().max().item() <= 1e-5 * max(gs.abs().max().item(), 1.0)


def test_cull_counters_match_oracle_count(pair):
    """The render kernel's own post-cull test counters (the work the
    roofline credits) against the oracle's independent count of the same
    frustum rule at the same states: equal, up to the tests that decisions
    within 1e-6 of a threshold could move (none in most cases)."""
    p = pair.p
    if p["cam"] is None and p["lidar"] is None:
        pytest.skip("no sensor")
    sim = Simulator(p, pair.inp, cull=1)
    T = pair.rec["r_ctrl"].shape[0]
    exact = 0
    for t in sorted(set([0, T // 2, T])):
        s32 = pair.rec["states"][t].astype(np.float32).astype(np.float64)
        sim.reset(dev(s32))
        sim.counters(reset=True)
        sim.render()
        c = sim.counters(reset=True)
        oc = pair.orc.cull_counts(s32)
        assert c["rays"] == oc["rays"], (t, c, oc)
        diff = abs(c["sphere_tests"] - oc["sphere_tests"]) + abs(c["box_tests"] - oc["other_tests"])
        assert diff <= oc["ambiguous"], (t, c, oc)
        exact += diff == 0
    assert exact >= 1
    # counting off: the same images, no counts
    s32 = pair.rec["states"][0].astype(np.float32).astype(np.float64)
    sim.reset(dev(s32))
    d_on = sim.render()
    sim.counters(reset=True)
    sim.set_counting(False)
    d_off = sim.render()
    c = sim.counters(reset=True)
    assert c["sphere_tests"] == 0 and c["box_tests"] == 0 and c["rays"] == 0, c
    for x, y in zip(d_on, d_off):
        if x is not None:
            assert torch.equal(x, y)
    sim.set_counting(True)
    sim.close()
