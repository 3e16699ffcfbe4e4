"""CUDA-graph capture of reset + rollout + adjoint, per-kernel timing and
launch counting, all through the C ABI."""
import pytest
import torch

from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.binding import SimError, Simulator
from parity_util import dev

pytestmark = pytest.mark.gpu

CASES = {
    "swarm": lambda: synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=40, horizon=10),
    "rigid_lidar": lambda: synth.preset("rigid_65536env_256obst_depth_lidar", n_env=5, horizon=6,
                                        ckpt_every=4),
}


def _direct(sim, inp, act, g_r, g_d, g_l):
    sim.reset(dev(inp["s0"]))
    o = sim.rollout(act)
    ga, gs = sim.backward(g_r, g_d, g_l)
    return o, ga, gs


@pytest.mark.parametrize("case", list(CASES))
def test_graph_equals_direct_calls(case):
    p = CASES[case]()
    inp = synth.make_inputs(p, seed=3)
    cot = synth.cotangents(p, seed=5)
    sim = Simulator(p, inp)
    act, s0 = dev(inp["actions"]), dev(inp["s0"])
    g_r = dev(cot["g_r"])
    g_d = dev(cot["g_depth"]) if "g_depth" in cot else None
    g_l = dev(cot["g_lidar"]) if "g_lidar" in cot else None
    o_ref, ga_ref, gs_ref = _direct(sim, inp, act, g_r, g_d, g_l)
    o_ref = {k: None if v is None else v.clone() for k, v in o_ref.items()}
    ga_ref, gs_ref = ga_ref.clone(), gs_ref.clone()
    g = sim.graph(act, s0=s0, g_r=g_r, g_depth=g_d, g_lidar=g_l)
    assert g.kernels == 4
    sim.kernel_times(reset=True)
    for _ in range(2):  # a graph replays: the second launch starts from s0 again
        g.launch()
        torch.cuda.synchronize()
        for k, v in o_ref.items():
            if v is not None:
                assert torch.equal(g.out[k], v), k
        assert torch.equal(g.tensors["g_a"], ga_ref)
        assert torch.equal(g.tensors["g_s0"], gs_ref)
    kt = sim.kernel_times(reset=True)
    assert [kt[k][1] for k in ("physics", "render", "render_vjp", "physics_bwd")] == [2, 2, 2, 2]
    # the handle holds the graph's rollout: a direct backward reproduces its gradient
    ga2, gs2 = sim.backward(g_r, g_d, g_l)
    assert torch.equal(ga2, ga_ref) and torch.equal(gs2, gs_ref)
    assert sim.status() == 0
    g.close()


def test_graph_forward_only_and_pool_reset():
    p = CASES["swarm"]()
    inp = synth.make_inputs(p, seed=4)
    sim = Simulator(p, inp)
    act = dev(inp["actions"])
    g = sim.graph(act)  # no s0: pool entry 0, no adjoint
    assert g.kernels == 2
    g.launch()
    sim.reset(None)
    o = sim.rollout(act)
    torch.cuda.synchronize()
    assert torch.equal(g.out["depth"], o["depth"]) and torch.equal(g.out["r_ctrl"], o["r_ctrl"])


def test_graph_refuses_after_scene_change_and_handle_destroy():
    p = CASES["swarm"]()
    inp = synth.make_inputs(p, seed=4)
    sim = Simulator(p, inp)
    act = dev(inp["actions"])
    g = sim.graph(act, s0=dev(inp["s0"]))
    g.launch()
    torch.cuda.synchronize()
    from paper_2509_10247_b300 import binding
    binding.sim_set_scene(sim.h, inp["spheres"], inp["sph_off"], inp["boxes"], inp["box_off"],
                          inp["env_map"], inp["targets"])
    with pytest.raises(SimError) as e:
        g.launch()
    assert e.value.code == -5
    g2 = sim.graph(act, s0=dev(inp["s0"]))
    g2.launch()
    torch.cuda.synchronize()
    sim.close()
    with pytest.raises(SimError) as e:
        g2.launch()
    assert e.value.code == -5
    g2.close()
    g.close()


def test_kernel_times_cover_direct_launches():
    p = CASES["swarm"]()
    inp = synth.make_inputs(p, seed=1)
    cot = synth.cotangents(p, seed=1)
    sim = Simulator(p, inp)
    sim.profile(True)
    sim.kernel_times(reset=True)
    act = dev(inp["actions"])
    _direct(sim, inp, act, dev(cot["g_r"]), dev(cot["g_depth"]), None)
    kt = sim.kernel_times(reset=True)
    for k, (ms, n) in kt.items():
        assert n == 1 and ms > 0.0, k
    sim.profile(False)
    _direct(sim, inp, act, dev(cot["g_r"]), dev(cot["g_depth"]), None)
    kt = sim.kernel_times(reset=True)
    for k, (ms, n) in kt.items():
        assert n == 1 and ms == 0.0, k


def test_autotune_admits_candidates_and_runs(tmp_path):
    from paper_2509_10247_b300 import autotune
    p = CASES["swarm"]()
    inp = synth.make_inputs(p, seed=2)
    cands = [dict(rays_per_thread=r, warps_per_cta=w, cull=c, tape_hits=-1)
             for r, w, c in ((1, 8, 1), (5, 8, 2), (3, 4, 1), (8, 4, 2))]
    e = autotune.tune(p, inp, cands=cands, path=str(tmp_path / "t.json"), reps=1)
    # four render shapes, then the checkpoint intervals around the best one
    assert e["tried"] >= 4 and e["admitted"] == e["tried"], e
    sim = Simulator(p, inp, **e["exec"])
    sim.reset(dev(inp["s0"]))
    sim.rollout(dev(inp["actions"]))
    assert sim.status() == 0
