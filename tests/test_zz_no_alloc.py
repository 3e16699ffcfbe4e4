"""sim_step_static, the step for callers that cannot allocate device memory
(their device memory comes from a pool or arena they do not control, or was
fixed up front): every buffer is the caller's and the library's scratch is a
static device array.  Two calls in a row must give what sim_step gives for
the same inputs.  Collected last so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest
import torch

from paper_2509_10247_b300 import binding, synth
from paper_2509_10247_b300.binding import Simulator
from parity_util import DEPTH_TOL, STATE_TF

pytestmark = pytest.mark.gpu


def device_scene(inp, dev):
    """The scene in the library's device layout: per map, spheres (c, r) then
    boxes as (min, 0), (max, 0), all float4."""
    so, bo = inp["sph_off"], inp["box_off"]
    blocks, off, ns, nb = [], [], [], []
    n = 0
    for m in range(len(so) - 1):
        sp = inp["spheres"][so[m]:so[m + 1]].reshape(-1, 4)
        bx = inp["boxes"][bo[m]:bo[m + 1]].reshape(-1, 6)
        bb = np.zeros((2 * len(bx), 4))
        bb[0::2, :3] = bx[:, :3]
        bb[1::2, :3] = bx[:, 3:]
        blk = np.concatenate([sp, bb], axis=0)
        off.append(n)
        ns.append(len(sp))
        nb.append(len(bx))
        blocks.append(blk)
        n += len(blk)
    prims = torch.as_tensor(np.concatenate(blocks).astype(np.float32), device=dev).contiguous()
    i32 = lambda x: torch.as_tensor(np.asarray(x, np.int32), device=dev)
    return prims, i32(off), i32(ns), i32(nb), max(ns), max(nb)


@pytest.mark.parametrize("name,kw", [
    ("swarm_16384env_8agent_8maps_depth16x9", dict(n_env=40, horizon=2)),
    ("rigid_65536env_256obst_depth_lidar", dict(n_env=5, horizon=2)),
])
def test_static_step_matches_sim_step_twice(name, kw):
    dev = torch.device("cuda", 0)
    p = synth.preset(name, **kw)
    inp = synth.make_inputs(p, seed=3)
    f32 = lambda x: torch.as_tensor(np.asarray(x, np.float32), device=dev).contiguous()
    act = f32(inp["actions"])
    # reference: the handle-based sim_step, two steps
    sim = Simulator(p, inp, device=dev)
    sim.reset(f32(inp["s0"]))
    ref = []
    for t in range(2):
        o = sim.step(act[t])
        ref.append((sim.get_state().clone(), {k: (None if v is None else v.clone()) for k, v in o.items()}))
    # the static entry point on caller-owned buffers, two calls in a row
    prims, off, ns, nb, ns_max, nb_max = device_scene(inp, dev)
    cfg = binding.make_config(p)
    env_map = torch.as_tensor(inp["env_map"], device=dev)
    targets, pool = f32(inp["targets"]), f32(inp["pool"])
    state = f32(inp["s0"])
    pool_k = torch.zeros(p["n_env"], dtype=torch.int32, device=dev)
    NM = p["n_env"] * p["n_agent"]
    Rc = p["cam"][0] * p["cam"][1] if p["cam"] else 0
    Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] else 0
    for t in range(2):
        depth = torch.full((NM, Rc), -1.0, device=dev) if Rc else None
        lidar = torch.full((NM, Rl), -1.0, device=dev) if Rl else None
        r = torch.empty(NM, device=dev)
        g = torch.empty(NM, dtype=torch.int8, device=dev)
        d = torch.empty(NM, dtype=torch.uint8, device=dev)
        status = torch.full((1,), -1, dtype=torch.int32, device=dev)
        binding.sim_step_static(cfg, prims, off, ns, nb, ns_max, nb_max, env_map, targets, pool, state,
                                act[t], depth, lidar, r, g, d, pool_k, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, t
        s_ref, o_ref = ref[t]
        assert torch.all((state - s_ref).abs() <= STATE_TF * s_ref.abs().clamp(min=1.0)), t
        assert torch.all((r - o_ref["r_ctrl"]).abs() <= 1e-6 * o_ref["r_ctrl"].abs().clamp(min=1.0)), t
        assert torch.equal(g, o_ref["r_goal"]) and torch.equal(d, o_ref["done"]), t
        if Rc:
            assert torch.all((depth - o_ref["depth"]).abs() <= DEPTH_TOL), t
        if Rl:
            assert torch.all((lidar - o_ref["lidar"]).abs() <= DEPTH_TOL), t
    sim.close()


def test_static_step_flags_understated_map_capacity():
    """ns_max / nb_max size the kernel's shared-memory map block and cull
    lists; a map with more primitives is caught on the device before it is
    staged: SIM_STATUS_MAP_CAPACITY is reported and that map's environments
    are left untouched, while the others step as sim_step does."""
    dev = torch.device("cuda", 0)
    p = synth.preset("swarm_16384env_8agent_8maps_depth16x9", n_env=24, horizon=1)
    inp = synth.make_inputs(p, seed=4)
    f32 = lambda x: torch.as_tensor(np.asarray(x, np.float32), device=dev).contiguous()
    act = f32(inp["actions"])
    sim = Simulator(p, inp, device=dev)
    sim.reset(f32(inp["s0"]))
    o_ref = sim.step(act[0])
    s_ref = sim.get_state()
    prims, off, ns, nb, ns_max, nb_max = device_scene(inp, dev)
    n_s = np.diff(inp["sph_off"])
    big = int(np.argmax(n_s))
    cap = int(np.sort(n_s)[-2])  # below the largest map's sphere count only
    assert cap < n_s[big]
    cfg = binding.make_config(p)
    env_map = torch.as_tensor(inp["env_map"], device=dev)
    state = f32(inp["s0"])
    s_before = state.clone()
    NM = p["n_env"] * p["n_agent"]
    r = torch.full((NM,), 7.0, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    binding.sim_step_static(cfg, prims, off, ns, nb, cap, nb_max, env_map, f32(inp["targets"]), f32(inp["pool"]),
                            state, act[0], None, None, r, None, None, None, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 4  # SIM_STATUS_MAP_CAPACITY
    skipped = np.repeat(inp["env_map"] == big, p["n_agent"])
    sk = torch.as_tensor(skipped, device=dev)
    assert skipped.any() and (~skipped).any()
    assert torch.equal(state[sk], s_before[sk])
    assert torch.all(r[sk] == 7.0)
    kept = ~sk
    assert torch.all((state[kept] - s_ref[kept]).abs() <= STATE_TF * s_ref[kept].abs().clamp(min=1.0))
    assert torch.all((r[kept] - o_ref["r_ctrl"][kept]).abs() <= 1e-6 * o_ref["r_ctrl"][kept].abs().clamp(min=1.0))
    sim.close()


def test_static_step_rejects_oversized_ray_tables():
    p = synth.preset("pointmass_64env_depth16x9_10sph", n_env=2, cam=(128, 128, 90.0, 10.0))
    cfg = binding.make_config(p)
    dev = torch.device("cuda", 0)
    z = torch.zeros(16, device=dev)
    zi = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(binding.SimError) as e:
        binding.sim_step_static(cfg, z, zi, zi, zi, 0, 0, zi, z, None, z, z)
    assert e.value.code == -3
