"""Parity at the benchmark's full size (16384 environments x 8 agents, 64
steps, 8 obstacle maps) in the benchmark's launch configuration: the whole
batch runs on the GPU; sampled environments (two per map) are recomputed by
the oracle and compared one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.binding import Simulator
from parity_util import (TF_FLAGS, compare_grads, compare_grads_strict, compare_rollout, dev, grad_spread, host,
                         masked_cotangents, subset, teacher_forced_chain)

pytestmark = pytest.mark.gpu


def test_bench_workload_sampled_parity():
    import bench
    p = synth.preset(bench.WORKLOAD)
    inp = synth.make_inputs(p, seed=0)
    N, M, T = p["n_env"], p["n_agent"], p["horizon"]
    nmaps = synth.n_maps_of(p)
    envs = np.array(sorted({m + nmaps * k for m in range(nmaps) for k in (3, N // nmaps - 5)}))
    q, sub, rows = subset(p, inp, envs)
    orc = oracle.Oracle(q, sub)
    rec = orc.rollout(sub["s0"], sub["actions"])
    g_r_s, g_d_s, _ = masked_cotangents(q, rec, seed=1)

    sim = Simulator(p, inp, **bench.BENCH_EXEC)
    info = sim.launch_info()
    assert info["grid"] > 0
    sim.reset(dev(inp["s0"]))
    act = dev(inp["actions"])
    out = sim.rollout(act)
    sT = sim.get_state()
    torch.cuda.synchronize()
    assert sim.status() == 0
    out_s = {k: (None if v is None else v[:, torch.as_tensor(rows, device="cuda")]) for k, v in out.items()}
    bad = compare_rollout(q, rec, out_s, sT[torch.as_tensor(rows, device="cuda")])
    assert bad.sum() <= 1

    g_r = torch.zeros(T, N * M, device="cuda")
    g_d = torch.zeros(T, N * M, sim.Rc, device="cuda")
    ri = torch.as_tensor(rows, device="cuda")
    g_r[:, ri] = dev(g_r_s)
    g_d[:, ri] = dev(g_d_s)
    g_a, g_s0 = sim.backward(g_r, g_d)
    torch.cuda.synchronize()
    ga_o, gs_o = orc.backward(rec, g_r_s, g_d_s)
    sa, ss = grad_spread(orc, q, sub, rec, g_r_s, g_d_s)
    wa, ia = compare_grads(q, host(g_a[:, ri]), ga_o, bad, "g_a", spread=sa)
    ws, is_ = compare_grads(q, host(g_s0[ri]), gs_o, bad, "g_s0", spread=ss)
    print("full size: worst rel g_a %.2e g_s0 %.2e within the 1e-3 bar; on the widened bar %d, %d of %d"
          % (wa, ws, ia, is_, len(envs)))
    # environments outside the sample got zero cotangents: their gradient is 0
    mask = torch.ones(N * M, dtype=torch.bool, device="cuda")
    mask[ri] = False
    assert g_a[:, mask].abs().max().item() == 0.0
    sim.close()


def test_bench_workload_teacher_forced_adjoint_chain():
    """The headline gradient bar on the benchmark's full batch (16384
    environments x 8 agents, 64 steps) in its launch configuration, with no
    conditioning carve-out: the step adjoint (Eq. 5) is chained over all 64
    steps at the oracle's own trajectory (rounded to FP32) for 32 sampled
    environments (four per map), the rest of the batch at the GPU's own
    states; every sampled environment's g_a and g_s0 within 1e-3 of the
    oracle's BPTT gradient."""
    import bench
    p = synth.preset(bench.WORKLOAD)
    inp = synth.make_inputs(p, seed=0)
    N, M, T = p["n_env"], p["n_agent"], p["horizon"]
    nmaps = synth.n_maps_of(p)
    envs = np.array(sorted({m + nmaps * k for m in range(nmaps) for k in (1, 7, N // nmaps // 2, N // nmaps - 3)}))
    q, sub, rows = subset(p, inp, envs)
    orc = oracle.Oracle(q, sub)
    rec = orc.rollout(sub["s0"], sub["actions"])
    rep = {}
    g_r, g_d, _ = masked_cotangents(q, rec, seed=21, ray_flags=TF_FLAGS, report=rep)
    g_sT = np.random.default_rng(22).standard_normal((len(rows), orc.D)).astype(np.float32).astype(np.float64)
    ga_o, gs_o = orc.backward(rec, g_r, g_d, None, g_sT)

    sim = Simulator(p, inp, **bench.BENCH_EXEC)
    act = dev(inp["actions"])
    sim.reset(dev(inp["s0"]))
    states, dones = [sim.get_state()], []
    for t in range(T):
        o = sim.step(act[t])
        dones.append(o["done"])
        states.append(sim.get_state())
    ga, gs = teacher_forced_chain(sim, q, rec, act, rows, g_r, g_d, None, g_sT, s_other=states, done_other=dones)
    assert sim.status() == 0
    ra = compare_grads_strict(q, ga, ga_o, "g_a")
    rs = compare_grads_strict(q, gs, gs_o, "g_s0")
    print("full size teacher-forced chain: worst rel g_a %.2e g_s0 %.2e over all %d sampled envs; "
          "%.2e of ray cotangents masked" % (ra.max(), rs.max(), len(envs), rep["masked"]))
    sim.close()
