#!/usr/bin/env python
"""Benchmark of the fused, batched, differentiable quadrotor step on B300.

One bench step = one pass of the whole hot path over one batch: a rollout of
T = 64 steps of 16384 environments x 8 point-mass agents (8 obstacle maps of
10..200 spheres/boxes, a 16x9 depth camera per agent, inter-agent collisions,
resets) in one persistent launch, then its adjoint (BPTT, Eq. 5) with a
reward cotangent and a depth cotangent.  `value` is environment steps per
second (env-steps/s) over all ranks, inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle (the only other implementation of
the method) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "swarm_16384env_8agent_8maps_depth16x9"
METRIC = "env-steps/s (fwd+adjoint, with depth) at 16k envs vs roofline; Grays/s"
UNIT = "env-steps/s"
# launch configuration of the full-size parity test, and of the bench when
# it runs untuned (--no-tune); otherwise the bench times the autotuner's pick
# for this GPU (every candidate bitwise equal to the library default)
BENCH_EXEC = dict(ckpt_every=4, tape_hits=1, cull=1)
# algorithmic work of one ray-primitive test after the per-origin list entry,
# in FP32-pipe instructions (an FMA counts once): sphere 6 (3 for b = d.oc,
# 1 for b^2 - C, 1 subtraction, 1 min / select; the square root of a hit
# runs on the SFU), box 14 (6 slab products, 6 per-axis min / max, the
# entry max and exit min).  The same tests in FLOP (an FMA counts twice):
# sphere 10, box 16.
OPS_SPHERE_TEST = 6
OPS_BOX_TEST = 14
FLOP_SPHERE_TEST = 10
FLOP_BOX_TEST = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="time BENCH_EXEC instead of the autotuner's pick")
    ap.add_argument("--surr-epochs", type=int, default=3)
    ap.add_argument("--horizon", type=int, default=None, help="override the horizon (closed-loop workload)")
    ap.add_argument("--policy-only", action="store_true",
                    help="closed-loop workload: time the policy's act and backward on rendered observations only")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0,
                    help="reference arm: oracle seconds per step (the sample size follows)")
    ap.add_argument("--n-env", type=int, default=None,
                    help="override the number of environments (profiling on a smaller case)")
    return ap.parse_args()


def workload_params(name, n_env=None):
    from paper_2509_10247_b300 import synth
    return synth.preset(name) if n_env is None else synth.preset(name, n_env=n_env)


# sources that define the render kernel and its launch (the DRAM traffic
# recorded in profiles/traffic.txt is valid while they are unchanged)
RENDER_SOURCES = ("sim_split.cu", "sim_raycast.cuh", "sim_kernels.cuh", "sim_device.cuh", "sim_api.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_10247_b300", "csrc")
    for f in RENDER_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def peak_fp32_tinst(num_sms, sm_mhz):
    # FP32-pipe issue: 128 lanes per SM, one instruction per lane and cycle
    return 128.0 * num_sms * sm_mhz * 1e6 / 1e12


def measured_peaks():
    """The measured HBM and bf16 peaks (MEASURED_PEAKS.json), else the
    recipe's fallback figures; returns (dict, basis)."""
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(f):
        return json.load(open(f)), "measured (MEASURED_PEAKS.json)"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def render_vjp_bytes(NM, T, R, parts):
    """Algorithmic DRAM bytes of one taped render-adjoint launch: per ray its
    hit id (2 B) and output cotangent (4 B); per (step, agent) item its pose
    (48 B) and done flag (1 B); per item part the pose cotangent written
    (48 B)."""
    items = T * NM
    return items * R * 6 + items * (48 + 1) + items * parts * 48


def config_of(p, extra=None):
    c = {"workload": p["name"], "n_env": p["n_env"], "n_agent": p["n_agent"],
         "horizon": p["horizon"], "model": p["model"],
         "camera": None if p["cam"] is None else "%dx%d" % (p["cam"][0], p["cam"][1]),
         "lidar": None if p["lidar"] is None else "%dx%d" % (p["lidar"][0], p["lidar"][1]),
         "obstacles_per_map": [a + b for a, b in p["map_counts"]],
         "global_batch": p["n_env"], "seq_len": p["horizon"], "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------- CPU oracle
def oracle_sample(p, inp, n_envs, threads=0):
    """Oracle rollout + adjoint on the first n_envs environments (all maps
    represented); returns (seconds, env_steps)."""
    import oracle
    from paper_2509_10247_b300 import synth
    envs = np.arange(n_envs)
    M = p["n_agent"]
    rows = (envs[:, None] * M + np.arange(M)[None, :]).reshape(-1)
    q = dict(p, n_env=n_envs)
    sub = dict(inp)
    sub["s0"], sub["targets"] = inp["s0"][rows], inp["targets"][rows]
    sub["pool"], sub["actions"] = inp["pool"][:, rows], inp["actions"][:, rows]
    sub["env_map"] = inp["env_map"][envs]
    o = oracle.Oracle(q, sub)
    cot = synth.cotangents(q, seed=1)
    t0 = time.perf_counter()
    rec = o.rollout(sub["s0"], sub["actions"], n_threads=threads)
    o.backward(rec, cot["g_r"], cot.get("g_depth"), cot.get("g_lidar"), n_threads=threads)
    return time.perf_counter() - t0, n_envs * p["horizon"]


def cpu_rate(p, inp, target_s):
    """env-steps/s of the oracle on a sample sized to about target_s seconds."""
    import oracle
    n = max(1, min(8, p["n_env"]))
    dt, steps = oracle_sample(p, inp, n)
    while dt < 0.7 * target_s and n < p["n_env"]:
        n = min(p["n_env"], max(n + 1, int(n * min(8.0, target_s / max(dt, 1e-3)))))
        dt, steps = oracle_sample(p, inp, n)
    return steps / dt, n, dt, oracle.max_threads()


# ------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    p = workload_params(args.workload, args.n_env)
    from paper_2509_10247_b300 import synth
    inp = synth.make_inputs(p, seed=args.seed)
    import oracle
    oracle.build()
    # size the per-step sample like the CPU baseline: enough environments
    # (all maps, every host core busy) for about --ref-seconds of oracle work
    _, n, _, _ = cpu_rate(p, inp, args.ref_seconds)
    for _ in range(args.warmup):
        oracle_sample(p, inp, n)
    times = []
    for _ in range(args.steps):
        dt, steps = oracle_sample(p, inp, n)
        times.append(dt)
    tot = sum(times)
    value = n * p["horizon"] * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": "%d of %d envs (all maps), full horizon, rollout + adjoint per step"
                                       % (n, p["n_env"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our arm
def max_over_ranks(ms, world, device=None):
    """The job's time: the slowest rank's (all ranks receive it)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_env_per_rank, horizon, steps, world, ms):
    """Whole-job env-steps/s: every rank simulates its own n_env environments
    (weak scaling), so the job does world times the work in the max time."""
    return n_env_per_rank * horizon * steps * world / (ms / 1e3)


def run_ours(args, rank, world):
    import torch
    from paper_2509_10247_b300 import build as B, synth
    from paper_2509_10247_b300.binding import Simulator
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workload_params(args.workload, args.n_env)
    inp = synth.make_inputs(p, seed=args.seed + rank)
    tuned = None
    exec_ = dict(BENCH_EXEC)
    if not args.no_tune:
        from paper_2509_10247_b300 import autotune
        t0 = time.perf_counter()
        tuned = autotune.tune(p, inp, device=dev, reps=2)
        tuned = dict(tuned, seconds=time.perf_counter() - t0)
        exec_ = dict(tuned["exec"])
    sim = Simulator(p, inp, device=dev, **exec_)
    T, NM, Rc = p["horizon"], sim.NM, sim.Rc
    s0 = torch.as_tensor(inp["s0"], dtype=torch.float32, device=dev)
    act = torch.as_tensor(inp["actions"], dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + rank)
    g_r = torch.randn(T, NM, device=dev, generator=g)
    g_d = torch.randn(T, NM, Rc, device=dev, generator=g) if Rc else None
    out = dict(r_ctrl=torch.empty(T, NM, device=dev), r_goal=torch.empty(T, NM, dtype=torch.int8, device=dev),
               done=torch.empty(T, NM, dtype=torch.uint8, device=dev),
               depth=torch.empty(T, NM, Rc, device=dev) if Rc else None, lidar=None)
    g_a = torch.empty(T, NM, sim.A, device=dev)
    g_s0 = torch.empty(NM, sim.D, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        sim.reset(s0)
        if ev:
            ev[0].record(stream)
        sim.rollout(act, out=out)
        if ev:
            ev[1].record(stream)
        sim.backward(g_r, g_d, None, None, g_a, g_s0)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sim.counters(reset=True)
    # one counted pass for the algorithmic work of a render launch
    step()
    cnt = sim.counters(reset=True)
    if sim.status() != 0:
        raise RuntimeError("device status flagged during warm-up")
    # the timed steps take the counts from that pass and skip the counting
    sim.set_counting(False)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    # the library brackets each of its kernel launches with CUDA events on the
    # launching stream: per-kernel device time inside the timed region
    sim.profile(True)
    sim.kernel_times(reset=True)
    clocks = Clocks(local) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop() if clocks else None
    kt = sim.kernel_times(reset=True)
    sim.profile(False)
    ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    fwd_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    bwd_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    if sim.status() != 0:
        raise RuntimeError("device status flagged during the timed region")
    value = job_throughput(p["n_env"], T, args.steps, world, ms)
    rays_per_step = NM * (Rc + sim.Rl) * T  # per rollout launch
    grays = rays_per_step * args.steps * world / (ms / 1e3) / 1e9
    launches = sum(n for _, n in kt.values())

    # the same pass captured once into a CUDA graph (reset + rollout + adjoint)
    graph = None
    if not args.no_graph:
        gr = sim.graph(act, s0=s0, out=out, g_r=g_r, g_depth=g_d, g_a=g_a, g_s0=g_s0)
        for _ in range(args.warmup):
            gr.launch()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            gr.launch()
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.steps
        graph = {"ms_per_step": gms, "value": p["n_env"] * T / (gms / 1e3), "kernels": gr.kernels}
        gr.close()
        if sim.status() != 0:
            raise RuntimeError("device status flagged during the graph replay")

    if rank != 0:
        return 0
    # roofline of the dominant kernel: k_render (FP32 ray casting), per launch;
    # the FP32 peak is measured on this GPU right after the timed region
    from paper_2509_10247_b300.binding import sim_fp32_issue_rate
    props = torch.cuda.get_device_properties(dev)
    fma_s, ffma2_s = sim_fp32_issue_rate(dev)
    ops = OPS_SPHERE_TEST * cnt["sphere_tests"] + OPS_BOX_TEST * cnt["box_tests"]
    flop = FLOP_SPHERE_TEST * cnt["sphere_tests"] + FLOP_BOX_TEST * cnt["box_tests"]
    render_ms = kt["render"][0] / max(kt["render"][1], 1)
    achieved = ops / (render_ms / 1e3) / 1e12
    peak = max(fma_s, ffma2_s) / 1e12
    sm_mhz = (ck or {}).get("sm_mhz") or 2032.0
    peak_derived = peak_fp32_tinst(props.multi_processor_count, sm_mhz)
    traffic = traffic_vjp = None
    tfile = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(tfile):
        tj = dict(l.split(": ", 1) for l in open(tfile).read().splitlines() if ": " in l and not l.startswith("#"))
        if tj.get("source_hash") == source_hash() and tj.get("workload") == p["name"]:
            traffic = float(tj["render_bytes_per_launch"]) if "render_bytes_per_launch" in tj else None
            traffic_vjp = float(tj["render_vjp_bytes_per_launch"]) if "render_vjp_bytes_per_launch" in tj else None
    per_kernel = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1]} for k, v in kt.items()}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_render (ray casting of all T steps)", "kernel_ms": render_ms,
                "peak_basis": "measured: FP32 multiply-adds per second of this GPU (sim_fp32_issue_rate, "
                              "scalar %.2f T/s, packed pairs %.2f T/s; the larger), right after the timed region"
                              % (fma_s / 1e12, ffma2_s / 1e12),
                "peak_derived_at_sampled_clock": peak_derived,
                "derived_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (median SM clock sampled in the timed "
                                 "region)" % (props.multi_processor_count, sm_mhz),
                "work_basis": "per test after culling: sphere %d, box %d FP32-pipe instructions"
                              % (OPS_SPHERE_TEST, OPS_BOX_TEST),
                "tests_per_launch": cnt["sphere_tests"] + cnt["box_tests"],
                "sphere_tests_per_launch": cnt["sphere_tests"], "box_tests_per_launch": cnt["box_tests"],
                "ops_per_launch": ops, "flop_per_launch": flop,
                "tflops": flop / (render_ms / 1e3) / 1e12, "frac_flop": flop / (render_ms / 1e3) / 1e12 / (2 * peak),
                "kernels": per_kernel}
    # second roofline: the ray adjoint (taped: reads hit ids and cotangents, HBM)
    vjp_ms = kt["render_vjp"][0] / max(kt["render_vjp"][1], 1)
    pk, pk_basis = measured_peaks()
    # the library splits a rollout adjoint's items into ceil(8 / (T M)) ray parts (at most 8)
    parts = min(8, max(1, -(-8 // (T * p["n_agent"]))))
    vjp_b = render_vjp_bytes(NM, T, Rc + sim.Rl, parts)
    roofline_vjp = {"bound": "hbm", "achieved": vjp_b / (vjp_ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                    "unit": "GB/s", "frac": vjp_b / (vjp_ms / 1e3) / 1e9 / pk["hbm_gbs"], "traffic": traffic_vjp,
                    "kernel": "k_render_vjp (taped ray adjoint of all T steps)", "kernel_ms": vjp_ms,
                    "bytes_per_launch": vjp_b, "peak_basis": pk_basis,
                    "work_basis": "per ray 2 B hit id + 4 B cotangent; per (step, agent) 48 B pose + 1 B done; "
                                  "per item part 48 B pose cotangent written"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(p),
            "l2": "inputs larger than L2: %.1f GB depth written and %.1f GB depth cotangent read per step"
                  % (4e-9 * T * NM * Rc, 4e-9 * T * NM * Rc),
            "exec": exec_,
            "autotune": None if tuned is None else dict(
                {k: tuned[k] for k in ("tried", "admitted", "ms", "default_ms", "seconds")},
                best_thread_per_ray_ms=min([r["ms"] for r in tuned.get("results", [])
                                            if r["ok"] and r["ms"] and not r["exec"].get("cast_mode")], default=None),
                best_warp_per_ray_ms=min([r["ms"] for r in tuned.get("results", [])
                                          if r["ok"] and r["ms"] and r["exec"].get("cast_mode") == 1], default=None)),
            "grays_per_s": grays, "agent_steps_per_s": value * p["n_agent"],
            "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
            "roofline": roofline, "roofline_render_vjp": roofline_vjp,
            "gpu_launches": launches, "clocks": ck, "graph": graph}
    # end to end: host actions and initial state in, rewards and action gradients out
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, sim, inp, dev, g_r, g_d, out, g_a, g_s0, p)
    if world == 1 and not args.no_cpu:
        rate, n, dt, cores = cpu_rate(p, inp, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d of %d envs (all maps), full horizon, rollout + adjoint, %.1f s"
                                          % (n, p["n_env"], dt)}
    print(json.dumps(line), flush=True)
    return 0


SURROGATE_WORKLOAD = "surrogate_rigid_65536env_32step"
SURR_TRANSITIONS = (65536, 153)  # envs x steps: 10.03M transitions of the rigid step
SURR_FLOP_PER_SAMPLE = 2 * (17 * 256 + 256 * 256 + 256 * 13)  # forward multiply-adds x 2


def run_surrogate(args, rank, world):
    """Learned surrogate of the rigid step: 10M simulator transitions, GPU
    training with the library's tensor-core kernels, then the 65536 x 32
    rollout timed against the plain GPU rigid step; the state error is taken
    against that plain step (itself held to the FP64 oracle by the tests)."""
    import torch
    from paper_2509_10247_b300 import build as B, synth
    from paper_2509_10247_b300.binding import Simulator
    from paper_2509_10247_b300.surrogate import Surrogate, collect_transitions, train
    B.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workload_params(SURROGATE_WORKLOAD, args.n_env)
    N, T = p["n_env"], p["horizon"]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # 1. transitions from the simulator's own rigid step
    e0, e1 = ev(), ev()
    e0.record()
    X, S1 = collect_transitions(p, n_env=SURR_TRANSITIONS[0], steps=SURR_TRANSITIONS[1], seed=args.seed + 100,
                                device=dev)
    e1.record()
    torch.cuda.synchronize()
    collect_ms = e0.elapsed_time(e1)
    # 2. training
    sur = Surrogate(p, batch=8192, device=dev)
    flat, _ = synth.surrogate_init(args.seed + 101)
    sur.set_params(flat)
    sur.fit_stats(X, S1)
    e0, e1 = ev(), ev()
    e0.record()
    losses = train(sur, X, S1, epochs=args.surr_epochs, seed=args.seed + 102)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    steps = args.surr_epochs * (X.shape[0] // 8192)
    if sur.status() != 0:
        raise RuntimeError("surrogate status flagged during training")
    # 3. rollout: surrogate vs plain rigid step, same states and actions
    inp = synth.make_inputs(p, seed=args.seed + 103)
    s0 = torch.as_tensor(inp["s0"], dtype=torch.float32, device=dev)
    act = torch.as_tensor(inp["actions"], dtype=torch.float32, device=dev)
    sim = Simulator(p, inp, device=dev)
    sim.profile(True)

    def plain():
        sim.reset(s0)
        return sim.rollout(act, depth=False, lidar=False)

    def surr():
        return sur.rollout(s0, act, states=False, fallback=True)

    for _ in range(args.warmup):
        plain(); surr()
    torch.cuda.synchronize()
    sim.kernel_times(reset=True)
    clocks = Clocks(local)
    times = {}
    for name, fn in (("surrogate", surr), ("plain", plain)):
        a0, a1 = ev(), ev()
        a0.record()
        for _ in range(args.steps):
            o = fn()
        a1.record()
        torch.cuda.synchronize()
        times[name] = a0.elapsed_time(a1) / args.steps
    ck = clocks.stop()
    so = surr()
    plain()
    ref = sim.get_state()
    torch.cuda.synchronize()
    d = (so["sT"] - ref).double()
    rmse = float(torch.sqrt(torch.mean(torch.sum(d[:, :3] ** 2, dim=1))))
    dq = torch.abs(torch.sum(so["sT"][:, 3:7].double() * ref[:, 3:7].double(), dim=1)).clamp(max=1.0)
    ang = float(torch.mean(2 * torch.acos(dq)))
    fb = float(so["fallback"].float().mean())
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1800.0}
    flop = SURR_FLOP_PER_SAMPLE * N * T
    achieved = flop / (times["surrogate"] / 1e3) / 1e12
    line = {"metric": "surrogate rollout env-steps/s at 65536 envs x 32 steps", "workload": SURROGATE_WORKLOAD,
            "value": N * T / (times["surrogate"] / 1e3), "unit": "env-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": times["surrogate"],
            "higher_is_better": True, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "plain_step": {"ms": times["plain"], "value": N * T / (times["plain"] / 1e3)},
            "speedup_vs_plain_step": times["plain"] / times["surrogate"],
            "state_error_vs_plain_step_t32": {"position_rmse_m": rmse, "attitude_mean_rad": ang,
                                              "fallback_fraction": fb},
            "training": {"transitions": int(X.shape[0]), "epochs": args.surr_epochs, "batch": 8192,
                         "steps": steps, "ms": train_ms, "samples_per_s": steps * 8192 / (train_ms / 1e3),
                         "tflops": 3 * SURR_FLOP_PER_SAMPLE * steps * 8192 / (train_ms / 1e3) / 1e12,
                         "loss_per_epoch": losses, "collect_ms": collect_ms},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops"], "traffic": None,
                         "kernel": "k_surr_fwd (fused persistent rollout)",
                         "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"},
            "clocks": ck}
    print(json.dumps(line), flush=True)
    return 0


CLOSED_LOOP_WORKLOAD = "rigid_65536env_256obst_depth_lidar"


def run_closed_loop(args, rank, world):
    """Closed-loop policy gradient at full scale: 65536 rigid agents, 256
    obstacles each, depth 64x48 + LiDAR 16x360, 128 steps; a two-layer policy
    (8848 -> 256 -> 4) acts on the rendered observations, and the gradient of
    the rollout's reward w.r.t. the policy parameters is taken by
    backpropagation through time (per step: re-render, policy forward, the
    simulator's step adjoint, the policy backward)."""
    import torch
    from paper_2509_10247_b300 import build as B, synth
    from paper_2509_10247_b300.policy import ClosedLoop
    B.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workload_params(CLOSED_LOOP_WORKLOAD, args.n_env)
    if args.horizon:
        p["horizon"] = args.horizon
    N, T = p["n_env"], p["horizon"]
    inp = synth.make_inputs(p, seed=args.seed, actions=False)
    cl = ClosedLoop(p, inp, device=dev)
    cl.pol.set_params(synth.policy_init(p, seed=args.seed + 1))
    s0 = torch.as_tensor(inp["s0"], dtype=torch.float32, device=dev)
    g_r = torch.full((T, N), -1.0 / (N * T), device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        cl.gradient(s0, g_r, T=2)
    torch.cuda.synchronize()
    # the policy's layer-1 GEMM (M = agents, N = 256, K = 8848): one act on rendered observations
    depth, lidar = cl.sim.render()
    a = torch.empty(N, 4, device=dev)
    cl.pol.act(s0, cl.targets, depth, lidar, out=a)
    e0, e1 = ev(), ev()
    reps = 20
    e0.record()
    for _ in range(reps):
        cl.pol.act(s0, cl.targets, depth, lidar, out=a)
    e1.record()
    torch.cuda.synchronize()
    act_ms = e0.elapsed_time(e1) / reps
    F = synth.policy_width(p)
    gemm_flop = 2.0 * N * F * 256
    if args.policy_only:
        g_a = torch.randn(N, 4, device=dev)
        g_s = torch.zeros(N, 13, device=dev)
        g_d, g_l = torch.empty_like(depth), torch.empty_like(lidar)
        cl.pol.backward(g_a, g_s, g_d, g_l)
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(reps):
            cl.pol.backward(g_a, g_s, g_d, g_l)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"metric": "policy act / backward ms at %d agents x %d features" % (N, F),
                          "workload": CLOSED_LOOP_WORKLOAD, "act_ms": act_ms,
                          "backward_ms": e0.elapsed_time(e1) / reps, "reps": reps}))
        return
    K = p.get("ckpt_every", 16)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    base_mem = torch.cuda.memory_allocated(dev)
    clocks = Clocks(local)
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(args.steps):
        L, g, rec = cl.gradient(s0, g_r, ckpt_every=K)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    peak_gb = (torch.cuda.max_memory_allocated(dev) - base_mem) / 1e9
    if cl.sim.status() != 0 or cl.pol.status() != 0:
        raise RuntimeError("device status flagged in the closed loop")
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1800.0}
    line = {"metric": "closed-loop policy-gradient env-steps/s (fwd + BPTT, depth 64x48 + LiDAR 16x360)",
            "workload": CLOSED_LOOP_WORKLOAD, "value": N * T / (ms / 1e3), "unit": "env-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32 simulator, bf16 policy (fp32 accumulate)", "data": "synthetic",
            "config": {"n_env": N, "horizon": T, "policy": "%d -> 256 -> 4" % F, "obstacles": 256,
                       "ckpt_every": K,
                       "backward": "checkpoints (state, reset counters) every %d steps; each segment replayed "
                                   "in the backward pass, its observations rebuilt from the replay's hit ids "
                                   "(%.1f GB per segment)" % (K, cl.hits_bytes(K + 1) / 1e9)},
            "peak_gb_per_gradient": peak_gb,
            "simulator_workspace_gb": cl.sim.workspace_bytes() / 1e9,
            "loss": L, "grad_norm": float(np.linalg.norm(g)),
            "policy_act_ms": act_ms,
            "roofline": {"bound": "tensor", "achieved": gemm_flop / (act_ms / 1e3) / 1e12,
                         "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": gemm_flop / (act_ms / 1e3) / 1e12 / peaks["bf16_tflops"], "traffic": None,
                         "kernel": "policy act (observation packing + layer-1 k_gemm + head), layer-1 FLOP",
                         "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"},
            "clocks": ck}
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(args, sim, inp, dev, g_r, g_d, out, g_a, g_s0, p):
    """End to end through the public API: every step copies its actions and
    initial state in from pinned host memory and its rewards and action
    gradients out.  Copies run on a second stream, double-buffered, so step
    k + 1's inputs arrive and step k - 1's results leave while step k
    computes (events order each buffer's reuse)."""
    import torch
    T, NM = p["horizon"], sim.NM
    act_h = torch.as_tensor(inp["actions"], dtype=torch.float32).pin_memory()
    s0_h = torch.as_tensor(inp["s0"], dtype=torch.float32).pin_memory()
    r_h = [torch.empty(T, NM, dtype=torch.float32).pin_memory() for _ in range(2)]
    ga_h = [torch.empty(T, NM, sim.A, dtype=torch.float32).pin_memory() for _ in range(2)]
    act_d = [torch.empty_like(act_h, device=dev) for _ in range(2)]
    s0_d = [torch.empty_like(s0_h, device=dev) for _ in range(2)]
    outs = [out, {k: (None if v is None else torch.empty_like(v)) for k, v in out.items()}]
    gas = [g_a, torch.empty_like(g_a)]
    comp = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    h2d_done = [ev(), ev()]    # inputs of buffer b are on the device
    comp_done = [ev(), ev()]   # step using buffer b finished (inputs free, outputs ready)
    d2h_done = [ev(), ev()]    # outputs of buffer b are on the host

    def h2d(b):
        with torch.cuda.stream(copy):
            copy.wait_event(comp_done[b])      # the previous step on b has read its inputs
            act_d[b].copy_(act_h, non_blocking=True)
            s0_d[b].copy_(s0_h, non_blocking=True)
            h2d_done[b].record(copy)

    def compute(b):
        comp.wait_event(h2d_done[b])
        comp.wait_event(d2h_done[b])           # its output buffers have been read out
        sim.reset(s0_d[b])
        sim.rollout(act_d[b], out=outs[b])
        sim.backward(g_r, g_d, None, None, gas[b], g_s0)
        comp_done[b].record(comp)

    def d2h(b):
        with torch.cuda.stream(copy):
            copy.wait_event(comp_done[b])
            r_h[b].copy_(outs[b]["r_ctrl"], non_blocking=True)
            ga_h[b].copy_(gas[b], non_blocking=True)
            d2h_done[b].record(copy)

    def run(n):
        for b in range(2):
            comp_done[b].record(comp)
            d2h_done[b].record(comp)
        h2d(0)
        for k in range(n):
            b = k % 2
            if k + 1 < n:
                h2d(1 - b)
            compute(b)
            d2h(b)
        comp.wait_event(d2h_done[(n - 1) % 2])

    run(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    run(args.steps)
    e1.record(comp)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d_b = act_h.numel() * 4 + s0_h.numel() * 4
    d2h_b = r_h[0].numel() * 4 + ga_h[0].numel() * 4
    return {"value": p["n_env"] * T * args.steps / (ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
            "what": "pinned host actions + initial state in; rewards + action gradients out, on a copy "
                    "stream double-buffered against the compute",
            "device_resident": "the depth images written by the rollout (%.1f GB per step) and the reward "
                               "and depth cotangents read by the adjoint (%.1f GB per step) stay on the device, "
                               "as for a policy that consumes depth on the GPU; they are not copied"
                               % (4e-9 * T * NM * sim.Rc, 4e-9 * T * NM * (sim.Rc + 1))}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        if args.workload == SURROGATE_WORKLOAD:
            return run_surrogate(args, rank, world)
        if args.workload == CLOSED_LOOP_WORKLOAD:
            return run_closed_loop(args, rank, world)
        return run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
