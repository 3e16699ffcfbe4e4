"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs and compare what is unique.

Tolerances (written here, used by every test):
  STATE_TF   teacher-forced one-step state: |x_gpu - x_oracle| <= 1e-5 max(|x|, 1)
  DEPTH_TOL  depth / LiDAR per ray, unambiguous rays: 1e-4 m (teacher-forced)
  DEPTH_DRIFT  the same on a full rollout, where FP32 state drift enters: 2e-3 m
  GRAD_RTOL  gradients: per env |g - g*| / |g*| <= 1e-3, and elementwise
             |g - g*| <= 1e-3 max|g*| (floor).  Unconditional (every
             environment) for the trajectory-teacher-forced adjoint chain
             (teacher_forced_chain: the step adjoint chained over the whole
             horizon on the oracle's own trajectory, rounded to FP32).  For a
             free-running BPTT gradient, where FP32 state drift enters, the bar
             applies to environments whose FP64 gradient is itself stable to
             FP32-level perturbations of the inputs (spread <= GRAD_RTOL / 4,
             N_PERTURB probes); the others must agree within COND_FACTOR times
             their measured spread, capped at GRAD_COND_CAP, and at most
             MAX_ILL_FRAC of the environments may take that widened bar.
  MAX_MASK_FRAC  largest fraction of ray cotangents that the oracle's
             ambiguity flags may zero (reported by masked_cotangents).
  DRIFT      full-rollout (non teacher-forced) state drift bound: 1e-4 max(|x|, 1)
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2509_10247_b300 import synth
from paper_2509_10247_b300.binding import Simulator

STATE_TF = 1e-5
DEPTH_TOL = 1e-4
DEPTH_DRIFT = 2e-3
GRAD_RTOL = 1e-3
COND_FACTOR = 4.0
GRAD_COND_CAP = 1e-2  # hard ceiling of a conditioning-widened gradient bar
MAX_ILL_FRAC = 0.25   # at most this fraction of environments may be ill-conditioned
N_PERTURB = 4         # perturbations per conditioning probe
MAX_MASK_FRAC = 0.01  # at most this fraction of ray cotangents may be zeroed
PERTURB = 3e-7  # relative input perturbation of the conditioning probe (FP32 scale)
DRIFT = 1e-4
MAX_AMB_FRAC = 2e-2
# oracle ray flags: bit 0 value decision, bit 1 gradient decision, bit 2 FP32
# value conditioning, bit 3 gradient conditioning under drift, bit 4 gradient
# conditioning under FP32 rounding of the pose (no drift)
VALUE_FLAGS = 1 | 4
# flags that zero a cotangent when the linearisation points of both sides
# differ only by FP32 rounding (no drift): every decision / value flag and
# the rounding-conditioning bit 4, not the drift-conditioning bit 3
TF_FLAGS = 1 | 2 | 4 | 16


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")


def host(t):
    return None if t is None else t.detach().cpu().numpy().astype(np.float64)


def subset(p, inp, envs):
    """Sub-workload of the given environments (maps shared)."""
    envs = np.asarray(envs)
    M = p["n_agent"]
    rows = (envs[:, None] * M + np.arange(M)[None, :]).reshape(-1)
    q = dict(p, n_env=len(envs))
    sub = dict(inp)
    sub["s0"] = inp["s0"][rows]
    sub["targets"] = inp["targets"][rows]
    sub["pool"] = inp["pool"][:, rows]
    sub["actions"] = None if inp["actions"] is None else inp["actions"][:, rows]
    sub["env_map"] = inp["env_map"][envs]
    for k in ("drag_env", "lam_env"):
        sub[k] = None if inp.get(k) is None else inp[k][envs]
    return q, sub, rows


class Pair:
    """A workload run through both the CUDA path and the oracle."""

    def __init__(self, p, seed=0, ex=None, inp=None):
        self.p = p
        self.inp = synth.make_inputs(p, seed=seed) if inp is None else inp
        self.ex = ex or {}
        self.orc = oracle.Oracle(p, self.inp)
        self.sim = Simulator(p, self.inp, **self.ex)

    def run_oracle(self):
        self.rec = self.orc.rollout(self.inp["s0"], self.inp["actions"])
        return self.rec

    def run_gpu(self):
        self.sim.reset(dev(self.inp["s0"]))
        self.act = dev(self.inp["actions"])
        self.out = self.sim.rollout(self.act)
        self.sT = self.sim.get_state()
        torch.cuda.synchronize()
        assert self.sim.status() == 0
        return self.out


def env_divergence(p, rec, out):
    """Environments whose discrete trajectory (done flags) differs; only
    allowed where the oracle flags the decision as ambiguous."""
    M = p["n_agent"]
    d_g = out["done"].cpu().numpy().astype(np.uint8)
    d_o = rec["done"]
    bad_env = np.zeros(p["n_env"], bool)
    mism = (d_g != d_o).reshape(d_o.shape[0], p["n_env"], M).any(axis=(0, 2))
    amb = (rec["amb_step"] & 1).reshape(d_o.shape[0], p["n_env"], M).any(axis=(0, 2))
    assert not (mism & ~amb).any(), "done flags differ without an ambiguous decision"
    bad_env |= mism
    return bad_env


def compare_rollout(p, rec, out, sT, check_depth=True):
    """Compare rewards, done, sensors and final state of a full rollout."""
    M = p["n_agent"]
    bad = env_divergence(p, rec, out)
    keep_agents = np.repeat(~bad, M)
    T = rec["r_ctrl"].shape[0]
    rg = out["r_goal"].cpu().numpy()
    amb_goal = (rec["amb_step"] & 1) != 0
    ok = (rg == rec["r_goal"]) | amb_goal | ~keep_agents[None, :]
    assert ok.all(), "r_goal differs at %s" % (np.argwhere(~ok)[:5],)
    if p.get("task", "reach") == "racing":
        # an ambiguous gate pass taken differently changes the targeted gate
        # (and the reward) from then on: such environments are compared no further
        bad |= (rg != rec["r_goal"]).reshape(T, p["n_env"], M).any(axis=(0, 2))
        keep_agents = np.repeat(~bad, M)
    r = host(out["r_ctrl"])
    err = np.abs(r - rec["r_ctrl"])[:, keep_agents]
    assert (err <= DRIFT * np.maximum(1.0, np.abs(rec["r_ctrl"][:, keep_agents]))).all(), err.max()
    s = host(sT)
    so = rec["states"][T]
    e = np.abs(s - so)[keep_agents]
    assert (e <= 10 * DRIFT * np.maximum(1.0, np.abs(so[keep_agents]))).all(), e.max()
    if check_depth:
        for key, amb_key, hit_key, rng in (("depth", "amb_cam", "hit_cam", p["cam"]),
                                            ("lidar", "amb_lid", "hit_lid", p["lidar"])):
            if rng is None or out[key] is None:
                continue
            g = host(out[key])[:, keep_agents]
            o = rec[key][:, keep_agents]
            amb = (rec[amb_key][:, keep_agents] & VALUE_FLAGS) != 0
            assert amb.mean() < MAX_AMB_FRAC, amb.mean()
            d = np.abs(g - o)
            assert (d[~amb] <= DEPTH_DRIFT).all(), (d[~amb].max(), np.argwhere(d * ~amb > DEPTH_DRIFT)[:5])
    return bad


def masked_cotangents(p, rec, seed=1, ray_flags=0xFF, report=None):
    """N(0,1) cotangents with the entries of ambiguous rays / steps zeroed
    (rays: any oracle flag in `ray_flags`).  The fraction of ray cotangents
    zeroed must stay below MAX_MASK_FRAC; it is stored in report["masked"]
    when a dict is given."""
    cot = synth.cotangents(p, seed=seed)
    g_r = cot["g_r"] * ((rec["amb_step"] & 6) == 0)
    n_ray = n_zero = 0
    g_d = cot.get("g_depth")
    if g_d is not None:
        keep = (rec["amb_cam"] & ray_flags) == 0
        g_d = g_d * keep
        n_ray += keep.size
        n_zero += int((~keep).sum())
    g_l = cot.get("g_lidar")
    if g_l is not None:
        keep = (rec["amb_lid"] & ray_flags) == 0
        g_l = g_l * keep
        n_ray += keep.size
        n_zero += int((~keep).sum())
    frac = n_zero / max(n_ray, 1)
    if report is not None:
        report["masked"] = frac
    assert frac <= MAX_MASK_FRAC, "%.3g of the ray cotangents are masked" % frac
    return g_r, g_d, g_l


def teacher_forced_chain(sim, p, rec, actions, rows, g_r, g_d=None, g_l=None, g_sT=None, s_other=None,
                         done_other=None):
    """Eq. 5 chained over the whole horizon on the oracle's own trajectory.

    The GPU's single-step adjoint (sim_step_backward) is called for t = T-1
    .. 0 at the oracle's states s_t (rounded to FP32) and done flags, carrying
    its own cotangent g_s from step to step, so that both sides linearise at
    the same points: what remains is the adjoint's arithmetic, with no FP32
    trajectory drift.  `rows` are the agent rows (of the simulator's batch)
    that rec covers; the other rows (when rows is not the whole batch) take
    s_other[t] / done_other[t] (device tensors, e.g. the GPU's own
    trajectory) and zero cotangents.  Cotangents g_r [T, rows], g_d [T, rows, Rc], g_l, g_sT
    [rows, D] are host arrays.  Returns (g_a [T, rows, A], g_s0 [rows, D])."""
    T, NM, D = rec["r_ctrl"].shape[0], sim.NM, sim.D
    ri = torch.as_tensor(np.asarray(rows), device="cuda")
    full = len(rows) == NM

    def spread(x, shape, dtype=torch.float32):
        out = torch.zeros(shape, dtype=dtype, device="cuda")
        if x is not None:
            out[ri] = dev(x, dtype)
        return out
    g_s = spread(g_sT, (NM, D))
    g_a = torch.zeros(T, len(rows), sim.A, device="cuda")
    assert full or (s_other is not None and done_other is not None)
    for t in reversed(range(T)):
        if full:
            s_t = dev(rec["states"][t])
            d_t = dev(rec["done"][t], torch.uint8)
        else:
            s_t = s_other[t].clone()
            d_t = done_other[t].clone()
            s_t[ri] = dev(rec["states"][t])
            d_t[ri] = dev(rec["done"][t], torch.uint8)
        gr = spread(g_r[t], (NM,))
        gd = spread(None if g_d is None else g_d[t], (NM, sim.Rc)) if sim.Rc else None
        gl = spread(None if g_l is None else g_l[t], (NM, sim.Rl)) if sim.Rl else None
        ga_t, g_s = sim.step_backward(s_t, actions[t], d_t, g_s, gr, gd, gl)
        g_a[t] = ga_t[ri]
    torch.cuda.synchronize()
    return host(g_a), host(g_s[ri])


def compare_grads_strict(p, g_gpu, g_orc, what):
    """Every environment at GRAD_RTOL, norm-wise per environment and
    elementwise against GRAD_RTOL x the largest |g*| (no carve-out).
    Returns the per-environment relative errors."""
    N = p["n_env"]
    gg = g_gpu.reshape(g_gpu.shape[0], N, -1) if g_gpu.ndim == 3 else g_gpu.reshape(N, -1)[None]
    go = g_orc.reshape(gg.shape)
    norms = np.array([np.linalg.norm(go[:, e]) for e in range(N)])
    floor = max(1e-3 * norms.max(), 1e-4)
    rel = np.array([np.linalg.norm(gg[:, e] - go[:, e]) / max(norms[e], floor) for e in range(N)])
    bad = np.nonzero(rel > GRAD_RTOL)[0]
    assert bad.size == 0, "%s: %d of %d environments above %.0e: %s" % (
        what, bad.size, N, GRAD_RTOL, [(int(e), float(rel[e])) for e in bad[:8]])
    scale = max(np.abs(go).max(), 1e-4)
    el = np.abs(gg - go)
    assert (el <= GRAD_RTOL * scale).all(), (what, el.max() / scale)
    return rel


def grad_spread(orc, p, inp, rec, g_r, g_d=None, g_l=None, g_sT=None, n=N_PERTURB, seed=0, g_imu=None, s0=None):
    """Per-env conditioning of the oracle's BPTT gradient: the largest relative
    change of (g_a, g_s0) when the actions and initial state are perturbed at
    FP32 rounding scale (PERTURB).  Envs whose discrete trajectory changes get
    +inf.  Returns (spread_a, spread_s) arrays of length N."""
    N, M = p["n_env"], p["n_agent"]
    s0 = inp["s0"] if s0 is None else s0
    ga, gs = orc.backward(rec, g_r, g_d, g_l, g_sT, g_imu=g_imu)
    rng = np.random.default_rng(seed)
    sa, ss = np.zeros(N), np.zeros(N)
    for _ in range(n):
        a2 = inp["actions"] * (1 + PERTURB * rng.standard_normal(inp["actions"].shape))
        s2 = s0 * (1 + PERTURB * rng.standard_normal(s0.shape))
        r2 = orc.rollout(s2, a2)
        ga2, gs2 = orc.backward(r2, g_r, g_d, g_l, g_sT, g_imu=g_imu)
        for e in range(N):
            sl = slice(e * M, (e + 1) * M)
            if (r2["done"][:, sl] != rec["done"][:, sl]).any():
                sa[e] = ss[e] = np.inf
                continue
            sa[e] = max(sa[e], np.linalg.norm(ga2[:, sl] - ga[:, sl]) / max(np.linalg.norm(ga[:, sl]), 1e-4))
            ss[e] = max(ss[e], np.linalg.norm(gs2[sl] - gs[sl]) / max(np.linalg.norm(gs[sl]), 1e-4))
    return sa, ss


def compare_grads(p, g_gpu, g_orc, bad_env, what, spread=None):
    """Per-env norm-wise and elementwise gradient comparison of a free-running
    BPTT gradient.  Every compared env is held to GRAD_RTOL, except that an
    env whose FP64 gradient is itself ill-conditioned under FP32-level input
    perturbations (`spread` from grad_spread above GRAD_RTOL / 4, or a
    discrete trajectory that changes under the probe) may instead agree
    within COND_FACTOR x its spread, never more than GRAD_COND_CAP; at most
    MAX_ILL_FRAC of the compared envs may take that widened bar, and they
    are left out of the elementwise check.  Returns (worst rel of the envs
    within GRAD_RTOL, number of envs on the widened bar)."""
    N, M = p["n_env"], p["n_agent"]
    gg = g_gpu.reshape(g_gpu.shape[0], N, -1) if g_gpu.ndim == 3 else g_gpu.reshape(N, -1)[None]
    go = g_orc.reshape(gg.shape)
    scale = np.abs(go).max()
    norms = [np.linalg.norm(go[:, e]) for e in range(N)]
    floor = max(1e-3 * max(norms), 1e-4)
    worst = 0.0
    ill = np.zeros(N, bool) if spread is None else spread > GRAD_RTOL / 4
    wide = np.zeros(N, bool)
    for e in range(N):
        if bad_env[e]:
            continue
        a, b = gg[:, e], go[:, e]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)
        if rel <= GRAD_RTOL:
            worst = max(worst, rel)
            continue
        tol = min(max(GRAD_RTOL, COND_FACTOR * spread[e]), GRAD_COND_CAP) if ill[e] else GRAD_RTOL
        wide[e] = True
        if rel > tol:
            diff = np.abs(a - b)
            top = np.argsort(diff.reshape(-1))[::-1][:5]
            idx = [np.unravel_index(i, diff.shape) for i in top]
            raise AssertionError("%s env %d rel %.3g (bar %.3g, spread %.3g) |g*| %.3g top diffs %s" % (
                what, e, rel, tol, spread[e] if spread is not None else 0.0, np.linalg.norm(b),
                [(tuple(int(x) for x in ix), float(a[ix]), float(b[ix])) for ix in idx]))
    n_cmp = int((~bad_env).sum())
    n_wide = int(wide.sum())
    assert n_wide <= max(1, int(MAX_ILL_FRAC * n_cmp)), "%s: %d of %d environments on the widened bar" % (
        what, n_wide, n_cmp)
    keep = ~bad_env & ~wide
    el = np.abs(gg - go)[:, keep]
    if el.size:
        assert (el <= GRAD_RTOL * max(scale, 1e-4)).all(), (what, el.max() / max(scale, 1e-4))
    return worst, n_wide
