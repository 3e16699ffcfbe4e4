"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs and compare what is unique.

Tolerances (written here, used by every test):
  STATE_TF   teacher-forced one-step state: |x_gpu - x_oracle| <= 1e-5 max(|x|, 1)
  DEPTH_TOL  depth / LiDAR per ray, unambiguous rays: 1e-4 m (teacher-forced)
  DEPTH_DRIFT  the same on a full rollout, where FP32 state drift enters: 2e-3 m
  GRAD_RTOL  gradients: per env |g - g*| / |g*| <= 1e-3, and elementwise
             |g - g*| <= 1e-3 max|g*| (floor).  Strict for the teacher-forced
             step adjoint.  For a full-horizon BPTT gradient the bar applies
             to environments whose FP64 gradient is itself stable to FP32-level
             perturbations of the inputs (spread <= GRAD_RTOL / 4); the others
             must agree within COND_FACTOR times their measured spread.
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
PERTURB = 3e-7  # relative input perturbation of the conditioning probe (FP32 scale)
DRIFT = 1e-4
MAX_AMB_FRAC = 2e-2
# oracle ray flags: bit 0 value decision, bit 1 gradient decision, bit 2 FP32
# value conditioning, bit 3 gradient conditioning under drift
VALUE_FLAGS = 1 | 4


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


def masked_cotangents(p, rec, seed=1):
    """N(0,1) cotangents with the entries of ambiguous rays / steps zeroed."""
    cot = synth.cotangents(p, seed=seed)
    g_r = cot["g_r"] * ((rec["amb_step"] & 6) == 0)
    g_d = cot.get("g_depth")
    if g_d is not None:
        g_d = g_d * (rec["amb_cam"] == 0)
    g_l = cot.get("g_lidar")
    if g_l is not None:
        g_l = g_l * (rec["amb_lid"] == 0)
    return g_r, g_d, g_l


def grad_spread(orc, p, inp, rec, g_r, g_d=None, g_l=None, g_sT=None, n=2, seed=0, g_imu=None, s0=None):
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
    """Per-env norm-wise and elementwise gradient comparison.  With `spread`
    (grad_spread), ill-conditioned envs get COND_FACTOR x their spread and are
    left out of the elementwise check; returns (worst rel, n ill-conditioned)."""
    N, M = p["n_env"], p["n_agent"]
    gg = g_gpu.reshape(g_gpu.shape[0], N, -1) if g_gpu.ndim == 3 else g_gpu.reshape(N, -1)[None]
    go = g_orc.reshape(gg.shape)
    scale = np.abs(go).max()
    norms = [np.linalg.norm(go[:, e]) for e in range(N)]
    floor = max(1e-3 * max(norms), 1e-4)
    worst = 0.0
    ill = np.zeros(N, bool)
    if spread is not None:
        ill = spread > GRAD_RTOL / 4
    for e in range(N):
        if bad_env[e] or not np.isfinite(spread[e] if spread is not None else 0.0):
            continue
        a, b = gg[:, e], go[:, e]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)
        tol = max(GRAD_RTOL, COND_FACTOR * spread[e]) if ill[e] else GRAD_RTOL
        if not ill[e]:
            worst = max(worst, rel)
        if rel > tol:
            diff = np.abs(a - b)
            top = np.argsort(diff.reshape(-1))[::-1][:5]
            idx = [np.unravel_index(i, diff.shape) for i in top]
            raise AssertionError("%s env %d rel %.3g |g*| %.3g top diffs %s" % (
                what, e, rel, np.linalg.norm(b),
                [(tuple(int(x) for x in ix), float(a[ix]), float(b[ix])) for ix in idx]))
    keep = ~bad_env & ~ill
    el = np.abs(gg - go)[:, keep]
    if el.size:
        assert (el <= GRAD_RTOL * max(scale, 1e-4)).all(), (what, el.max() / max(scale, 1e-4))
    return worst, int(ill[~bad_env].sum())
