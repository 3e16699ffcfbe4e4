"""FP64 oracle of the closed-loop policy gradient (test infrastructure: only
the tests, the smoke check and the CPU baseline load it; it shares no code
with the CUDA path).

A two-layer policy MLP (Sec. IV, the MLP backbone of the paper's learners)
maps each rigid-body agent's observation to its action at every step:

    obs    = (p - p*, q, v, omega, p  [16],  depth / cam_range [Rc],
              lidar / lidar_range [Rl])                       F = 16 + Rc + Rl
    x      = bf16(obs)
    h      = bf16(silu(W1 x + b1))                            256
    a      = tanh(W2 h + b2)                                  4 actions in (-1, 1)

with W1, W2 rounded to bf16, sums in FP64 here (fp32 on the GPU).  The
closed loop renders s_t, acts, steps the simulator (Eq. 1 with the sensors
of Sec. III-B), and the gradient of L = sum_t <g_r[t], r_ctrl[t]> with
respect to (W1, b1, W2, b2) is taken by backpropagation through time
(Eq. 5): at each step the simulator's adjoint gives the action cotangent,
the policy's backward pass turns it into parameter gradients and an
observation cotangent, whose depth / LiDAR part is the cotangent of the
previous step's rendered output and whose state part joins the state
cotangent.  The backward pass rounds the hidden-layer cotangent dZ1 to bf16
where the kernels do (it is an operand of both backward matrix products).
`rounding=False` is the plain FP64 network.
"""
from __future__ import annotations

import numpy as np

from .surrogate import bf16_round, dsilu, silu

N_STATE_FEAT, N_HID, N_ACT = 16, 256, 4


def n_features(p):
    Rc = p["cam"][0] * p["cam"][1] if p["cam"] is not None else 0
    Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] is not None else 0
    return N_STATE_FEAT + Rc + Rl


def shapes(p):
    F = n_features(p)
    return (("W1", (N_HID, F)), ("b1", (N_HID,)), ("W2", (N_ACT, N_HID)), ("b2", (N_ACT,)))


def split(p, flat):
    out, o = {}, 0
    flat = np.asarray(flat, np.float64)
    for k, s in shapes(p):
        n = int(np.prod(s))
        out[k] = flat[o:o + n].reshape(s)
        o += n
    return out


def features(p, s, targets, depth, lidar):
    """Observation rows [n, F] of rigid states s [n, 13] (FP64)."""
    s = np.asarray(s, np.float64)
    parts = [s[:, 0:3] - np.asarray(targets, np.float64), s[:, 3:7], s[:, 7:10], s[:, 10:13], s[:, 0:3]]
    if p["cam"] is not None:
        parts.append(np.asarray(depth, np.float64) / p["cam"][3])
    if p["lidar"] is not None:
        parts.append(np.asarray(lidar, np.float64) / p["lidar"][4])
    return np.concatenate(parts, axis=1)


def forward(P, obs, rounding=True):
    q = bf16_round if rounding else (lambda v: np.asarray(v, np.float64))
    x = q(obs)
    W1, W2 = q(P["W1"]), q(P["W2"])
    z1 = x @ W1.T + P["b1"]
    h = q(silu(z1))
    u = h @ W2.T + P["b2"]
    return dict(x=x, z1=z1, h=h, u=u, y=np.tanh(u), W1=W1, W2=W2)


def backward(P, f, g_y, rounding=True):
    """Parameter gradients and the observation cotangent for action
    cotangents g_y [n, 4] at the forward record f."""
    q = bf16_round if rounding else (lambda v: np.asarray(v, np.float64))
    g_u = np.asarray(g_y, np.float64) * (1.0 - f["y"] ** 2)
    g = {"W2": g_u.T @ f["h"], "b2": g_u.sum(axis=0)}
    dh = g_u @ f["W2"]
    dz1 = dh * dsilu(f["z1"])
    dz1b = q(dz1)
    g["W1"] = dz1b.T @ f["x"]
    g["b1"] = dz1.sum(axis=0)
    g_obs = dz1b @ f["W1"]
    return g, g_obs


def state_feature_vjp(g_f):
    """Cotangent of the state from the cotangent of its 16 observation features."""
    g = np.zeros((g_f.shape[0], 13))
    g[:, 0:3] = g_f[:, 0:3] + g_f[:, 13:16]
    g[:, 3:13] = g_f[:, 3:13]
    return g


def closed_loop(orc, P, s0, g_r, rounding=True, T=None):
    """Closed-loop rollout of the policy P over orc's horizon (or T steps)
    from s0 and the gradient of L = sum_t <g_r[t], r_ctrl[t]>.  orc is an
    oracle.Oracle of a rigid workload (no agent coupling, M = 1).  Returns
    (L, grads, record) with record the per-step states, actions, rewards."""
    p = orc.p
    T = orc.T if T is None else T
    one = orc.with_horizon(1)
    tg = orc._keep["targets"]
    Rc, Rl = orc.Rc, orc.Rl
    dep, lid = orc.render(s0)[:2]
    s = np.asarray(s0, np.float64)
    pk = np.zeros(orc.N, np.int32)
    recs, fs, L = [], [], 0.0
    for t in range(T):
        f = forward(P, features(p, s, tg, dep, lid), rounding)
        rec = one.rollout(s, f["y"][None], pool_k=pk)
        pk = rec["pool_k"]
        L += float(np.sum(np.asarray(g_r[t], np.float64) * rec["r_ctrl"][0]))
        recs.append(rec)
        fs.append(f)
        s = rec["states"][1]
        dep, lid = rec["depth"][0], rec["lidar"][0]
    grads = {k: np.zeros(sh) for k, sh in shapes(p)}
    g_s = np.zeros_like(s)
    g_dep = np.zeros((orc.NM, Rc))
    g_lid = np.zeros((orc.NM, Rl))
    for t in range(T - 1, -1, -1):
        g_a, g_st = one.backward(recs[t], np.asarray(g_r[t], np.float64)[None], g_dep[None], g_lid[None], g_s)
        g, g_obs = backward(P, fs[t], g_a[0], rounding)
        for k in grads:
            grads[k] += g[k]
        g_s = g_st + state_feature_vjp(g_obs[:, :N_STATE_FEAT])
        o = N_STATE_FEAT
        if Rc:
            g_dep = g_obs[:, o:o + Rc] / p["cam"][3]
            o += Rc
        if Rl:
            g_lid = g_obs[:, o:o + Rl] / p["lidar"][4]
    record = dict(states=np.stack([r["states"][0] for r in recs] + [s]),
                  actions=np.stack([f["y"] for f in fs]), r_ctrl=np.stack([r["r_ctrl"][0] for r in recs]),
                  done=np.stack([r["done"][0] for r in recs]),
                  amb=np.stack([(r["amb_cam"][0] != 0).sum() + (r["amb_lid"][0] != 0).sum() for r in recs]))
    return L, grads, record
