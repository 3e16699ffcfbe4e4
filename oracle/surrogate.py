"""FP64 oracle of the learned surrogate of the rigid-body step (test
infrastructure: only the tests, the smoke check and the CPU baseline load
it; it shares no code with the CUDA path).

The surrogate replaces one explicit step of the rigid quadrotor (Eq. 1) by a
residual MLP, the kind of learned dynamics model the paper's world-model
learners (Sec. IV, DreamerV3-style) fit to simulator transitions:

    x      = (s [13], clip(a, -1, 1) [4])                       17 inputs
    xh     = bf16((x - mu_x) * rs_x)      (FP32 subtract and multiply)
    h1     = bf16(silu(W1 xh + b1))       256
    h2     = bf16(silu(W2 h1 + b2))       256
    y      = W3 h2 + b3                   13, the normalised residual
    s'     = s + (sd_d * y + mu_d),  quaternion renormalised

with weights rounded to bf16 (round to nearest, ties to even), sums and
biases in FP64 here (FP32 on the GPU).  silu(z) = z / (1 + exp(-z)).
Training minimises the mean of (y - t)^2 over the batch and the 13 outputs,
t = ((s' - s) - mu_d) * rs_d (FP32), with Adam.

`rounding=False` switches every bf16 rounding off: the plain FP64 network,
used to pin the backward pass against finite differences.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 17, 256, 13


# --------------------------------------------------------------- bf16
def bf16_round(x):
    """Round to the nearest bfloat16 value (8 exponent bits, 8 significant
    bits), ties to even, from the IEEE 754 definition: the representable
    values around |x| = m 2^e (1 <= m < 2) are spaced 2^(e-7); below the
    smallest normal 2^-126 the spacing stays 2^-133; beyond the largest finite
    value (2 - 2^-7) 2^127 rounding gives infinity.  Works on float64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.array(x, copy=True)
    fin = np.isfinite(x) & (x != 0)
    xf = x[fin]
    _, E = np.frexp(xf)  # xf = f 2^E with 0.5 <= |f| < 1, so e = E - 1
    e = np.maximum(E - 1, -126)
    q = np.ldexp(xf, 7 - e)  # exact: a power-of-two scaling
    r = np.rint(q)  # round half to even
    v = np.ldexp(r, e - 7)
    big = np.abs(v) > np.ldexp(2.0 - 2.0 ** -7, 127)
    v[big] = np.copysign(np.inf, v[big])
    out[fin] = v
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


# --------------------------------------------------------------- model
def normalise_inputs(s, a, mu_x, rs_x):
    """xh in FP32 (subtract then multiply, no fused multiply-add), exactly as
    the kernel forms it; returns float32 [n, 17]."""
    x = np.concatenate([np.asarray(s, np.float32), np.clip(np.asarray(a, np.float32), -1, 1)], axis=1)
    return ((x - np.asarray(mu_x, np.float32)) * np.asarray(rs_x, np.float32)).astype(np.float32)


def targets(s, s1, mu_d, rs_d):
    """Normalised residual targets in FP32: ((s1 - s) - mu_d) * rs_d."""
    s, s1 = np.asarray(s, np.float32), np.asarray(s1, np.float32)
    return (((s1 - s) - np.asarray(mu_d, np.float32)) * np.asarray(rs_d, np.float32)).astype(np.float32)


def forward(P, xh, rounding=True):
    """P: dict W1 [256,17], b1, W2 [256,256], b2, W3 [13,256], b3 (the
    master FP32 values).  xh [n, 17] (the normalised FP32 inputs)."""
    q = bf16_round if rounding else (lambda v: np.asarray(v, np.float64))
    x = q(np.asarray(xh, np.float64))
    W1, W2, W3 = q(P["W1"]), q(P["W2"]), q(P["W3"])
    z1 = x @ W1.T + P["b1"]
    h1 = q(silu(z1))
    z2 = h1 @ W2.T + P["b2"]
    h2 = q(silu(z2))
    y = h2 @ W3.T + P["b3"]
    return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, y=y, W1=W1, W2=W2, W3=W3)


def loss_grads(P, xh, t, rounding=True):
    """Mean squared error over the batch and the outputs and its gradient
    with respect to every parameter.  The backward pass rounds the operands
    of its matrix products to bf16 where the kernels do (the output
    cotangent dY, the pre-activation cotangents dZ2 and dZ1); bias gradients
    sum the unrounded cotangents."""
    q = bf16_round if rounding else (lambda v: np.asarray(v, np.float64))
    f = forward(P, xh, rounding)
    n = f["y"].shape[0]
    diff = f["y"] - np.asarray(t, np.float64)
    loss = float(np.mean(diff ** 2))
    dY = 2.0 * diff / (n * N_OUT)
    dYb = q(dY)
    g = {}
    g["W3"] = dYb.T @ f["h2"]
    g["b3"] = dY.sum(axis=0)
    dH2 = dYb @ f["W3"]
    dZ2 = dH2 * dsilu(f["z2"])
    dZ2b = q(dZ2)
    g["W2"] = dZ2b.T @ f["h1"]
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2b @ f["W2"]
    dZ1 = dH1 * dsilu(f["z1"])
    dZ1b = q(dZ1)
    g["W1"] = dZ1b.T @ f["x"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, g, f


ADAM = dict(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)


def adam_step(w, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------- statistics
def column_stats(X, D):
    """Normalisation statistics of a transition set: inputs X [n, 17] (state,
    clipped action) and residuals D [n, 13] (s' - s).  Returns mean, 1/std
    (1 where the standard deviation is below 1e-6), std, min and max, each
    in FP64 (the kernel rounds them to FP32)."""
    X = np.asarray(X, np.float64)
    D = np.asarray(D, np.float64)
    out = {}
    for k, A in (("x", X), ("d", D)):
        mu = A.mean(axis=0)
        sd = np.sqrt(np.mean((A - mu) ** 2, axis=0))
        out["mu_" + k] = mu
        out["sd_" + k] = sd
        out["rs_" + k] = np.where(sd < 1e-6, 1.0, 1.0 / np.where(sd < 1e-6, 1.0, sd))
        out["lo_" + k] = A.min(axis=0)
        out["hi_" + k] = A.max(axis=0)
    return out


def in_range(x, lo, hi, margin=0.1):
    """Rows of x whose every feature lies within [lo - m, hi + m], m =
    margin (hi - lo): where the surrogate was trained."""
    x = np.asarray(x, np.float64)
    span = np.asarray(hi, np.float64) - np.asarray(lo, np.float64)
    m = margin * span if margin > 0 else np.zeros_like(span)  # no 0 * inf for unbounded features
    return np.all((x >= lo - m) & (x <= hi + m), axis=1)


# --------------------------------------------------------------- rollout
def step(P, stats, s, a, rounding=True):
    """One surrogate step of states s [n, 13] (FP32 values) under actions a
    [n, 4]; returns s' in FP64 with the quaternion renormalised."""
    xh = normalise_inputs(s, a, stats["mu_x"], stats["rs_x"])
    y = forward(P, xh, rounding)["y"]
    s64 = np.asarray(s, np.float64)
    sp = s64 + (np.asarray(stats["sd_d"], np.float64) * y + np.asarray(stats["mu_d"], np.float64))
    qn = np.sqrt(np.sum(sp[:, 3:7] ** 2, axis=1, keepdims=True))
    sp[:, 3:7] = sp[:, 3:7] / qn
    return sp


def rollout(P, stats, s0, actions, plain_step, rounding=True, margin=0.1):
    """T surrogate steps from s0 [n, 13] under actions [T, n, 4]; an
    environment whose inputs leave the trained range (in_range) takes the
    plain simulator step `plain_step(s, a) -> s'` for that step instead.
    Each step's state is rounded to FP32 before the next, as the kernel
    keeps it.  Returns (states [T+1, n, 13], fallback [T, n] bool)."""
    T = actions.shape[0]
    s = np.asarray(s0, np.float32)
    states = [s.astype(np.float64)]
    fb = np.zeros((T, s.shape[0]), bool)
    for t in range(T):
        a = np.asarray(actions[t], np.float32)
        x = np.concatenate([s, np.clip(a, -1, 1)], axis=1)
        ok = in_range(x, stats["lo_x"], stats["hi_x"], margin)
        sp = step(P, stats, s, a, rounding)
        if (~ok).any():
            sp[~ok] = plain_step(s[~ok].astype(np.float64), a[~ok].astype(np.float64))
        fb[t] = ~ok
        s = sp.astype(np.float32)
        states.append(s.astype(np.float64))
    return np.stack(states), fb
