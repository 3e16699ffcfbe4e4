"""ctypes binding of the surrogate MLP (include/surrogate.h) and the host
loops around it: transition collection with the simulator's own rigid step,
minibatch training, rollouts.

Argument marshalling only: the network's forward and backward passes, Adam,
the statistics and the rollout run in libdiffsim.so's tensor-core kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import synth
from .binding import SimConfig, SimError, Simulator, _ck, _ptr, _stream, lib, make_config

_i, _f, _vp = C.c_int32, C.c_float, C.c_void_p

NPARAM, NSTATS = 73741, 107

# every symbol include/surrogate.h declares
SYMBOLS = ["surr_create", "surr_destroy", "surr_set_params", "surr_get_params", "surr_set_stats",
           "surr_get_stats", "surr_fit_stats", "surr_forward", "surr_train_step", "surr_rollout",
           "surr_last_status"]

STATS_LAYOUT = (("mu_x", 17), ("rs_x", 17), ("lo_x", 17), ("hi_x", 17), ("mu_d", 13), ("sd_d", 13),
                ("rs_d", 13))


class SurrConfig(C.Structure):
    _fields_ = [("batch", _i), ("splits", _i), ("lr", _f), ("beta1", _f), ("beta2", _f), ("eps", _f),
                ("margin", _f), ("reserved", _i * 5)]


def _lib():
    L = lib()
    if not getattr(L, "_surr_typed", False):
        for n in SYMBOLS:
            getattr(L, n).restype = C.c_int
        L.surr_create.argtypes = [C.POINTER(SurrConfig), C.POINTER(SimConfig), C.POINTER(_vp)]
        L.surr_fit_stats.argtypes = [_vp, _vp, _vp, C.c_int64, _vp]
        L.surr_forward.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L._surr_typed = True
    return L


def stats_dict(v):
    out, o = {}, 0
    for k, n in STATS_LAYOUT:
        out[k] = np.asarray(v[o:o + n], dtype=np.float64)
        o += n
    return out


def stats_vector(d):
    return np.concatenate([np.asarray(d[k], np.float32).reshape(n) for k, n in STATS_LAYOUT]).astype(np.float32)


class Surrogate:
    """One surrogate handle.  `p`: a rigid-body workload (its dynamics
    parameters define the plain step of the trained-range fallback)."""

    def __init__(self, p, batch=8192, splits=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, margin=0.1,
                 device="cuda"):
        self.device = torch.device(device)
        self.cfg = SurrConfig(batch=batch, splits=splits, lr=lr, beta1=beta1, beta2=beta2, eps=eps, margin=margin)
        self.phys = make_config(p)
        self.batch = batch
        self.h = _vp()
        with torch.cuda.device(self.device):
            _ck(_lib().surr_create(C.byref(self.cfg), C.byref(self.phys), C.byref(self.h)), "surr_create")

    def close(self):
        if getattr(self, "h", None):
            _lib().surr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- parameters
    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == NPARAM
        _ck(_lib().surr_set_params(self.h, _vp(a.ctypes.data)), "surr_set_params")

    def get_params(self):
        a = np.empty(NPARAM, np.float32)
        _ck(_lib().surr_get_params(self.h, _vp(a.ctypes.data)), "surr_get_params")
        return a

    def set_stats(self, st):
        a = stats_vector(st) if isinstance(st, dict) else np.ascontiguousarray(st, dtype=np.float32)
        _ck(_lib().surr_set_stats(self.h, _vp(a.ctypes.data)), "surr_set_stats")

    def get_stats(self):
        a = np.empty(NSTATS, np.float32)
        _ck(_lib().surr_get_stats(self.h, _vp(a.ctypes.data)), "surr_get_stats")
        return stats_dict(a)

    # ---------------------------------------------------------- compute
    def fit_stats(self, X, S1, stream=None):
        _ck(_lib().surr_fit_stats(self.h, _ptr(X), _ptr(S1), X.shape[0], _stream(stream)), "surr_fit_stats")

    def forward(self, X, out=None, stream=None):
        Y = torch.empty(X.shape[0], 13, device=self.device) if out is None else out
        _ck(_lib().surr_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream(stream)), "surr_forward")
        return Y

    def train_step(self, X, S1, idx, apply=True, loss=None, grads=None, stream=None):
        """One Adam step on rows idx (int32 device tensor of length batch).
        Returns (loss, grads) device tensors (grads None unless given)."""
        assert idx.dtype == torch.int32 and idx.numel() == self.batch
        _ck(_lib().surr_train_step(self.h, _ptr(X), _ptr(S1), _ptr(idx), _ptr(loss), _ptr(grads),
                                   _i(1 if apply else 0), _stream(stream)), "surr_train_step")
        return loss, grads

    def rollout(self, s0, actions, states=True, fallback=True, stream=None):
        T, N = actions.shape[0], actions.shape[1]
        o = dict(states=torch.empty(T + 1, N, 13, device=self.device) if states else None,
                 sT=torch.empty(N, 13, device=self.device),
                 fallback=torch.empty(T, N, dtype=torch.uint8, device=self.device) if fallback else None)
        _ck(_lib().surr_rollout(self.h, _ptr(s0), _ptr(actions), _i(N), _i(T), _ptr(o["states"]), _ptr(o["sT"]),
                                _ptr(o["fallback"]), _stream(stream)), "surr_rollout")
        return o

    def status(self):
        st = C.c_int32()
        rc = _lib().surr_last_status(self.h, C.byref(st))
        if rc not in (0, -6, -7):
            _ck(rc, "surr_last_status")
        return st.value


def collect_transitions(p, n_env, steps, seed=0, device="cuda"):
    """Transitions of the simulator's rigid step under random actions from
    random rest states: X [n_env * steps, 17] (state, action) and S1
    [n_env * steps, 13] (next state), device tensors, step-major."""
    dev = torch.device(device)
    q = dict(p, n_env=n_env, horizon=1, cam=None, lidar=None, map_counts=[(0, 0)], n_maps=1, terminate=0)
    inp = synth.make_inputs(q, seed=seed, actions=False)
    sim = Simulator(q, inp, device=dev)
    acts = synth.surrogate_actions(n_env, steps, seed=seed + 1)
    X = torch.empty(steps, n_env, 17, device=dev)
    S1 = torch.empty(steps, n_env, 13, device=dev)
    s = torch.as_tensor(inp["s0"], dtype=torch.float32, device=dev)
    sim.reset(s)
    for t in range(steps):
        a = torch.as_tensor(acts[t], device=dev)
        X[t, :, :13] = s
        X[t, :, 13:] = a
        sim.step(a)
        s = sim.get_state()
        S1[t] = s
    sim.close()
    return X.reshape(-1, 17), S1.reshape(-1, 13)


def train(sur, X, S1, epochs=1, seed=0, log_every=0):
    """Minibatch Adam over the transition set for `epochs` passes; returns
    the per-epoch mean minibatch loss (read once per epoch)."""
    n = X.shape[0]
    B = sur.batch
    nb = n // B
    loss = torch.zeros(nb, device=sur.device)
    out = []
    for ep in range(epochs):
        order = torch.as_tensor(synth.minibatch_order(n, seed, ep), device=sur.device)
        for b in range(nb):
            sur.train_step(X, S1, order[b * B:(b + 1) * B], apply=True, loss=loss[b:b + 1])
        out.append(float(loss.mean()))
    return out
