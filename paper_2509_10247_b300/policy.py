"""ctypes binding of the closed-loop policy (include/policy.h) and the
closed-loop driver: a policy acting on the simulator's rendered
observations, and the gradient of the rollout's reward with respect to the
policy parameters by backpropagation through time.

Argument marshalling and the step loop only: observation packing, the policy
layers, their backward pass, the simulator step and its adjoint all run in
libdiffsim.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from .binding import Simulator, _ck, _ptr, _stream, lib

_vp = C.c_void_p

# every symbol include/policy.h declares
SYMBOLS = ["pol_create", "pol_destroy", "pol_nparams", "pol_set_params", "pol_get_params", "pol_act",
           "pol_backward", "pol_grads", "pol_last_status"]


def _lib():
    L = lib()
    if not getattr(L, "_pol_typed", False):
        for n in SYMBOLS:
            getattr(L, n).restype = C.c_int
        L.pol_create.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_int32, C.c_float, C.POINTER(_vp)]
        L._pol_typed = True
    return L


class Policy:
    """One policy handle for n_env agents observing Rc camera and Rl LiDAR rays."""

    def __init__(self, n_env, cam_rays=0, cam_range=1.0, lidar_rays=0, lidar_range=1.0, device="cuda"):
        self.device = torch.device(device)
        self.N, self.Rc, self.Rl = n_env, cam_rays, lidar_rays
        self.h = _vp()
        with torch.cuda.device(self.device):
            _ck(_lib().pol_create(n_env, cam_rays, cam_range, lidar_rays, lidar_range, C.byref(self.h)),
                "pol_create")
        n = C.c_int64()
        _ck(_lib().pol_nparams(self.h, C.byref(n)), "pol_nparams")
        self.nparams = n.value

    @classmethod
    def for_workload(cls, p, n_env=None, device="cuda"):
        Rc = p["cam"][0] * p["cam"][1] if p["cam"] is not None else 0
        Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] is not None else 0
        return cls(p["n_env"] if n_env is None else n_env, Rc, p["cam"][3] if Rc else 1.0, Rl,
                   p["lidar"][4] if Rl else 1.0, device=device)

    def close(self):
        if getattr(self, "h", None):
            _lib().pol_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        _ck(_lib().pol_set_params(self.h, _vp(a.ctypes.data)), "pol_set_params")

    def get_params(self):
        a = np.empty(self.nparams, np.float32)
        _ck(_lib().pol_get_params(self.h, _vp(a.ctypes.data)), "pol_get_params")
        return a

    def grads(self, reset=True):
        a = np.empty(self.nparams, np.float32)
        _ck(_lib().pol_grads(self.h, _vp(a.ctypes.data), C.c_int32(1 if reset else 0)), "pol_grads")
        return a

    def act(self, state, targets, depth, lidar, out=None, stream=None):
        a = torch.empty(self.N, 4, device=self.device) if out is None else out
        _ck(_lib().pol_act(self.h, _ptr(state), _ptr(targets), _ptr(depth), _ptr(lidar), _ptr(a),
                           _stream(stream)), "pol_act")
        return a

    def backward(self, g_actions, g_state, g_depth=None, g_lidar=None, stream=None):
        _ck(_lib().pol_backward(self.h, _ptr(g_actions), _ptr(g_state), _ptr(g_depth), _ptr(g_lidar),
                                _stream(stream)), "pol_backward")

    def status(self):
        st = C.c_int32()
        rc = _lib().pol_last_status(self.h, C.byref(st))
        if rc not in (0, -7):
            _ck(rc, "pol_last_status")
        return st.value


class ClosedLoop:
    """A policy flying the simulator: at each step the policy maps the
    agents' states and rendered depth / LiDAR to actions, the simulator steps
    and renders the next observation.  gradient() returns the loss
    L = sum_t <g_r[t], r_ctrl[t]> and dL/d(policy parameters) by
    backpropagation through time: states are kept per step; going back, each
    step's observation is re-rendered and the policy's forward re-run (both
    deterministic), then the simulator's step adjoint (sim_step_backward)
    gives the action cotangent, the policy's backward pass the parameter
    gradient and the observation cotangent, whose depth / LiDAR part feeds
    the previous step's adjoint and whose state part joins the state
    cotangent.  The last step's observation feeds no action, so its adjoint
    has no ray term.  Rays are cast once per step: the forward pass records
    every ray's hit primitive (2 bytes per ray and step, kept when it fits in
    free device memory; store_hits forces either way), the backward pass
    rebuilds each observation from its hits (sim_render_hits, bit for bit)
    and the adjoint of step t - 1 gathers the hits of state t.  Without the
    stored hits the backward pass re-renders state t, recording its hits
    for that adjoint.  Rigid-body agents, one per environment."""

    def __init__(self, p, inp, device="cuda", **ex):
        assert p["model"] == "rigid" and p["n_agent"] == 1
        self.p = p
        self.device = torch.device(device)
        self.sim = Simulator(p, inp, device=self.device, **ex)
        self.pol = Policy.for_workload(p, device=self.device)
        self.targets = torch.as_tensor(inp["targets"], dtype=torch.float32, device=self.device)

    def hits_bytes(self, T=None):
        T = self.p["horizon"] if T is None else T
        return 2 * T * self.p["n_env"] * (self.sim.Rc + self.sim.Rl)

    def gradient(self, s0, g_r, T=None, store_hits=None):
        sim, pol, dev = self.sim, self.pol, self.device
        T = self.p["horizon"] if T is None else T
        N = self.p["n_env"]
        Rc, Rl = sim.Rc, sim.Rl
        if not (Rc or Rl):
            store_hits = False
        elif store_hits is None:
            store_hits = self.hits_bytes(T) + (24 << 30) < torch.cuda.mem_get_info(dev)[0]
        self.stored_hits = store_hits
        if store_hits:
            tape = (torch.empty(T, N, Rc, dtype=torch.int16, device=dev) if Rc else None,
                    torch.empty(T, N, Rl, dtype=torch.int16, device=dev) if Rl else None)
            hits_of = lambda t: tuple(None if x is None else x[t] for x in tape)
        states = torch.empty(T + 1, N, 13, device=dev)
        actions = torch.empty(T, N, 4, device=dev)
        done = torch.empty(T, N, dtype=torch.uint8, device=dev)
        r = torch.empty(T, N, device=dev)
        states[0] = s0
        sim.reset(states[0])
        depth, lidar = sim.render(hits=hits_of(0) if store_hits else None)
        for t in range(T):
            pol.act(states[t], self.targets, depth, lidar, out=actions[t])
            o = sim.step(actions[t], hits=hits_of(t + 1) if store_hits and t + 1 < T else None)
            r[t], done[t] = o["r_ctrl"], o["done"]
            depth, lidar = o["depth"], o["lidar"]
            states[t + 1] = sim.get_state()
        loss = float((g_r[:T] * r).sum())
        g_s = torch.zeros(N, 13, device=dev)
        g_dep = g_lid = hits = None
        hit_buf = sim.hit_buffers() if (Rc or Rl) and not store_hits else None
        scratch = torch.empty(N, 4, device=dev)
        pol.grads(reset=True)
        for t in range(T - 1, -1, -1):
            g_a, g_st = sim.step_backward(states[t], actions[t], done[t], g_s, g_r[t], g_dep, g_lid, hits=hits)
            sim.set_state(states[t])
            if store_hits:
                hits = hits_of(t)
                depth, lidar = sim.render_from_hits(hits)
            else:
                depth, lidar = sim.render(hits=hit_buf)
                hits = hit_buf
            pol.act(states[t], self.targets, depth, lidar, out=scratch)
            g_dep = torch.empty(N, Rc, device=dev) if Rc else None
            g_lid = torch.empty(N, Rl, device=dev) if Rl else None
            pol.backward(g_a, g_st, g_dep, g_lid)
            g_s = g_st
        return loss, pol.grads(reset=True), dict(states=states, actions=actions, done=done, r_ctrl=r)
