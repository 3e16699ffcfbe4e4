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
    L = sum_t <g_r[t], r_ctrl[t]> (reported; the gradient is driven by the
    reward cotangent g_r alone) and dL/d(policy parameters) by
    backpropagation through time (Eq. 5): going back, each step's
    observation is rebuilt and the policy's forward re-run (both
    deterministic), then the simulator's step adjoint (sim_step_backward)
    gives the action cotangent, the policy's backward pass the parameter
    gradient and the observation cotangent, whose depth / LiDAR part feeds
    the previous step's adjoint and whose state part joins the state
    cotangent.  The last step's observation feeds no action, so its adjoint
    has no ray term.

    Memory: with ckpt_every = K > 0 (the workload's, 16 for the closed-loop
    configuration) the forward pass keeps only a checkpoint (state and reset
    counters) every K steps; the backward pass replays each segment of K
    steps from its checkpoint, recording its states, actions and every ray's
    hit primitive (2 bytes per ray), and runs the segment's adjoint from
    them: observations rebuilt from the hits (sim_render_hits, bit for bit)
    and the step adjoints gathering them.  With K = 0 every state is kept
    and the hits of all T steps too when they fit in free device memory
    (store_hits forces either way; without them each observation is
    re-rendered).  Both give the same gradient bit for bit.  Rigid-body
    agents, one per environment."""

    def __init__(self, p, inp, device="cuda", **ex):
        assert p["model"] == "rigid" and p["n_agent"] == 1
        self.p = p
        self.device = torch.device(device)
        self.sim = Simulator(p, inp, device=self.device, **ex)
        self.pol = Policy.for_workload(p, device=self.device)
        self.targets = torch.as_tensor(inp["targets"], dtype=torch.float32, device=self.device)
        self.stored_hits = False

    def hits_bytes(self, T=None):
        T = self.p["horizon"] if T is None else T
        return 2 * T * self.p["n_env"] * (self.sim.Rc + self.sim.Rl)

    def _tape(self, n):
        N, Rc, Rl, dev = self.p["n_env"], self.sim.Rc, self.sim.Rl, self.device
        tape = (torch.empty(n, N, Rc, dtype=torch.int16, device=dev) if Rc else None,
                torch.empty(n, N, Rl, dtype=torch.int16, device=dev) if Rl else None)
        return lambda t: tuple(None if x is None else x[t] for x in tape)

    def gradient(self, s0, g_r, T=None, store_hits=None, ckpt_every=None):
        T = self.p["horizon"] if T is None else T
        K = self.p.get("ckpt_every", 16) if ckpt_every is None else ckpt_every
        if 0 < K < T:
            return self._gradient_segments(s0, g_r, T, K)
        return self._gradient_stored(s0, g_r, T, store_hits)

    def _backward_step(self, t, state, action, done, g_s, g_r_t, g_obs, hits_next, hits_t, scratch, render_hits):
        """Adjoint of step t and of the policy's action at state t; returns
        (state cotangent at t, observation cotangent of state t)."""
        sim, pol, dev = self.sim, self.pol, self.device
        N, Rc, Rl = self.p["n_env"], sim.Rc, sim.Rl
        g_dep, g_lid = g_obs
        g_a, g_st = sim.step_backward(state, action, done, g_s, g_r_t, g_dep, g_lid, hits=hits_next)
        sim.set_state(state)
        if render_hits:
            depth, lidar = sim.render_from_hits(hits_t)
        else:
            depth, lidar = sim.render(hits=hits_t)
        pol.act(state, self.targets, depth, lidar, out=scratch)
        g_dep = torch.empty(N, Rc, device=dev) if Rc else None
        g_lid = torch.empty(N, Rl, device=dev) if Rl else None
        pol.backward(g_a, g_st, g_dep, g_lid)
        return g_st, (g_dep, g_lid)

    def _gradient_stored(self, s0, g_r, T, store_hits):
        sim, pol, dev = self.sim, self.pol, self.device
        N = self.p["n_env"]
        Rc, Rl = sim.Rc, sim.Rl
        if not (Rc or Rl):
            store_hits = False
        elif store_hits is None:
            store_hits = self.hits_bytes(T) + (24 << 30) < torch.cuda.mem_get_info(dev)[0]
        self.stored_hits = store_hits
        hits_of = self._tape(T) if store_hits else None
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
        g_obs, hits = (None, None), None
        hit_buf = sim.hit_buffers() if (Rc or Rl) and not store_hits else None
        scratch = torch.empty(N, 4, device=dev)
        pol.grads(reset=True)
        for t in range(T - 1, -1, -1):
            h_t = hits_of(t) if store_hits else hit_buf
            g_s, g_obs = self._backward_step(t, states[t], actions[t], done[t], g_s, g_r[t], g_obs, hits, h_t,
                                             scratch, store_hits)
            hits = h_t
        return loss, pol.grads(reset=True), dict(states=states, actions=actions, done=done, r_ctrl=r)

    def _gradient_segments(self, s0, g_r, T, K):
        sim, pol, dev = self.sim, self.pol, self.device
        N = self.p["n_env"]
        nseg = (T + K - 1) // K
        self.stored_hits = False
        ck_s = torch.empty(nseg, N, 13, device=dev)
        ck_k = torch.empty(nseg, N, dtype=torch.int32, device=dev)
        r = torch.empty(T, N, device=dev)
        done_all = torch.empty(T, N, dtype=torch.uint8, device=dev)
        act = torch.empty(N, 4, device=dev)
        sim.reset(s0)
        state = s0.contiguous()
        depth, lidar = sim.render()
        for t in range(T):
            if t % K == 0:
                ck_s[t // K] = state
                ck_k[t // K] = sim.get_reset_counters()
            pol.act(state, self.targets, depth, lidar, out=act)
            o = sim.step(act)
            r[t], done_all[t] = o["r_ctrl"], o["done"]
            depth, lidar = o["depth"], o["lidar"]
            state = sim.get_state()
        loss = float((g_r[:T] * r).sum())
        # the backward pass, segment by segment, from the last
        states = torch.empty(K + 1, N, 13, device=dev)
        actions = torch.empty(K, N, 4, device=dev)
        done = torch.empty(K, N, dtype=torch.uint8, device=dev)
        hits_of = self._tape(K + 1) if (sim.Rc or sim.Rl) else (lambda i: (None, None))
        g_s = torch.zeros(N, 13, device=dev)
        g_obs = (None, None)
        scratch = torch.empty(N, 4, device=dev)
        pol.grads(reset=True)
        for seg in range(nseg - 1, -1, -1):
            t0 = seg * K
            n = min(T, t0 + K) - t0
            sim.set_state(ck_s[seg])
            sim.set_reset_counters(ck_k[seg])
            states[0] = ck_s[seg]
            depth, lidar = sim.render(hits=hits_of(0))
            for i in range(n):
                pol.act(states[i], self.targets, depth, lidar, out=actions[i])
                o = sim.step(actions[i], hits=hits_of(i + 1))
                done[i] = o["done"]
                depth, lidar = o["depth"], o["lidar"]
                states[i + 1] = sim.get_state()
            for i in range(n - 1, -1, -1):
                t = t0 + i
                hits_next = hits_of(i + 1) if g_obs[0] is not None or g_obs[1] is not None else None
                g_s, g_obs = self._backward_step(t, states[i], actions[i], done[i], g_s, g_r[t], g_obs, hits_next,
                                                 hits_of(i), scratch, True)
        return loss, pol.grads(reset=True), dict(r_ctrl=r, done=done_all, checkpoints=ck_s)
