"""ctypes binding of libdiffsim.so (include/diffsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  torch supplies device memory (tensors) and streams.  The module-level
functions carry the C names; ``Simulator`` is a thin owner of one handle.
If the library is missing, loading raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdiffsim.so")

_i, _f = C.c_int32, C.c_float
_vp = C.c_void_p

SIM_OK = 0
SIM_MODEL_POINT_MASS, SIM_MODEL_RIGID, SIM_MODEL_POINT_MASS_DISCRETE, SIM_MODEL_SIMPLE = 0, 1, 2, 3
MODELS = {"pm": SIM_MODEL_POINT_MASS, "rigid": SIM_MODEL_RIGID, "pm_disc": SIM_MODEL_POINT_MASS_DISCRETE,
          "simple": SIM_MODEL_SIMPLE}
ERRORS = {0: "SIM_OK", -1: "SIM_ERR_INVALID_ARG", -2: "SIM_ERR_NULL_PTR", -3: "SIM_ERR_SIZE",
          -4: "SIM_ERR_CUDA", -5: "SIM_ERR_NOT_READY", -6: "SIM_ERR_NAN", -7: "SIM_ERR_TIMEOUT",
          -8: "SIM_ERR_OOM", -9: "SIM_ERR_UNSUPPORTED"}

# every symbol include/diffsim.h declares
SYMBOLS = ["sim_version", "sim_strerror", "sim_state_dim", "sim_action_dim", "sim_create",
           "sim_destroy", "sim_workspace_bytes", "sim_set_scene", "sim_set_pool",
           "sim_set_env_params", "sim_reset", "sim_get_state", "sim_set_state", "sim_render",
           "sim_step", "sim_rollout", "sim_backward", "sim_step_backward", "sim_last_status",
           "sim_launch_info", "sim_counters", "sim_set_counting", "sim_step_static", "sim_profile", "sim_kernel_times",
           "sim_graph_create", "sim_graph_launch", "sim_graph_kernels", "sim_graph_destroy",
           "sim_set_scene_ex", "sim_get_gate_index", "sim_set_gate_index", "sim_rollout_ex",
           "sim_step_ex", "sim_backward_ex", "sim_render_taped", "sim_step_backward_taped", "sim_render_hits",
           "sim_fp32_issue_rate", "sim_set_wait_limit", "sim_get_reset_counters", "sim_set_reset_counters"]

# flight tasks (Sec. III-C)
TASKS = {"reach": 0, "racing": 1}

KERNEL_KINDS = ("physics", "render", "render_vjp", "physics_bwd")


class SimError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, ERRORS.get(code, "?"), code))


class SimConfig(C.Structure):
    _fields_ = [
        ("model", _i), ("n_env", _i), ("n_agent", _i), ("horizon", _i),
        ("dt", _f), ("gravity", _f),
        ("lam", _f), ("drag", _f), ("act_scale", _f), ("ema_alpha", _f),
        ("mass", _f), ("inertia", _f * 3), ("k_rate", _f * 3), ("drag_body", _f * 3),
        ("rate_scale", _f * 3),
        ("cam_w", _i), ("cam_h", _i), ("cam_hfov", _f), ("cam_range", _f),
        ("lid_ch", _i), ("lid_az", _i), ("lid_elev_lo", _f), ("lid_elev_hi", _f), ("lid_range", _f),
        ("pos_sq", _i), ("w_pos", _f), ("w_obs", _f), ("d_safe", _f), ("w_act", _f),
        ("w_agent", _f), ("d_agent", _f), ("success_radius", _f), ("r_quad", _f),
        ("bound_lo", _f * 3), ("bound_hi", _f * 3),
        ("terminate", _i), ("pool_size", _i),
        ("ckpt_every", _i), ("tape_hits", _i), ("cull", _i), ("warps_per_cta", _i),
        ("rays_per_thread", _i), ("ctas_per_sm", _i),
        ("task", _i), ("imu_noise", _f * 2), ("imu_walk", _f * 2), ("cast_mode", _i),
    ]


class SimScene(C.Structure):
    _fields_ = [("n_maps", _i), ("spheres", _vp), ("sph_off", _vp), ("boxes", _vp), ("box_off", _vp),
                ("cylinders", _vp), ("cyl_off", _vp), ("gates", _vp), ("gate_off", _vp),
                ("env_map", _vp), ("targets", _vp)]


class SimRolloutIO(C.Structure):
    _fields_ = [("actions", _vp), ("r_ctrl", _vp), ("r_goal", _vp), ("done", _vp), ("depth", _vp),
                ("lidar", _vp), ("imu", _vp), ("imu_noise", _vp), ("hits_cam", _vp), ("hits_lidar", _vp)]


class SimGradIO(C.Structure):
    _fields_ = [("g_r", _vp), ("g_depth", _vp), ("g_lidar", _vp), ("g_sT", _vp), ("g_imu", _vp),
                ("g_a", _vp), ("g_s0", _vp)]


class SimGraphIO(C.Structure):
    _fields_ = [("state0", _vp), ("actions", _vp), ("r_ctrl", _vp), ("r_goal", _vp), ("done", _vp),
                ("depth", _vp), ("lidar", _vp), ("g_r", _vp), ("g_depth", _vp), ("g_lidar", _vp),
                ("g_sT", _vp), ("g_a", _vp), ("g_s0", _vp)]


_lib = None


def lib():
    """Load libdiffsim.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdiffsim.so not found at %s: build it with "
                               "`python -m paper_2509_10247_b300.build`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        L.sim_version.restype = C.c_char_p
        L.sim_strerror.restype = C.c_char_p
        L.sim_strerror.argtypes = [C.c_int]
        for name in SYMBOLS[2:]:
            getattr(L, name).restype = C.c_int
        L.sim_create.argtypes = [C.POINTER(SimConfig), C.POINTER(_vp)]
        _lib = L
    return _lib


def _ck(rc, what):
    if rc != SIM_OK:
        raise SimError(rc, what)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return _vp(t.data_ptr())


def _host(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _np_ptr(a):
    return None if a is None else _vp(a.ctypes.data)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def make_config(p, **ex):
    """sim_config from a workload parameter dict; `ex` sets the execution
    fields (ckpt_every, tape_hits, cull, warps_per_cta, rays_per_thread,
    ctas_per_sm)."""
    c = SimConfig()
    c.model = MODELS[p["model"]]
    c.n_env, c.n_agent, c.horizon = p["n_env"], p["n_agent"], p["horizon"]
    c.dt, c.gravity = p["dt"], p["gravity"]
    c.lam, c.drag, c.act_scale, c.ema_alpha = p["lam"], p["drag"], p["act_scale"], p["ema_alpha"]
    c.mass = p["mass"]
    for k in range(3):
        c.inertia[k], c.k_rate[k] = p["inertia"][k], p["k_rate"][k]
        c.drag_body[k], c.rate_scale[k] = p["drag_body"][k], p["rate_scale"][k]
        c.bound_lo[k], c.bound_hi[k] = p["bound_lo"][k], p["bound_hi"][k]
    if p["cam"] is not None:
        c.cam_w, c.cam_h = p["cam"][0], p["cam"][1]
        c.cam_hfov, c.cam_range = math.radians(p["cam"][2]), p["cam"][3]
    if p["lidar"] is not None:
        c.lid_ch, c.lid_az = p["lidar"][0], p["lidar"][1]
        c.lid_elev_lo, c.lid_elev_hi = math.radians(p["lidar"][2]), math.radians(p["lidar"][3])
        c.lid_range = p["lidar"][4]
    c.pos_sq = int(p["pos_sq"])
    c.w_pos, c.w_obs, c.d_safe, c.w_act = p["w_pos"], p["w_obs"], p["d_safe"], p["w_act"]
    c.w_agent, c.d_agent = p["w_agent"], p["d_agent"]
    c.success_radius, c.r_quad = p["success_radius"], p["r_quad"]
    c.terminate, c.pool_size = int(p["terminate"]), p["pool_size"]
    c.ckpt_every = ex.get("ckpt_every", p.get("ckpt_every", 16))
    c.tape_hits = ex.get("tape_hits", -1)
    c.cull = ex.get("cull", -1)
    c.warps_per_cta = ex.get("warps_per_cta", 0)
    c.rays_per_thread = ex.get("rays_per_thread", 0)
    c.ctas_per_sm = ex.get("ctas_per_sm", 0)
    c.cast_mode = ex.get("cast_mode", 0)
    c.task = TASKS[p.get("task", "reach")]
    for k in range(2):
        c.imu_noise[k] = p.get("imu_noise", (0.0, 0.0))[k]
        c.imu_walk[k] = p.get("imu_walk", (0.0, 0.0))[k]
    return c


# ------------------------------------------------------------ C-named calls
def sim_version():
    return lib().sim_version().decode()


def sim_strerror(code):
    return lib().sim_strerror(code).decode()


def sim_state_dim(model):
    return lib().sim_state_dim(model)


def sim_action_dim(model):
    return lib().sim_action_dim(model)


def sim_create(cfg):
    h = _vp()
    _ck(lib().sim_create(C.byref(cfg), C.byref(h)), "sim_create")
    return h


def sim_destroy(h):
    _ck(lib().sim_destroy(h), "sim_destroy")


def sim_workspace_bytes(h):
    n = C.c_size_t()
    _ck(lib().sim_workspace_bytes(h, C.byref(n)), "sim_workspace_bytes")
    return n.value


def sim_set_scene(h, spheres, sph_off, boxes, box_off, env_map, targets):
    sp = _host(spheres, np.float32).reshape(-1, 4)
    bx = _host(boxes, np.float32).reshape(-1, 6)
    so, bo = _host(sph_off, np.int32), _host(box_off, np.int32)
    em, tg = _host(env_map, np.int32), _host(targets, np.float32)
    _ck(lib().sim_set_scene(h, _np_ptr(sp), _np_ptr(so), _np_ptr(bx), _np_ptr(bo),
                            _i(len(so) - 1), _np_ptr(em), _np_ptr(tg)), "sim_set_scene")


def sim_set_scene_ex(h, spheres, sph_off, boxes, box_off, env_map, targets, cylinders=None, cyl_off=None,
                     gates=None, gate_off=None):
    keep = dict(sp=_host(spheres, np.float32).reshape(-1, 4), so=_host(sph_off, np.int32),
                bx=_host(boxes, np.float32).reshape(-1, 6), bo=_host(box_off, np.int32),
                em=_host(env_map, np.int32), tg=_host(targets, np.float32))
    if cylinders is not None:
        keep.update(cy=_host(cylinders, np.float32).reshape(-1, 5), co=_host(cyl_off, np.int32))
    if gates is not None:
        keep.update(gt=_host(gates, np.float32).reshape(-1, 7), go=_host(gate_off, np.int32))
    g = lambda k: _np_ptr(keep.get(k))
    sc = SimScene(len(keep["so"]) - 1, g("sp"), g("so"), g("bx"), g("bo"), g("cy"), g("co"), g("gt"),
                  g("go"), g("em"), g("tg"))
    _ck(lib().sim_set_scene_ex(h, C.byref(sc)), "sim_set_scene_ex")


def sim_get_gate_index(h, gate_k, stream=None):
    _ck(lib().sim_get_gate_index(h, _ptr(gate_k), _stream(stream)), "sim_get_gate_index")


def sim_set_gate_index(h, gate_k, stream=None):
    _ck(lib().sim_set_gate_index(h, _ptr(gate_k), _stream(stream)), "sim_set_gate_index")


def _rollout_io(actions, r_ctrl, r_goal, done, depth, lidar, imu, imu_noise, hits_cam=None, hits_lidar=None):
    return SimRolloutIO(*[None if t is None else _ptr(t).value
                          for t in (actions, r_ctrl, r_goal, done, depth, lidar, imu, imu_noise, hits_cam,
                                    hits_lidar)])


def sim_rollout_ex(h, actions, r_ctrl=None, r_goal=None, done=None, depth=None, lidar=None, imu=None,
                   imu_noise=None, stream=None):
    io = _rollout_io(actions, r_ctrl, r_goal, done, depth, lidar, imu, imu_noise)
    _ck(lib().sim_rollout_ex(h, C.byref(io), _stream(stream)), "sim_rollout_ex")


def sim_step_ex(h, actions, r_ctrl=None, r_goal=None, done=None, depth=None, lidar=None, imu=None,
                imu_noise=None, hits_cam=None, hits_lidar=None, stream=None):
    io = _rollout_io(actions, r_ctrl, r_goal, done, depth, lidar, imu, imu_noise, hits_cam, hits_lidar)
    _ck(lib().sim_step_ex(h, C.byref(io), _stream(stream)), "sim_step_ex")


def sim_backward_ex(h, g_r, g_a, g_depth=None, g_lidar=None, g_sT=None, g_imu=None, g_s0=None, stream=None):
    io = SimGradIO(*[None if t is None else _ptr(t).value for t in (g_r, g_depth, g_lidar, g_sT, g_imu, g_a, g_s0)])
    _ck(lib().sim_backward_ex(h, C.byref(io), _stream(stream)), "sim_backward_ex")


def sim_set_pool(h, pool):
    pl = _host(pool, np.float32)
    _ck(lib().sim_set_pool(h, _np_ptr(pl)), "sim_set_pool")


def sim_set_env_params(h, drag=None, lam=None):
    d = None if drag is None else _host(drag, np.float32)
    l = None if lam is None else _host(lam, np.float32)
    _ck(lib().sim_set_env_params(h, _np_ptr(d), _np_ptr(l)), "sim_set_env_params")


def sim_reset(h, state0=None, stream=None):
    _ck(lib().sim_reset(h, _ptr(state0), _stream(stream)), "sim_reset")


def sim_get_state(h, dst, stream=None):
    _ck(lib().sim_get_state(h, _ptr(dst), _stream(stream)), "sim_get_state")


def sim_set_state(h, src, stream=None):
    _ck(lib().sim_set_state(h, _ptr(src), _stream(stream)), "sim_set_state")


def sim_get_reset_counters(h, dst, stream=None):
    _ck(lib().sim_get_reset_counters(h, _ptr(dst), _stream(stream)), "sim_get_reset_counters")


def sim_set_reset_counters(h, src, stream=None):
    _ck(lib().sim_set_reset_counters(h, _ptr(src), _stream(stream)), "sim_set_reset_counters")


def sim_render(h, depth=None, lidar=None, stream=None):
    _ck(lib().sim_render(h, _ptr(depth), _ptr(lidar), _stream(stream)), "sim_render")


def sim_render_hits(h, hits_cam, hits_lidar, depth, lidar, stream=None):
    _ck(lib().sim_render_hits(h, _ptr(hits_cam), _ptr(hits_lidar), _ptr(depth), _ptr(lidar), _stream(stream)),
        "sim_render_hits")


def sim_render_taped(h, depth, lidar, hits_cam, hits_lidar, stream=None):
    _ck(lib().sim_render_taped(h, _ptr(depth), _ptr(lidar), _ptr(hits_cam), _ptr(hits_lidar), _stream(stream)),
        "sim_render_taped")


def sim_step(h, actions, depth=None, lidar=None, r_ctrl=None, r_goal=None, done=None, stream=None):
    _ck(lib().sim_step(h, _ptr(actions), _ptr(depth), _ptr(lidar), _ptr(r_ctrl), _ptr(r_goal),
                       _ptr(done), _stream(stream)), "sim_step")


def sim_rollout(h, actions, r_ctrl=None, r_goal=None, done=None, depth=None, lidar=None, stream=None):
    _ck(lib().sim_rollout(h, _ptr(actions), _ptr(r_ctrl), _ptr(r_goal), _ptr(done), _ptr(depth),
                          _ptr(lidar), _stream(stream)), "sim_rollout")


def sim_backward(h, g_r, g_depth, g_lidar, g_sT, g_a, g_s0=None, stream=None):
    _ck(lib().sim_backward(h, _ptr(g_r), _ptr(g_depth), _ptr(g_lidar), _ptr(g_sT), _ptr(g_a),
                           _ptr(g_s0), _stream(stream)), "sim_backward")


def sim_step_backward(h, s_t, a_t, done_t, g_s_next, g_r, g_depth, g_lidar, g_a, g_s=None, stream=None):
    _ck(lib().sim_step_backward(h, _ptr(s_t), _ptr(a_t), _ptr(done_t), _ptr(g_s_next), _ptr(g_r),
                                _ptr(g_depth), _ptr(g_lidar), _ptr(g_a), _ptr(g_s),
                                _stream(stream)), "sim_step_backward")


def sim_step_backward_taped(h, s_t, a_t, done_t, g_s_next, g_r, g_depth, g_lidar, hits_cam, hits_lidar, g_a,
                            g_s=None, stream=None):
    _ck(lib().sim_step_backward_taped(h, _ptr(s_t), _ptr(a_t), _ptr(done_t), _ptr(g_s_next), _ptr(g_r),
                                      _ptr(g_depth), _ptr(g_lidar), _ptr(hits_cam), _ptr(hits_lidar), _ptr(g_a),
                                      _ptr(g_s), _stream(stream)), "sim_step_backward_taped")


def sim_last_status(h):
    st = C.c_int32()
    rc = lib().sim_last_status(h, C.byref(st), None)
    if rc not in (SIM_OK, -6, -7):
        _ck(rc, "sim_last_status")
    return st.value


def sim_set_wait_limit(h, polls):
    _ck(lib().sim_set_wait_limit(h, _i(polls)), "sim_set_wait_limit")


def sim_set_counting(h, on=True):
    _ck(lib().sim_set_counting(h, _i(1 if on else 0)), "sim_set_counting")


def sim_counters(h, reset=True):
    v = (C.c_uint64 * 4)()
    _ck(lib().sim_counters(h, v, _i(1 if reset else 0)), "sim_counters")
    return dict(sphere_tests=v[0], box_tests=v[1], rays=v[2], env_steps=v[3])


def sim_launch_info(h):
    w, r, g, s = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _ck(lib().sim_launch_info(h, C.byref(w), C.byref(r), C.byref(g), C.byref(s)), "sim_launch_info")
    return dict(warps_per_cta=w.value, rays_per_thread=r.value, grid=g.value, smem_bytes=s.value)


def sim_step_static(cfg, prims, map_off, map_ns, map_nb, ns_max, nb_max, env_map, targets, pool,
                    state, actions, depth=None, lidar=None, r_ctrl=None, r_goal=None, done=None,
                    pool_k=None, status=None, stream=None):
    """One step without any device allocation by the library (all buffers are
    the caller's device tensors; status: an int32 device tensor of one
    element that receives the call's SIM_STATUS_* bits; see include/diffsim.h)."""
    _ck(lib().sim_step_static(C.byref(cfg), _ptr(prims), _ptr(map_off), _ptr(map_ns), _ptr(map_nb),
                              _i(ns_max), _i(nb_max), _ptr(env_map), _ptr(targets), _ptr(pool),
                              _ptr(state), _ptr(actions), _ptr(depth), _ptr(lidar), _ptr(r_ctrl),
                              _ptr(r_goal), _ptr(done), _ptr(pool_k), _ptr(status), _stream(stream)),
        "sim_step_static")


def sim_fp32_issue_rate(device=None, stream=None):
    """Measured FMAs per second of this GPU: (scalar, packed pairs)."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    n = torch.cuda.get_device_properties(dev).multi_processor_count * 2048
    scratch = torch.empty(n, dtype=torch.float32, device=dev)
    a, b = C.c_double(), C.c_double()
    with torch.cuda.device(dev):
        _ck(lib().sim_fp32_issue_rate(_ptr(scratch), C.c_int64(n), C.byref(a), C.byref(b), _stream(stream)),
            "sim_fp32_issue_rate")
    return a.value, b.value


def sim_profile(h, on=True):
    _ck(lib().sim_profile(h, _i(1 if on else 0)), "sim_profile")


def sim_kernel_times(h, reset=True):
    """Per kernel kind: summed device milliseconds of the profiled launches
    and the number of launches since the last reset."""
    ms = (C.c_double * len(KERNEL_KINDS))()
    n = (C.c_int64 * len(KERNEL_KINDS))()
    _ck(lib().sim_kernel_times(h, ms, n, _i(1 if reset else 0)), "sim_kernel_times")
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}


def sim_graph_create(h, io):
    g = _vp()
    _ck(lib().sim_graph_create(h, C.byref(io), C.byref(g)), "sim_graph_create")
    return g


def sim_graph_launch(g, stream=None):
    _ck(lib().sim_graph_launch(g, _stream(stream)), "sim_graph_launch")


def sim_graph_kernels(g):
    n = C.c_int32()
    _ck(lib().sim_graph_kernels(g, C.byref(n)), "sim_graph_kernels")
    return n.value


def sim_graph_destroy(g):
    _ck(lib().sim_graph_destroy(g), "sim_graph_destroy")


class SimGraph:
    """Owner of one captured reset + rollout (+ adjoint).  Keeps the tensors
    whose pointers the graph holds alive."""

    def __init__(self, h, tensors):
        self.tensors = tensors
        io = SimGraphIO(**{k: (None if v is None else v.data_ptr()) for k, v in tensors.items()})
        for k, v in tensors.items():
            if v is not None:
                assert v.is_cuda and v.is_contiguous(), k
        self.g = sim_graph_create(h, io)
        self.kernels = sim_graph_kernels(self.g)

    def launch(self, stream=None):
        sim_graph_launch(self.g, stream)

    def close(self):
        if getattr(self, "g", None):
            sim_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ owner class
class Simulator:
    """One handle bound to a workload: parameters `p` (synth.preset/params) and
    inputs `inp` (synth.make_inputs).  Device tensors are float32 on `device`."""

    def __init__(self, p, inp, device="cuda", **ex):
        self.p = p
        self.device = torch.device(device)
        self.N, self.M, self.T = p["n_env"], p["n_agent"], p["horizon"]
        self.NM = self.N * self.M
        self.D, self.A = synth.STATE_DIM[p["model"]], synth.ACTION_DIM[p["model"]]
        self.Rc = p["cam"][0] * p["cam"][1] if p["cam"] is not None else 0
        self.Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] is not None else 0
        self.cfg = make_config(p, **ex)
        with torch.cuda.device(self.device):
            self.h = sim_create(self.cfg)
            if inp.get("cylinders") is not None or inp.get("gates") is not None:
                sim_set_scene_ex(self.h, inp["spheres"], inp["sph_off"], inp["boxes"], inp["box_off"],
                                 inp["env_map"], inp["targets"], inp.get("cylinders"), inp.get("cyl_off"),
                                 inp.get("gates"), inp.get("gate_off"))
            else:
                sim_set_scene(self.h, inp["spheres"], inp["sph_off"], inp["boxes"], inp["box_off"],
                              inp["env_map"], inp["targets"])
            if p["pool_size"] > 0:
                sim_set_pool(self.h, inp["pool"])
            if inp.get("drag_env") is not None or inp.get("lam_env") is not None:
                sim_set_env_params(self.h, inp.get("drag_env"), inp.get("lam_env"))

    def close(self):
        if getattr(self, "h", None):
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape, dtype=torch.float32):
        return torch.empty(*shape, dtype=dtype, device=self.device)

    def reset(self, s0=None):
        sim_reset(self.h, None if s0 is None else s0.contiguous())

    def get_state(self):
        out = self._empty(self.NM, self.D)
        sim_get_state(self.h, out)
        return out

    def set_state(self, s):
        sim_set_state(self.h, s.contiguous())

    def get_reset_counters(self):
        out = self._empty(self.N, dtype=torch.int32)
        sim_get_reset_counters(self.h, out)
        return out

    def set_reset_counters(self, k):
        sim_set_reset_counters(self.h, k.to(device=self.device, dtype=torch.int32).contiguous())

    def render(self, hits=None):
        """Depth and LiDAR of the current state.  hits: None, or a pair of
        int16 tensors ([NM][Rc], [NM][Rl]; None where a sensor is absent),
        e.g. from hit_buffers(), that receive each ray's hit primitive id
        for step_backward(hits=...) of the step that produced this state."""
        depth = self._empty(self.NM, self.Rc) if self.Rc else None
        lidar = self._empty(self.NM, self.Rl) if self.Rl else None
        if hits is None:
            sim_render(self.h, depth, lidar)
        else:
            sim_render_taped(self.h, depth, lidar, hits[0], hits[1])
        return depth, lidar

    def hit_buffers(self):
        return (self._empty(self.NM, self.Rc, dtype=torch.int16) if self.Rc else None,
                self._empty(self.NM, self.Rl, dtype=torch.int16) if self.Rl else None)

    def step(self, actions, hits=None):
        """One step; hits: None or a pair from hit_buffers() that receives
        the rendered state's per-ray hit ids (as render(hits=...))."""
        o = dict(r_ctrl=self._empty(self.NM), r_goal=self._empty(self.NM, dtype=torch.int8),
                 done=self._empty(self.NM, dtype=torch.uint8),
                 depth=self._empty(self.NM, self.Rc) if self.Rc else None,
                 lidar=self._empty(self.NM, self.Rl) if self.Rl else None)
        if hits is None:
            sim_step(self.h, actions.contiguous(), o["depth"], o["lidar"], o["r_ctrl"], o["r_goal"], o["done"])
        else:
            sim_step_ex(self.h, actions.contiguous(), o["r_ctrl"], o["r_goal"], o["done"], o["depth"], o["lidar"],
                        hits_cam=hits[0], hits_lidar=hits[1])
        return o

    def render_from_hits(self, hits):
        """Depth and LiDAR of the current state from the hit ids recorded for
        it (render(hits=...) or step(hits=...)): equal to render() bit for
        bit, without casting."""
        depth = self._empty(self.NM, self.Rc) if self.Rc else None
        lidar = self._empty(self.NM, self.Rl) if self.Rl else None
        sim_render_hits(self.h, hits[0], hits[1], depth, lidar)
        return depth, lidar

    def rollout(self, actions, depth=True, lidar=True, out=None, imu=False, imu_noise=None):
        T, NM = self.T, self.NM
        o = out if out is not None else dict(
            r_ctrl=self._empty(T, NM), r_goal=self._empty(T, NM, dtype=torch.int8),
            done=self._empty(T, NM, dtype=torch.uint8),
            depth=self._empty(T, NM, self.Rc) if (self.Rc and depth) else None,
            lidar=self._empty(T, NM, self.Rl) if (self.Rl and lidar) else None)
        self._actions = actions.contiguous()
        if imu or imu_noise is not None:
            o["imu"] = self._empty(T, NM, 6)
            sim_rollout_ex(self.h, self._actions, o["r_ctrl"], o["r_goal"], o["done"], o["depth"], o["lidar"],
                           o["imu"], None if imu_noise is None else imu_noise.contiguous())
        else:
            sim_rollout(self.h, self._actions, o["r_ctrl"], o["r_goal"], o["done"], o["depth"], o["lidar"])
        return o

    def gate_index(self):
        out = self._empty(self.NM, dtype=torch.int32)
        sim_get_gate_index(self.h, out)
        return out

    def set_gate_index(self, k):
        sim_set_gate_index(self.h, k.to(device=self.device, dtype=torch.int32).contiguous())

    def backward(self, g_r, g_depth=None, g_lidar=None, g_sT=None, g_a=None, g_s0=None, g_imu=None):
        T, NM = self.T, self.NM
        g_a = self._empty(T, NM, self.A) if g_a is None else g_a
        g_s0 = self._empty(NM, self.D) if g_s0 is None else g_s0
        if g_imu is not None:
            c = lambda t: None if t is None else t.contiguous()
            sim_backward_ex(self.h, g_r.contiguous(), g_a, c(g_depth), c(g_lidar), c(g_sT), g_imu.contiguous(), g_s0)
            return g_a, g_s0
        sim_backward(self.h, g_r.contiguous(), None if g_depth is None else g_depth.contiguous(),
                     None if g_lidar is None else g_lidar.contiguous(),
                     None if g_sT is None else g_sT.contiguous(), g_a, g_s0)
        return g_a, g_s0

    def step_backward(self, s_t, a_t, done_t, g_s_next, g_r, g_depth=None, g_lidar=None, hits=None):
        """VJP of one step.  hits: the pair render(hits=...) wrote for the
        state this step produces; the ray adjoint then gathers them instead
        of casting the rays again (same result, bit for bit)."""
        g_a = self._empty(self.NM, self.A)
        g_s = self._empty(self.NM, self.D)
        c = lambda x: None if x is None else x.contiguous()
        if hits is None:
            sim_step_backward(self.h, c(s_t), c(a_t), c(done_t), c(g_s_next), c(g_r), c(g_depth),
                              c(g_lidar), g_a, g_s)
        else:
            sim_step_backward_taped(self.h, c(s_t), c(a_t), c(done_t), c(g_s_next), c(g_r), c(g_depth),
                                    c(g_lidar), hits[0], hits[1], g_a, g_s)
        return g_a, g_s

    def status(self):
        return sim_last_status(self.h)

    def launch_info(self):
        return sim_launch_info(self.h)

    def set_wait_limit(self, polls):
        sim_set_wait_limit(self.h, polls)

    def counters(self, reset=True):
        return sim_counters(self.h, reset)

    def set_counting(self, on=True):
        """Whether the forward kernels count their work (default on)."""
        sim_set_counting(self.h, on)

    def workspace_bytes(self):
        return sim_workspace_bytes(self.h)

    def profile(self, on=True):
        sim_profile(self.h, on)

    def kernel_times(self, reset=True):
        return sim_kernel_times(self.h, reset)

    def graph(self, actions, s0=None, out=None, g_r=None, g_depth=None, g_lidar=None, g_sT=None,
              g_a=None, g_s0=None):
        """Capture reset(s0) + rollout(actions) (+ backward when g_r is given)
        into one CUDA graph writing `out` (dict as returned by rollout) and
        g_a / g_s0.  Returns a SimGraph; launching it runs the whole pass."""
        T, NM = self.T, self.NM
        o = out if out is not None else dict(
            r_ctrl=self._empty(T, NM), r_goal=self._empty(T, NM, dtype=torch.int8),
            done=self._empty(T, NM, dtype=torch.uint8),
            depth=self._empty(T, NM, self.Rc) if self.Rc else None,
            lidar=self._empty(T, NM, self.Rl) if self.Rl else None)
        if g_r is not None:
            g_a = self._empty(T, NM, self.A) if g_a is None else g_a
            g_s0 = self._empty(NM, self.D) if g_s0 is None else g_s0
        tensors = dict(state0=s0, actions=actions, r_ctrl=o["r_ctrl"], r_goal=o["r_goal"], done=o["done"],
                       depth=o["depth"], lidar=o["lidar"], g_r=g_r, g_depth=g_depth, g_lidar=g_lidar,
                       g_sT=g_sT, g_a=g_a, g_s0=g_s0)
        g = SimGraph(self.h, tensors)
        g.out = o
        return g
