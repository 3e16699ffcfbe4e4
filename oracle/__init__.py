"""FP64 CPU oracle of the batched differentiable quadrotor environment step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg import this package.  It is independent of
the CUDA library: it shares no source, header, helper or constant with it, and
neither imports the other.  The arithmetic lives in ``diffsim_oracle.c`` (plain
C, double precision); this module only marshals numpy arrays through ctypes.

Parity status of each oracle function (what pins it, see tests/test_oracle_*):
  dynamics (Eq. 1, Eq. 3)      closed forms: hover, free fall, lag, drag decay,
                               constant body rate, tilted thrust; RK4 limit
  point-mass attitude          orthonormality, heading/thrust alignment cases
  ray casting (Sec. III-B)     closed-form hits, wall z-depth, SDF marching
  collisions and rewards       hand-computed cases
  adjoint (Eq. 5)              central finite differences of ``loss``
  culling work count           brute-force counts of hand-placed cases
                               (tests/test_oracle_cull.py)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diffsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_d = C.c_double
_i = C.c_int32
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int32)
_pu8 = C.POINTER(C.c_uint8)
_pi8 = C.POINTER(C.c_int8)


class OcConfig(C.Structure):
    _fields_ = [
        ("model", _i), ("n_env", _i), ("n_agent", _i), ("horizon", _i),
        ("dt", _d), ("gravity", _d),
        ("lam", _d), ("drag", _d), ("act_scale", _d), ("ema_alpha", _d),
        ("mass", _d), ("inertia", _d * 3), ("k_rate", _d * 3), ("drag_body", _d * 3),
        ("rate_scale", _d * 3),
        ("cam_w", _i), ("cam_h", _i), ("cam_hfov", _d), ("cam_range", _d),
        ("lid_ch", _i), ("lid_az", _i), ("lid_elev_lo", _d), ("lid_elev_hi", _d),
        ("lid_range", _d),
        ("pos_sq", _i), ("w_pos", _d), ("w_obs", _d), ("d_safe", _d), ("w_act", _d),
        ("w_agent", _d), ("d_agent", _d), ("success_radius", _d), ("r_quad", _d),
        ("bound_lo", _d * 3), ("bound_hi", _d * 3),
        ("terminate", _i), ("pool_size", _i),
        ("task", _i), ("imu_noise", _d * 2), ("imu_walk", _d * 2),
    ]


class OcExtra(C.Structure):
    _fields_ = [("gate_k", _pi), ("gate_tape", _pi), ("imu", _pd), ("imu_noise", _pd),
                ("imu_bias", _pd)]


class OcScene(C.Structure):
    _fields_ = [
        ("spheres", _pd), ("sph_off", _pi), ("boxes", _pd), ("box_off", _pi),
        ("cylinders", _pd), ("cyl_off", _pi), ("gates", _pd), ("gate_off", _pi),
        ("env_map", _pi), ("n_maps", _i), ("targets", _pd), ("pool", _pd),
        ("drag_env", _pd), ("lam_env", _pd),
    ]


def build(force=False):
    """Compile the oracle with gcc (plain -O2, OpenMP over environments only,
    no fast-math, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=gnu99",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


# dynamics models: continuous point mass (Eq. 3), rigid body (Eq. 1), discrete
# point mass (Eq. 4), simplified quadrotor (Eq. 2)
MODELS = {"pm": 0, "rigid": 1, "pm_disc": 2, "simple": 3}
# flight tasks (Sec. III-C): reaching / avoidance (targets), racing (gates)
TASKS = {"reach": 0, "racing": 1}
STATE_DIM = {"pm": 12, "rigid": 13, "pm_disc": 12, "simple": 15}
ACTION_DIM = {"pm": 3, "rigid": 4, "pm_disc": 3, "simple": 4}


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.oc_ray_sphere.restype = _d
        L.oc_ray_sphere.argtypes = [_pd, _pd, _pd]
        L.oc_ray_box.restype = _d
        L.oc_ray_box.argtypes = [_pd, _pd, _pd, _pi]
        L.oc_sdf_sphere.restype = _d
        L.oc_sdf_sphere.argtypes = [_pd, _pd]
        L.oc_sdf_box.restype = _d
        L.oc_sdf_box.argtypes = [_pd, _pd]
        L.oc_ray_cylinder.restype = _d
        L.oc_ray_cylinder.argtypes = [_pd, _pd, _pd, _pi]
        L.oc_ray_gate.restype = _d
        L.oc_ray_gate.argtypes = [_pd, _pd, _pd, _pi]
        L.oc_sdf_cylinder.restype = _d
        L.oc_sdf_cylinder.argtypes = [_pd, _pd]
        L.oc_sdf_gate.restype = _d
        L.oc_sdf_gate.argtypes = [_pd, _pd, _pi]
        L.oc_pose.restype = C.c_int
        L.oc_loss.restype = _d
        L.oc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ct=_pd):
    if a is None:
        return C.cast(None, ct)
    return a.ctypes.data_as(ct)


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_config(p):
    """oc_config from a workload parameter dict (angles given in degrees)."""
    c = OcConfig()
    c.model = MODELS[p["model"]]
    c.n_env, c.n_agent, c.horizon = p["n_env"], p["n_agent"], p["horizon"]
    c.dt, c.gravity = p["dt"], p["gravity"]
    c.lam, c.drag, c.act_scale, c.ema_alpha = p["lam"], p["drag"], p["act_scale"], p["ema_alpha"]
    c.mass = p["mass"]
    for k in range(3):
        c.inertia[k] = p["inertia"][k]
        c.k_rate[k] = p["k_rate"][k]
        c.drag_body[k] = p["drag_body"][k]
        c.rate_scale[k] = p["rate_scale"][k]
        c.bound_lo[k] = p["bound_lo"][k]
        c.bound_hi[k] = p["bound_hi"][k]
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
    c.task = TASKS[p.get("task", "reach")]
    for k in range(2):
        c.imu_noise[k] = p.get("imu_noise", (0.0, 0.0))[k]
        c.imu_walk[k] = p.get("imu_walk", (0.0, 0.0))[k]
    return c


class Oracle:
    """Oracle bound to one workload (parameters + scene)."""

    def __init__(self, p, inp):
        self.p = p
        self.cfg = make_config(p)
        self.D = STATE_DIM[p["model"]]
        self.A = ACTION_DIM[p["model"]]
        self.N, self.M, self.T = p["n_env"], p["n_agent"], p["horizon"]
        self.NM = self.N * self.M
        self.Rc = p["cam"][0] * p["cam"][1] if p["cam"] is not None else 0
        self.Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] is not None else 0
        self._keep = dict(
            spheres=_c64(inp["spheres"].reshape(-1, 4)),
            sph_off=np.ascontiguousarray(inp["sph_off"], dtype=np.int32),
            boxes=_c64(inp["boxes"].reshape(-1, 6)),
            box_off=np.ascontiguousarray(inp["box_off"], dtype=np.int32),
            cylinders=_c64(inp["cylinders"].reshape(-1, 5)) if inp.get("cylinders") is not None else None,
            cyl_off=np.ascontiguousarray(inp["cyl_off"], dtype=np.int32) if inp.get("cylinders") is not None else None,
            gates=_c64(inp["gates"].reshape(-1, 7)) if inp.get("gates") is not None else None,
            gate_off=np.ascontiguousarray(inp["gate_off"], dtype=np.int32) if inp.get("gates") is not None else None,
            env_map=np.ascontiguousarray(inp["env_map"], dtype=np.int32),
            targets=_c64(inp["targets"]), pool=_c64(inp["pool"]),
            drag_env=_c64(inp.get("drag_env")), lam_env=_c64(inp.get("lam_env")),
        )
        k = self._keep
        if p.get("task", "reach") == "racing":
            assert k["gates"] is not None and (np.diff(k["gate_off"]) > 0).all(), "racing needs gates"
        self.scene = OcScene(_p(k["spheres"]), _p(k["sph_off"], _pi), _p(k["boxes"]),
                             _p(k["box_off"], _pi), _p(k["cylinders"]), _p(k["cyl_off"], _pi),
                             _p(k["gates"]), _p(k["gate_off"], _pi), _p(k["env_map"], _pi),
                             len(k["sph_off"]) - 1, _p(k["targets"]), _p(k["pool"]),
                             _p(k["drag_env"]), _p(k["lam_env"]))

    def with_horizon(self, T):
        o = Oracle.__new__(Oracle)
        o.__dict__.update(self.__dict__)
        o.cfg = make_config(dict(self.p, horizon=T))
        o.T = T
        return o

    def rollout(self, s0, actions, pool_k=None, n_threads=0, gate_k=None, imu_noise=None,
                imu_bias=None):
        """Run T steps from s0 [NM, D] with actions [T, NM, A].  Returns a dict:
        states [T+1,NM,D], spre [T,NM,D], r_ctrl, r_goal, done [T,NM],
        depth/hit_cam/amb_cam [T,NM,Rc], lidar/hit_lid/amb_lid [T,NM,Rl],
        amb_step, sdf_id [T,NM], pool_k [N] (advanced), imu [T,NM,6],
        gate_tape [T,NM] and gate_k [NM] (racing, advanced from gate_k, default
        0), imu_bias [NM,6] (advanced when imu_noise [T,NM,12] is given)."""
        T, NM, D = self.T, self.NM, self.D
        s0 = _c64(s0).reshape(NM, D)
        act = _c64(actions).reshape(T, NM, self.A)
        pk = np.zeros(self.N, np.int32) if pool_k is None else np.array(pool_k, np.int32)
        gk = np.zeros(NM, np.int32) if gate_k is None else np.array(gate_k, np.int32)
        gt = np.zeros((T, NM), np.int32)
        imu = np.zeros((T, NM, 6))
        nz = None if imu_noise is None else _c64(imu_noise).reshape(T, NM, 12)
        bias = np.zeros((NM, 6)) if imu_bias is None else np.array(imu_bias, np.float64).reshape(NM, 6)
        ex = OcExtra(_p(gk, _pi), _p(gt, _pi), _p(imu), _p(nz), _p(bias))
        out = dict(
            states=np.zeros((T + 1, NM, D)), spre=np.zeros((T, NM, D)),
            r_ctrl=np.zeros((T, NM)), r_goal=np.zeros((T, NM), np.int8),
            done=np.zeros((T, NM), np.uint8),
            depth=np.zeros((T, NM, self.Rc)), lidar=np.zeros((T, NM, self.Rl)),
            hit_cam=np.zeros((T, NM, self.Rc), np.int32), hit_lid=np.zeros((T, NM, self.Rl), np.int32),
            amb_cam=np.zeros((T, NM, self.Rc), np.uint8), amb_lid=np.zeros((T, NM, self.Rl), np.uint8),
            amb_step=np.zeros((T, NM), np.uint8), sdf_id=np.zeros((T, NM), np.int32),
        )
        o = out
        lib().oc_rollout(C.byref(self.cfg), C.byref(self.scene), _p(s0), _p(pk, _pi), _p(act),
                         _p(o["states"]), _p(o["spre"]), _p(o["r_ctrl"]), _p(o["r_goal"], _pi8),
                         _p(o["done"], _pu8), _p(o["depth"]), _p(o["lidar"]),
                         _p(o["hit_cam"], _pi), _p(o["hit_lid"], _pi), _p(o["amb_cam"], _pu8),
                         _p(o["amb_lid"], _pu8), _p(o["amb_step"], _pu8), _p(o["sdf_id"], _pi),
                         C.byref(ex), C.c_int(n_threads))
        out["pool_k"] = pk
        out["actions"] = act
        out.update(gate_k=gk, gate_tape=gt, imu=imu, imu_bias=bias)
        return out

    def backward(self, rec, g_r, g_depth=None, g_lidar=None, g_sT=None, n_threads=0, g_imu=None):
        """Adjoint of a recorded rollout.  Returns (g_a [T,NM,A], g_s0 [NM,D])."""
        T, NM, D, A = self.T, self.NM, self.D, self.A
        g_a = np.zeros((T, NM, A))
        g_s0 = np.zeros((NM, D))
        gr = _c64(g_r).reshape(T, NM)
        gd = None if (g_depth is None or self.Rc == 0) else _c64(g_depth).reshape(T, NM, self.Rc)
        gl = None if (g_lidar is None or self.Rl == 0) else _c64(g_lidar).reshape(T, NM, self.Rl)
        gs = None if g_sT is None else _c64(g_sT).reshape(NM, D)
        gi = None if g_imu is None else _c64(g_imu).reshape(T, NM, 6)
        lib().oc_backward(C.byref(self.cfg), C.byref(self.scene), _p(rec["actions"]),
                          _p(rec["states"]), _p(rec["spre"]), _p(rec["done"], _pu8),
                          _p(rec["hit_cam"], _pi), _p(rec["hit_lid"], _pi), _p(gr), _p(gd),
                          _p(gl), _p(gs), _p(gi), _p(rec["gate_tape"], _pi), _p(g_a), _p(g_s0),
                          C.c_int(n_threads))
        return g_a, g_s0

    def loss(self, s0, actions, g_r, g_depth=None, g_lidar=None, g_sT=None, g_imu=None,
             gate_k=None, imu_noise=None, imu_bias=None):
        """L = <g_r, r_ctrl> + <g_depth, depth> + <g_lidar, lidar> + <g_sT, s_T>
        + <g_imu, imu>."""
        T, NM = self.T, self.NM
        gd = None if (g_depth is None or self.Rc == 0) else _c64(g_depth).reshape(T, NM, self.Rc)
        gl = None if (g_lidar is None or self.Rl == 0) else _c64(g_lidar).reshape(T, NM, self.Rl)
        gs = None if g_sT is None else _c64(g_sT).reshape(NM, self.D)
        gi = None if g_imu is None else _c64(g_imu).reshape(T, NM, 6)
        gk = None if gate_k is None else np.ascontiguousarray(gate_k, dtype=np.int32)
        return lib().oc_loss(C.byref(self.cfg), C.byref(self.scene), _p(_c64(s0)),
                             _p(_c64(actions)), _p(_c64(g_r)), _p(gd), _p(gl), _p(gs), _p(gi),
                             _p(gk, _pi), _p(_c64(imu_noise)), _p(_c64(imu_bias)))

    def cull_counts(self, s):
        """Post-cull work of one render of states s [NM, D] under the
        frustum culling rule (see oc_cull_counts): dict of sphere_tests,
        other_tests (boxes, cylinders, gates), rays, and ambiguous (tests
        that near-threshold decisions could move)."""
        s = _c64(s).reshape(self.NM, self.D)
        out = np.zeros(4)
        lib().oc_cull_counts(C.byref(self.cfg), C.byref(self.scene), _p(s), _p(out))
        return dict(sphere_tests=int(out[0]), other_tests=int(out[1]), rays=int(out[2]), ambiguous=int(out[3]))

    def render(self, s):
        """Sensor outputs of states s [NM, D]: (depth, lidar, hit_cam, hit_lid, amb_cam, amb_lid)."""
        NM = self.NM
        s = _c64(s).reshape(NM, self.D)
        dep, lid = np.zeros((NM, self.Rc)), np.zeros((NM, self.Rl))
        hc, hl = np.zeros((NM, self.Rc), np.int32), np.zeros((NM, self.Rl), np.int32)
        ac, al = np.zeros((NM, self.Rc), np.uint8), np.zeros((NM, self.Rl), np.uint8)
        lib().oc_render(C.byref(self.cfg), C.byref(self.scene), _p(s), _p(dep), _p(lid),
                        _p(hc, _pi), _p(hl, _pi), _p(ac, _pu8), _p(al, _pu8))
        return dep, lid, hc, hl, ac, al


# ----------------------------------------------------------- primitive calls
def _v(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a


def ray_sphere(o, d, sphere):
    return lib().oc_ray_sphere(_p(_v(o)), _p(_v(d)), _p(_v(sphere)))


def ray_box(o, d, box):
    ax = np.zeros(1, np.int32)
    t = lib().oc_ray_box(_p(_v(o)), _p(_v(d)), _p(_v(box)), _p(ax, _pi))
    return t, int(ax[0])


def ray_cylinder(o, d, cyl):
    """(t, face): face 0 side, 1 cap; cyl = (cx, cy, r, zmin, zmax)."""
    f = np.zeros(1, np.int32)
    t = lib().oc_ray_cylinder(_p(_v(o)), _p(_v(d)), _p(_v(cyl)), _p(f, _pi))
    return t, int(f[0])


def ray_gate(o, d, gate):
    """(t, axis): gate = (cx, cy, cz, yaw, w, b, hd); axis 0..2 outer face, 3..4 inner wall."""
    ax = np.zeros(1, np.int32)
    t = lib().oc_ray_gate(_p(_v(o)), _p(_v(d)), _p(_v(gate)), _p(ax, _pi))
    return t, int(ax[0])


def sdf_cylinder(p, cyl):
    return lib().oc_sdf_cylinder(_p(_v(p)), _p(_v(cyl)))


def sdf_gate(p, gate):
    return lib().oc_sdf_gate(_p(_v(p)), _p(_v(gate)), None)


def sdf_sphere(p, sphere):
    return lib().oc_sdf_sphere(_p(_v(p)), _p(_v(sphere)))


def sdf_box(p, box):
    return lib().oc_sdf_box(_p(_v(p)), _p(_v(box)))


def quat_to_rot(q):
    R = np.zeros(9)
    lib().oc_quat_to_rot(_p(_v(q)), _p(R))
    return R.reshape(3, 3)


def pm_step(p, s, a, drag=None, lam=None):
    cfg = make_config(p)
    o = np.zeros(12)
    lib().oc_pm_step(C.byref(cfg), _d(p["drag"] if drag is None else drag),
                     _d(p["lam"] if lam is None else lam), _p(_v(s)), _p(_v(a)), _p(o))
    return o


def pmd_step(p, s, a):
    """One discrete point-mass step (Eq. 4)."""
    cfg = make_config(p)
    o = np.zeros(12)
    lib().oc_pmd_step(C.byref(cfg), _p(_v(s)), _p(_v(a)), _p(o))
    return o


def simple_step(p, s, a):
    """One simplified-quadrotor step (Eq. 2); state (p, v, R row-major)."""
    cfg = make_config(p)
    o = np.zeros(15)
    lib().oc_simple_step(C.byref(cfg), _p(_v(s)), _p(_v(a)), _p(o))
    return o


def rb_step(p, s, a):
    cfg = make_config(p)
    o = np.zeros(13)
    lib().oc_rb_step(C.byref(cfg), _p(_v(s)), _p(_v(a)), _p(o))
    return o


def pose(p, s):
    cfg = make_config(p)
    o, R = np.zeros(3), np.zeros(9)
    f = lib().oc_pose(C.byref(cfg), _p(_v(s)), _p(o), _p(R))
    return o, R.reshape(3, 3), f


def cam_dirs(p):
    cfg = make_config(p)
    R = p["cam"][0] * p["cam"][1]
    d, f = np.zeros((R, 3)), np.zeros(R)
    lib().oc_cam_dirs(C.byref(cfg), _p(d), _p(f))
    return d, f


def lidar_dirs(p):
    cfg = make_config(p)
    R = p["lidar"][0] * p["lidar"][1]
    d = np.zeros((R, 3))
    lib().oc_lidar_dirs(C.byref(cfg), _p(d))
    return d


def max_threads():
    return lib().oc_max_threads()
