"""Seeded synthetic workloads for the batched quadrotor environment step.

This module only draws inputs: initial states, action sequences, obstacle maps,
targets and the reset pool, for the workloads of the paper's tasks (position
control and obstacle avoidance, Sec. III-C) with the dynamics of Eq. 1 (rigid
body) and Eq. 3 (continuous point mass).  It holds none of the method's
arithmetic: both the CUDA library and the FP64 oracle consume what it returns.

Every array is drawn from ``numpy.random.default_rng(seed)`` in one fixed order:
  1. initial positions            [N*M, 3]
  2. per-env targets              [N, 3]
  3. actions                      [T, N*M, A]
  4. per map: sphere centres, sphere radii, box centres, box half-extents
  5. reset-pool positions         [P, N*M, 3]
  6. per-env drag and latency factors (only when ranges are given)
  7. per map with cylinders or gates: cylinder centres (xy), radii, centre
     heights and half-heights, then gate positions, yaw jitters and
     half-widths (only for maps whose counts name them)
All floating-point values are rounded to float32 once, so the FP32 device path
and the FP64 oracle start from bit-identical numbers.

State layout (one agent, float components in this order):
  point mass (Eq. 3, Eq. 4) (D=12): p[3], v[3], a[3], ema_v[3]
  rigid body (Eq. 1)        (D=13): p[3], q[4] (w, x, y, z), v[3], omega[3]
  simplified (Eq. 2)        (D=15): p[3], v[3], R[9] (row-major, body -> world)
Action layout: point mass A=3 (acceleration command in [-1, 1]^3),
rigid body and simplified A=4 (collective thrust, then three body rates,
each in [-1, 1]).
"""
from __future__ import annotations

import copy
import math

import numpy as np

INF = float("inf")

STATE_DIM = {"pm": 12, "rigid": 13, "pm_disc": 12, "simple": 15}
ACTION_DIM = {"pm": 3, "rigid": 4, "pm_disc": 3, "simple": 4}

# Parameters shared by every workload.  Values the paper leaves open are the
# readings listed in the design notes (thrust along +z_B, lag lambda = 1/tau, ...).
_BASE = dict(
    model="pm", n_env=64, n_agent=1, horizon=32, dt=0.01, gravity=9.81,
    # continuous point mass, Eq. 3
    lam=10.0, drag=0.0, act_scale=10.0, ema_alpha=0.1,
    # rigid body, Eq. 1, with the body-rate part of the geometric controller
    mass=1.0, inertia=(0.01, 0.01, 0.02), k_rate=(20.0, 20.0, 10.0),
    drag_body=(0.0, 0.0, 0.0), rate_scale=(3.0, 3.0, 1.5),
    # sensors: camera (W, H, hfov_deg, range_m); lidar (channels, azimuths,
    # elev_lo_deg, elev_hi_deg, range_m); None disables a sensor
    cam=(16, 9, 90.0, 10.0), lidar=None,
    # task / reward (Sec. III-C, Sec. III-E reward split)
    pos_sq=1, w_pos=1.0, w_obs=0.0, d_safe=1.0, w_act=0.01, w_agent=0.0,
    d_agent=0.4, success_radius=0.5, r_quad=0.2,
    bound_lo=(-INF, -INF, -INF), bound_hi=(INF, INF, INF),
    terminate=0, pool_size=4, ckpt_every=16,
    # flight task (Sec. III-C): "reach" (targets; position control and
    # obstacle avoidance) or "racing" (the map's gates in order)
    task="reach",
    # IMU noise (Sec. III-B): white-noise std of specific force / angular
    # rate samples and the std per sqrt(s) of their bias random walks
    imu_noise=(0.0, 0.0), imu_walk=(0.0, 0.0),
    # scene recipe: map_counts is a list of (n_spheres, n_boxes) or
    # (n_spheres, n_boxes, n_cylinders, n_gates) per map; n_maps None means
    # one map per environment with map_counts[0]
    n_maps=None, map_counts=[(10, 0)],
    obst_lo=(-8.0, -8.0, -8.0), obst_hi=(8.0, 8.0, 8.0),
    sph_radius=(0.3, 1.0), box_half=(0.2, 1.5),
    cyl_radius=(0.2, 0.8), cyl_half_height=(0.5, 3.0),
    # racing course: gates on a circle of race_radius around the middle of
    # the obstacle box, each jittered by race_jitter, facing along the loop
    # (counter-clockwise); opening half-width, border width, half-depth
    race_radius=6.0, race_jitter=1.0, gate_half=(0.6, 1.0), gate_border=0.15, gate_depth=0.1,
    init_lo=(-5.0, -5.0, -5.0), init_hi=(5.0, 5.0, 5.0), formation_radius=1.0,
    drag_range=None, lam_range=None,
)


def _split(n, frac_sph=0.7):
    s = int(round(frac_sph * n))
    return (s, n - s)


PRESETS = {
    # 64 point-mass envs, 16x9 depth vs 10 spheres, horizon 32
    "pointmass_64env_depth16x9_10sph": dict(),
    # 4096 rigid-body envs, 64x48 depth vs 40 spheres + 20 boxes, horizon 64
    "rigid_4096env_depth64x48_40sph20box": dict(
        model="rigid", n_env=4096, horizon=64, dt=0.005, cam=(64, 48, 90.0, 10.0),
        map_counts=[(40, 20)], pos_sq=0, w_obs=10.0, terminate=1),
    # 16384 envs x 8 point-mass agents, 8 uneven maps, 16x9 depth per agent, horizon 64
    "swarm_16384env_8agent_8maps_depth16x9": dict(
        n_env=16384, n_agent=8, horizon=64, n_maps=8,
        map_counts=[_split(n) for n in (10, 20, 40, 60, 100, 140, 170, 200)],
        w_obs=10.0, w_agent=10.0, terminate=1),
    # 65536 rigid envs, 256 obstacles each, depth 64x48 + lidar 16x360, horizon 128
    "rigid_65536env_256obst_depth_lidar": dict(
        model="rigid", n_env=65536, horizon=128, dt=0.005,
        cam=(64, 48, 90.0, 20.0), lidar=(16, 360, -15.0, 15.0, 20.0),
        map_counts=[(179, 77)], obst_lo=(-20.0, -20.0, 0.0), obst_hi=(20.0, 20.0, 10.0),
        init_lo=(-18.0, -18.0, 1.0), init_hi=(18.0, 18.0, 9.0),
        bound_lo=(-INF, -INF, 0.0), bound_hi=(INF, INF, 10.0),
        pos_sq=0, w_obs=10.0, terminate=1),
    # rigid-body dynamics alone (no sensor, no obstacle, no termination): the
    # transition source and the rollout workload of the learned surrogate,
    # 65536 envs x 32 steps
    "surrogate_rigid_65536env_32step": dict(
        model="rigid", n_env=65536, horizon=32, dt=0.005, cam=None, map_counts=[(0, 0)],
        n_maps=1, pos_sq=0, terminate=0),
}

# Surrogate MLP sizes (inputs: state 13 + action 4; two hidden layers of 256;
# outputs: the 13 residuals), parameter order W1, b1, W2, b2, W3, b3.
SURR_SHAPES = (("W1", (256, 17)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
               ("W3", (13, 256)), ("b3", (13,)))


def preset(name, **overrides):
    """Return the parameter dict of a named workload, with overrides applied."""
    p = copy.deepcopy(_BASE)
    p.update(copy.deepcopy(PRESETS[name]))
    p.update(overrides)
    p["name"] = name
    return p


def params(**kw):
    """Parameter dict built from the base values and keyword overrides."""
    p = copy.deepcopy(_BASE)
    p.update(kw)
    p.setdefault("name", "custom")
    return p


def n_maps_of(p):
    return p["n_env"] if p["n_maps"] is None else p["n_maps"]


def counts_of_map(p, m):
    """(spheres, boxes) of map m; see counts4_of_map for all four kinds."""
    return tuple(counts4_of_map(p, m)[:2])


def counts4_of_map(p, m):
    """(spheres, boxes, cylinders, gates) of map m."""
    mc = p["map_counts"][m % len(p["map_counts"])]
    return tuple(mc) + (0,) * (4 - len(mc))


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def make_inputs(p, seed=0, actions=True):
    """Draw one workload.  Returns a dict of float64 arrays (float32-exact values)
    and int32 index arrays.  Keys: s0 [NM,D], targets [NM,3], actions [T,NM,A],
    spheres [Ks,4] (cx,cy,cz,r), sph_off [n_maps+1], boxes [Kb,6]
    (min xyz, max xyz), box_off [n_maps+1], env_map [N], pool [P,NM,D],
    drag_env [N] or None, lam_env [N] or None; when a map has cylinders or
    gates also cylinders [Kc,5] (cx,cy,r,zmin,zmax), cyl_off, gates [Kg,7]
    (cx,cy,cz,yaw,w,b,hd), gate_off."""
    rng = np.random.default_rng(seed)
    N, M, T = p["n_env"], p["n_agent"], p["horizon"]
    NM = N * M
    D, A = STATE_DIM[p["model"]], ACTION_DIM[p["model"]]
    lo, hi = np.array(p["init_lo"]), np.array(p["init_hi"])

    # 1. initial positions
    pos0 = rng.uniform(lo, hi, size=(NM, 3))
    # 2. targets: one per env, agents placed on a ring around it (formation)
    tgt_env = rng.uniform(lo, hi, size=(N, 3))
    targets = np.repeat(tgt_env, M, axis=0)
    if M > 1:
        ang = 2.0 * math.pi * np.arange(M) / M
        ring = p["formation_radius"] * np.stack(
            [np.cos(ang), np.sin(ang), np.zeros(M)], axis=1)
        targets = targets + np.tile(ring, (N, 1))
    # 3. actions
    act = rng.uniform(-1.0, 1.0, size=(T, NM, A)) if actions else None
    # 4. obstacle maps
    nm = n_maps_of(p)
    olo, ohi = np.array(p["obst_lo"]), np.array(p["obst_hi"])
    sph, box, so, bo = [], [], [0], [0]
    for m in range(nm):
        ns, nb = counts4_of_map(p, m)[:2]
        c = rng.uniform(olo, ohi, size=(ns, 3))
        r = rng.uniform(p["sph_radius"][0], p["sph_radius"][1], size=(ns, 1))
        bc = rng.uniform(olo, ohi, size=(nb, 3))
        bh = rng.uniform(p["box_half"][0], p["box_half"][1], size=(nb, 3))
        sph.append(np.concatenate([c, r], axis=1))
        box.append(np.concatenate([bc - bh, bc + bh], axis=1))
        so.append(so[-1] + ns)
        bo.append(bo[-1] + nb)
    spheres = np.concatenate(sph, axis=0) if sph else np.zeros((0, 4))
    boxes = np.concatenate(box, axis=0) if box else np.zeros((0, 6))
    env_map = (np.arange(N) % nm).astype(np.int32)
    # 5. reset pool
    P = p["pool_size"]
    pool_pos = rng.uniform(lo, hi, size=(P, NM, 3))
    # 6. domain randomisation of drag and latency (Sec. IV-D)
    drag_env = lam_env = None
    if p.get("drag_range") is not None:
        drag_env = rng.uniform(*p["drag_range"], size=N)
    if p.get("lam_range") is not None:
        lam_env = rng.uniform(*p["lam_range"], size=N)

    # 7. cylinders and racing gates
    cyl, gat, co, go = [], [], [0], [0]
    for m in range(nm):
        _, _, nc, ng = counts4_of_map(p, m)
        if nc:
            cxy = rng.uniform(olo[:2], ohi[:2], size=(nc, 2))
            cr = rng.uniform(p["cyl_radius"][0], p["cyl_radius"][1], size=(nc, 1))
            cz = rng.uniform(olo[2], ohi[2], size=(nc, 1))
            hz = rng.uniform(p["cyl_half_height"][0], p["cyl_half_height"][1], size=(nc, 1))
            cyl.append(np.concatenate([cxy, cr, cz - hz, cz + hz], axis=1))
        if ng:
            mid = 0.5 * (olo + ohi)
            ang = 2.0 * math.pi * np.arange(ng) / ng
            ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(ng)], axis=1) * p["race_radius"]
            gc = mid + ring + rng.uniform(-1.0, 1.0, size=(ng, 3)) * p["race_jitter"]
            yaw = ang + 0.5 * math.pi + rng.uniform(-0.3, 0.3, size=ng)
            gw = rng.uniform(p["gate_half"][0], p["gate_half"][1], size=ng)
            gat.append(np.stack([gc[:, 0], gc[:, 1], gc[:, 2], yaw, gw,
                                 np.full(ng, p["gate_border"]), np.full(ng, p["gate_depth"])], axis=1))
        co.append(co[-1] + nc)
        go.append(go[-1] + ng)
    any4 = co[-1] > 0 or go[-1] > 0

    s0 = _rest_state(p["model"], pos0)
    pool = np.stack([_rest_state(p["model"], pool_pos[k]) for k in range(P)], axis=0)
    out = dict(
        s0=_f32(s0), targets=_f32(targets), actions=None if act is None else _f32(act),
        spheres=_f32(spheres), sph_off=np.array(so, dtype=np.int32),
        boxes=_f32(boxes), box_off=np.array(bo, dtype=np.int32), env_map=env_map,
        pool=_f32(pool),
        drag_env=None if drag_env is None else _f32(drag_env),
        lam_env=None if lam_env is None else _f32(lam_env),
    )
    if any4:
        out.update(cylinders=_f32(np.concatenate(cyl, axis=0) if cyl else np.zeros((0, 5))),
                   cyl_off=np.array(co, dtype=np.int32),
                   gates=_f32(np.concatenate(gat, axis=0) if gat else np.zeros((0, 7))),
                   gate_off=np.array(go, dtype=np.int32))
    return out


def _rest_state(model, pos):
    """Agents at rest at the given positions (level attitude for the rigid body)."""
    n = pos.shape[0]
    s = np.zeros((n, STATE_DIM[model]))
    s[:, 0:3] = pos
    if model == "rigid":
        s[:, 3] = 1.0  # unit quaternion (w, x, y, z) = identity
    if model == "simple":
        s[:, 6] = s[:, 10] = s[:, 14] = 1.0  # rotation matrix = identity
    return s


def cotangents(p, seed=1, depth=True, lidar=True):
    """Seeded N(0, 1) cotangents for the rollout outputs (reward, depth, lidar),
    as the loss-side input of the adjoint.  float64 arrays with float32 values."""
    rng = np.random.default_rng(seed)
    N, M, T = p["n_env"], p["n_agent"], p["horizon"]
    NM = N * M
    out = dict(g_r=_f32(rng.standard_normal((T, NM))))
    if depth and p["cam"] is not None:
        R = p["cam"][0] * p["cam"][1]
        out["g_depth"] = _f32(rng.standard_normal((T, NM, R)))
    if lidar and p["lidar"] is not None:
        R = p["lidar"][0] * p["lidar"][1]
        out["g_lidar"] = _f32(rng.standard_normal((T, NM, R)))
    return out


def surrogate_init(seed=0, scale=1.0):
    """Initial surrogate parameters: weights U(-1, 1) * scale / sqrt(fan_in),
    biases U(-0.1, 0.1) * scale; returns (flat float32 vector, dict of float64
    views with float32 values)."""
    rng = np.random.default_rng(seed)
    parts, views = [], {}
    for name, shape in SURR_SHAPES:
        if name.startswith("W"):
            a = rng.uniform(-1.0, 1.0, size=shape) * scale / math.sqrt(shape[1])
        else:
            a = rng.uniform(-0.1, 0.1, size=shape) * scale
        a = _f32(a)
        views[name] = a
        parts.append(a.reshape(-1))
    return np.concatenate(parts).astype(np.float32), views


def surrogate_split(flat):
    """Dict of float64 arrays from a flat parameter vector."""
    out, o = {}, 0
    flat = np.asarray(flat, dtype=np.float64)
    for name, shape in SURR_SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def surrogate_actions(n_env, steps, seed=0):
    """Random rigid-body actions U(-1, 1)^4 per env and step, float32 [steps, n_env, 4]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(steps, n_env, 4)).astype(np.float32)


def minibatch_order(n, seed, epoch):
    """Seeded permutation of the n transition rows for one epoch (int32)."""
    rng = np.random.default_rng([seed, epoch])
    return rng.permutation(n).astype(np.int32)


# Closed-loop policy (two layers, 256 hidden units, 4 actions); the input
# width is 16 state features + camera rays + LiDAR rays of the workload.
POLICY_HIDDEN = 256


def policy_width(p):
    Rc = p["cam"][0] * p["cam"][1] if p["cam"] is not None else 0
    Rl = p["lidar"][0] * p["lidar"][1] if p["lidar"] is not None else 0
    return 16 + Rc + Rl


def policy_init(p, seed=0, scale=1.0):
    """Initial policy parameters, flat float32 in the order W1 [256, F],
    b1 [256], W2 [4, 256], b2 [4]: weights U(-1, 1) * scale / sqrt(fan_in),
    biases U(-0.1, 0.1) * scale."""
    rng = np.random.default_rng(seed)
    F = policy_width(p)
    parts = []
    for shape in ((POLICY_HIDDEN, F), (POLICY_HIDDEN,), (4, POLICY_HIDDEN), (4,)):
        if len(shape) == 2:
            a = rng.uniform(-1.0, 1.0, size=shape) * scale / math.sqrt(shape[1])
        else:
            a = rng.uniform(-0.1, 0.1, size=shape) * scale
        parts.append(_f32(a).reshape(-1))
    return np.concatenate(parts).astype(np.float32)
