"""Pins of the oracle's cylinder and racing-gate primitives (Sec. III-B: one
ray-casting function per primitive shape; Sec. III-C racing gates as
obstacles).

Hits are checked against closed forms worked out by hand and against sphere
tracing of signed distances written here independently of the oracle (a
cylinder as a 2D box in (radius, height); a gate as the outer box minus the
opening, max(d_outer, -d_opening), a lower bound of the distance that is
exactly zero on the surface, so tracing still lands on the first hit).
Signed distances are checked at points whose nearest surface point is known.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth

CYL = np.array([5.0, 0.0, 1.0, -1.0, 1.0])           # (cx, cy, r, zmin, zmax)
GATE = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 0.2, 0.1])  # (c, yaw, w, b, hd)


# ---------------------------------------------------------------- cylinder
def test_cylinder_closed_form_hits():
    t, f = oracle.ray_cylinder([0, 0, 0], [1, 0, 0], CYL)
    assert t == pytest.approx(4.0, abs=1e-14) and f == 0            # side, x = cx - r
    t, f = oracle.ray_cylinder([5, 0.3, 10], [0, 0, -1], CYL)
    assert t == pytest.approx(9.0, abs=1e-14) and f == 1            # top cap
    t, f = oracle.ray_cylinder([5.2, 0.1, -7], [0, 0, 1], CYL)
    assert t == pytest.approx(6.0, abs=1e-14) and f == 1            # bottom cap from below
    assert math.isinf(oracle.ray_cylinder([7, 0, 5], [0, 0, -1], CYL)[0])   # parallel, outside
    assert math.isinf(oracle.ray_cylinder([0, 0, 1.5], [1, 0, 0], CYL)[0])  # passes above
    assert math.isinf(oracle.ray_cylinder([0, 0, 0], [-1, 0, 0], CYL)[0])   # behind
    assert oracle.ray_cylinder([5.1, 0.2, 0.3], [0, 1, 0], CYL)[0] == 0.0    # inside
    # oblique in a horizontal plane: |t d_xy - c_xy| = r, a circle hit in 2D
    d = np.array([math.cos(0.1), math.sin(0.1), 0.0])
    c = np.array([5.0, 0.0])
    b = c @ d[:2]
    t_exp = b - math.sqrt(1.0 - (c @ c - b * b))
    assert oracle.ray_cylinder([0, 0, 0.5], d, CYL)[0] == pytest.approx(t_exp, abs=1e-13)
    # slanted ray entering through the top cap: z = 1 reached at t = 2 sqrt(2)
    e = np.array([1.0, 0.0, -1.0]) / math.sqrt(2)
    t, f = oracle.ray_cylinder([3, 0, 3], e, CYL)
    assert t == pytest.approx(2 * math.sqrt(2), abs=1e-13) and f == 1


def _sdf_cyl(p, c):
    q = np.array([math.hypot(p[0] - c[0], p[1] - c[1]) - c[2],
                  abs(p[2] - 0.5 * (c[3] + c[4])) - 0.5 * (c[4] - c[3])])
    return np.linalg.norm(np.maximum(q, 0)) + min(q.max(), 0.0)


def _march(o, d, sdf, tmax=60.0):
    t = 0.0
    for _ in range(100000):
        s = sdf(o + t * d)
        if s < 1e-13:
            return t
        t += s
        if t > tmax:
            return math.inf
    return math.nan


def test_cylinder_vs_sphere_tracing():
    rng = np.random.default_rng(3)
    n = hits = caps = 0
    while n < 400:
        o = rng.uniform(-6, 6, 3)
        cxy = rng.uniform(-3, 3, 2)
        r = rng.uniform(0.3, 1.5)
        z0 = rng.uniform(-3, 1)
        cyl = np.array([cxy[0], cxy[1], r, z0, z0 + rng.uniform(0.5, 4)])
        if _sdf_cyl(o, cyl) <= 1e-3:
            continue
        d = np.array([cxy[0], cxy[1], 0.5 * (cyl[3] + cyl[4])]) - o + rng.normal(0, 1.0, 3)
        d /= np.linalg.norm(d)
        t, f = oracle.ray_cylinder(o, d, cyl)
        tm = _march(o, d, lambda p: _sdf_cyl(p, cyl))
        if math.isnan(tm):
            continue  # grazing the rim: tracing stalls
        if math.isinf(tm):
            assert math.isinf(t)
        else:
            hits += 1
            caps += f == 1
            assert t == pytest.approx(tm, abs=1e-9)
        n += 1
    assert hits > 100 and caps > 20


def test_cylinder_sdf_closed_forms():
    assert oracle.sdf_cylinder([5, 0, 3], CYL) == pytest.approx(2.0)          # above the cap
    assert oracle.sdf_cylinder([7.5, 0, 0], CYL) == pytest.approx(1.5)        # beside
    assert oracle.sdf_cylinder([5, 9, 5], CYL) == pytest.approx(math.hypot(8, 4))  # rim
    assert oracle.sdf_cylinder([5, 0, 0], CYL) == pytest.approx(-1.0)         # centre
    assert oracle.sdf_cylinder([5.8, 0, 0.1], CYL) == pytest.approx(-0.2)     # near the side
    assert oracle.sdf_cylinder([5, 0, 0.9], CYL) == pytest.approx(-0.1)       # near the cap


# -------------------------------------------------------------------- gate
def test_gate_closed_form_hits():
    # normal +x, opening |y|, |z| < 1, frame to 1.2, depth |x| <= 0.1
    assert math.isinf(oracle.ray_gate([-5, 0, 0], [1, 0, 0], GATE)[0])      # through the opening
    t, ax = oracle.ray_gate([-5, 0, 1.1], [1, 0, 0], GATE)
    assert t == pytest.approx(4.9, abs=1e-14) and ax == 0                    # top bar, front face
    t, ax = oracle.ray_gate([5, -1.1, 0], [-1, 0, 0], GATE)
    assert t == pytest.approx(4.9, abs=1e-14) and ax == 0                    # right bar from behind
    assert math.isinf(oracle.ray_gate([-5, 0, 1.3], [1, 0, 0], GATE)[0])    # above the frame
    t, ax = oracle.ray_gate([0, 0, 0], [0, 0, 1], GATE)
    assert t == pytest.approx(1.0, abs=1e-14) and ax == 4                    # inner wall (top)
    t, ax = oracle.ray_gate([0.05, 0, 0], [0, 1, 0], GATE)
    assert t == pytest.approx(1.0, abs=1e-14) and ax == 3                    # inner wall (side)
    t, ax = oracle.ray_gate([0, 0, 5], [0, 0, -1], GATE)
    assert t == pytest.approx(3.8, abs=1e-14) and ax == 2                    # top face from above
    assert oracle.ray_gate([0, 0, 1.1], [1, 0, 0], GATE)[0] == 0.0           # inside a bar
    # enters the opening's prism through its open face, then meets the top wall:
    # from (-1, 0, 0) towards (0.05, 0, 1): wall z = 1 at t = |(1.05, 0, 1)|
    e = np.array([1.05, 0.0, 1.0])
    t, ax = oracle.ray_gate([-1, 0, 0], e / np.linalg.norm(e), GATE)
    assert t == pytest.approx(np.linalg.norm(e), abs=1e-13) and ax == 4
    # yaw 90 deg: the normal is +y
    g = GATE.copy()
    g[3] = math.pi / 2
    t, ax = oracle.ray_gate([0, -5, 1.1], [0, 1, 0], g)
    assert t == pytest.approx(4.9, abs=1e-13) and ax == 0
    assert math.isinf(oracle.ray_gate([0, -5, 0.5], [0, 1, 0], g)[0])


def _sdf_box(p, c, h):
    q = np.abs(p - c) - h
    return np.linalg.norm(np.maximum(q, 0)) + min(q.max(), 0.0)


def _gate_local(p, g):
    cs, sn = math.cos(g[3]), math.sin(g[3])
    r = p - g[:3]
    return np.array([cs * r[0] + sn * r[1], -sn * r[0] + cs * r[1], r[2]])


def _sdf_gate_bound(p, g):
    # frame = outer box minus the open square prism: max(d_outer, -d_opening),
    # the opening as a 2D box in (u_l, u_z)
    u = _gate_local(p, g)
    W = g[4] + g[5]
    d_out = _sdf_box(u, np.zeros(3), np.array([g[6], W, W]))
    d_open = _sdf_box(u[1:], np.zeros(2), np.array([g[4], g[4]]))
    return max(d_out, -d_open)


def test_gate_vs_sphere_tracing():
    rng = np.random.default_rng(4)
    n = hits = inner = 0
    while n < 400:
        g = np.array([*rng.uniform(-2, 2, 3), rng.uniform(-math.pi, math.pi),
                      rng.uniform(0.5, 1.2), rng.uniform(0.1, 0.4), rng.uniform(0.05, 0.3)])
        o = rng.uniform(-5, 5, 3)
        if _sdf_gate_bound(o, g) <= 1e-3:
            continue
        d = g[:3] - o + rng.normal(0, 0.8, 3)
        d /= np.linalg.norm(d)
        t, ax = oracle.ray_gate(o, d, g)
        tm = _march(o, d, lambda p: _sdf_gate_bound(p, g))
        if math.isnan(tm):
            continue
        if math.isinf(tm):
            assert math.isinf(t)
        else:
            hits += 1
            inner += ax >= 3
            assert t == pytest.approx(tm, abs=1e-8)
        n += 1
    assert hits > 100 and inner > 10


def test_gate_sdf_closed_forms():
    assert oracle.sdf_gate([-0.6, 0, 1.1], GATE) == pytest.approx(0.5)        # in front of the top bar
    assert oracle.sdf_gate([0, 0, 0], GATE) == pytest.approx(1.0)             # centre of the opening
    assert oracle.sdf_gate([-3, 0, 0], GATE) == pytest.approx(math.hypot(2.9, 1.0))
    assert oracle.sdf_gate([0, 0, 3], GATE) == pytest.approx(1.8)             # above
    assert oracle.sdf_gate([0, 0, 1.1], GATE) == pytest.approx(-0.1)          # inside the top bar
    g = GATE.copy()
    g[3] = math.pi / 2
    assert oracle.sdf_gate([1.1, -0.6, 0], g) == pytest.approx(0.5)           # yawed: side bar


# -------------------------------------------------- rendering with the new kinds
def _scene(p, spheres=(), boxes=(), cyl=(), gates=()):
    NM = p["n_env"] * p["n_agent"]
    D = synth.STATE_DIM[p["model"]]
    arr = lambda x, k: np.array(x, float).reshape(-1, k)
    sp, bx, cy, gt = arr(spheres, 4), arr(boxes, 6), arr(cyl, 5), arr(gates, 7)
    off = lambda a: np.array([0, len(a)], np.int32)
    return dict(spheres=sp, sph_off=off(sp), boxes=bx, box_off=off(bx), cylinders=cy,
                cyl_off=off(cy), gates=gt, gate_off=off(gt), env_map=np.zeros(p["n_env"], np.int32),
                targets=np.zeros((NM, 3)), pool=np.zeros((max(p["pool_size"], 1), NM, D)))


def test_render_cylinder_depth_and_lowest_id_ties():
    p = synth.params(model="rigid", n_env=1, cam=(16, 9, 90.0, 10.0))
    level = np.array([[0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0]], float)
    # a tall cylinder ahead: z-depth of each hit pixel from the circle in xy
    dep, _, hc, _, _, _ = oracle.Oracle(p, _scene(p, cyl=[(5, 0.3, 1, -10, 10)])).render(level)
    dirs, fac = oracle.cam_dirs(p)
    c = np.array([5.0, 0.3])
    n = 0
    for r in range(len(fac)):
        d = dirs[r]
        a, b = d[:2] @ d[:2], c @ d[:2]
        disc = b * b - a * (c @ c - 1.0)
        if disc <= 0:
            assert hc[0, r] == -1
            continue
        n += 1
        assert hc[0, r] == 0
        assert dep[0, r] == pytest.approx((b - math.sqrt(disc)) / a * fac[r], abs=1e-12)
    assert n > 5
    # a gate whose front face is flush with a wall's face: every tie goes to
    # the lower id (the wall), so the gate is never reported
    gate = [(4.1, 0, 0, 0, 1, 0.2, 0.1)]
    _, _, hc, _, _, _ = oracle.Oracle(p, _scene(p, gates=gate)).render(level)
    assert (hc == 0).any()
    sc = _scene(p, boxes=[(4, -100, -100, 5, 100, 100)], gates=gate)
    dep, _, hc, _, _, _ = oracle.Oracle(p, sc).render(level)
    assert (hc == 0).all()
    # a wall behind a gate: the opening shows the wall, the bars are nearer
    sc = _scene(p, boxes=[(8, -100, -100, 9, 100, 100)], gates=[(3, 0, 0, 0, 1, 0.5, 0.1)])
    dep, _, hc, _, _, _ = oracle.Oracle(p, sc).render(level)
    assert (hc == 0).any() and (hc == 1).any()
    np.testing.assert_allclose(dep[hc == 0], 8.0, atol=1e-12)      # the wall
    np.testing.assert_allclose(dep[hc == 1], 2.9, atol=1e-12)      # the frame's front face
