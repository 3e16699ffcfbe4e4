"""Pins of the oracle's sensors (Sec. III-B): ray-primitive hits, camera and
LiDAR ray layout, z-depth, the range clamp, signed distances and the
point-mass attitude.

Hits are checked against hand-derived fixtures (tests/golden) and against an
independent method, sphere tracing of the signed distance written here, so a
wrong root, sign or slab in the oracle fails.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _t(x):
    return math.inf if x == "inf" else float(x)


def test_ray_sphere_golden():
    gold = json.load(open(os.path.join(GOLD, "sphere_hits.json")))
    for c in gold["cases"]:
        t = oracle.ray_sphere(c["o"], c["d"], c["sphere"])
        assert t == pytest.approx(_t(c["t"]), abs=1e-12), c["why"]


def test_ray_box_golden():
    gold = json.load(open(os.path.join(GOLD, "box_hits.json")))
    for c in gold["cases"]:
        t, ax = oracle.ray_box(c["o"], c["d"], c["box"])
        assert t == pytest.approx(_t(c["t"]), abs=1e-12), c["why"]
        if 0 < t < math.inf:
            assert ax == c["axis"], c["why"]


# independent signed distances (Euclidean) for sphere tracing
def _sdf_sphere(p, s):
    return np.linalg.norm(p - s[:3]) - s[3]


def _sdf_box(p, b):
    c, h = 0.5 * (b[:3] + b[3:]), 0.5 * (b[3:] - b[:3])
    q = np.abs(p - c) - h
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


def test_ray_sphere_vs_sphere_tracing():
    rng = np.random.default_rng(0)
    n = 0
    while n < 300:
        o = rng.uniform(-5, 5, 3)
        c = rng.uniform(-5, 5, 3)
        r = rng.uniform(0.3, 2.0)
        if np.linalg.norm(o - c) <= r + 1e-3:
            continue
        d = (c - o) + rng.normal(0, 1.0, 3)
        d /= np.linalg.norm(d)
        oc = c - o
        b = d @ oc
        disc = b * b - (oc @ oc - r * r)
        if abs(disc) < 1e-2:  # grazing rays stall sphere tracing
            continue
        s = np.array([*c, r])
        t = oracle.ray_sphere(o, d, s)
        tm = _march(o, d, lambda p: _sdf_sphere(p, s))
        if math.isinf(tm):
            assert math.isinf(t)
        else:
            assert t == pytest.approx(tm, abs=1e-9)
        n += 1


def test_ray_box_vs_sphere_tracing():
    rng = np.random.default_rng(1)
    n = hits = 0
    while n < 300:
        o = rng.uniform(-5, 5, 3)
        c = rng.uniform(-4, 4, 3)
        h = rng.uniform(0.2, 1.5, 3)
        b = np.concatenate([c - h, c + h])
        if _sdf_box(o, b) <= 1e-3:
            continue
        d = (c - o) + rng.normal(0, 1.0, 3)
        d /= np.linalg.norm(d)
        t, _ = oracle.ray_box(o, d, b)
        tm = _march(o, d, lambda p: _sdf_box(p, b))
        if math.isnan(tm):
            continue  # grazing an edge: tracing stalls
        if math.isinf(tm):
            assert math.isinf(t)
        else:
            hits += 1
            assert t == pytest.approx(tm, abs=1e-9)
        n += 1
    assert hits > 50


def test_origin_inside_gives_zero():
    assert oracle.ray_sphere([0.1, 0, 0], [0, 0, 1], [0, 0, 0, 1]) == 0.0
    t, _ = oracle.ray_box([0.1, 0.2, 0.3], [0, 0, 1], [-1, -1, -1, 1, 1, 1])
    assert t == 0.0


def test_sdf_closed_forms():
    assert oracle.sdf_sphere([3, 4, 0], [0, 0, 0, 1]) == pytest.approx(4.0)
    assert oracle.sdf_sphere([0.5, 0, 0], [0, 0, 0, 1]) == pytest.approx(-0.5)
    b = [-1, -2, -3, 1, 2, 3]
    assert oracle.sdf_box([4, 0, 0], b) == pytest.approx(3.0)            # face
    assert oracle.sdf_box([4, 6, 0], b) == pytest.approx(5.0)            # edge: 3-4-5
    assert oracle.sdf_box([3, 4, 5], b) == pytest.approx(math.sqrt(4 + 4 + 4))  # corner
    assert oracle.sdf_box([0.5, 0, 0], b) == pytest.approx(-0.5)         # inside, nearest face x
    assert oracle.sdf_box([0, 0, 2.5], b) == pytest.approx(-0.5)         # inside, nearest face z


def test_camera_rays_layout():
    W, H, hfov = 8, 6, 90.0
    p = synth.params(cam=(W, H, hfov, 10.0))
    d, f = oracle.cam_dirs(p)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=1e-15)
    np.testing.assert_allclose(f, d[:, 0], atol=1e-15)
    th = math.tan(math.radians(hfov) / 2)
    # left-most column centre: horizontal offset (1 - 1/W) tan(hfov/2), to +y_B
    r = 0 * W + 0
    assert d[r, 1] / d[r, 0] == pytest.approx((1 - 1 / W) * th)
    # top row centre: vertical offset (1 - 1/H) tan(vfov/2) upward, square pixels
    assert d[r, 2] / d[r, 0] == pytest.approx((1 - 1 / H) * th * H / W)
    # right-bottom pixel mirrors top-left
    r2 = (H - 1) * W + (W - 1)
    np.testing.assert_allclose(d[r2], [d[r, 0], -d[r, 1], -d[r, 2]], atol=1e-15)


def _single_env(p, spheres=(), boxes=()):
    sp = np.array(spheres, float).reshape(-1, 4)
    bx = np.array(boxes, float).reshape(-1, 6)
    NM = p["n_env"] * p["n_agent"]
    D = synth.STATE_DIM[p["model"]]
    return dict(spheres=sp, sph_off=np.array([0, len(sp)], np.int32), boxes=bx,
                box_off=np.array([0, len(bx)], np.int32),
                env_map=np.zeros(p["n_env"], np.int32), targets=np.zeros((NM, 3)),
                pool=np.zeros((max(p["pool_size"], 1), NM, D)))


def test_wall_gives_constant_z_depth():
    # a wall x in [5, 6] facing a level camera: z-depth is 5 at every pixel
    p = synth.params(model="rigid", n_env=1, cam=(16, 9, 90.0, 10.0))
    o = oracle.Oracle(p, _single_env(p, boxes=[(5, -100, -100, 6, 100, 100)]))
    s = np.array([[0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0]], float)
    dep, _, hc, _, _, _ = o.render(s)
    np.testing.assert_allclose(dep, 5.0, atol=1e-12)
    assert (hc == 0).all()


def test_depth_clamped_at_range_and_miss():
    p = synth.params(model="rigid", n_env=1, cam=(4, 3, 90.0, 10.0))
    o = oracle.Oracle(p, _single_env(p, boxes=[(12, -100, -100, 13, 100, 100)]))
    s = np.array([[0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0]], float)
    dep, _, hc, _, _, _ = o.render(s)
    np.testing.assert_allclose(dep, 10.0)
    o = oracle.Oracle(p, _single_env(p))
    dep, _, hc, _, _, _ = o.render(s)
    np.testing.assert_allclose(dep, 10.0)
    assert (hc == -1).all()


def test_yawed_camera_sees_wall_to_the_left():
    # yaw +90 deg: the optical axis (+x_B) points to world +y
    p = synth.params(model="rigid", n_env=1, cam=(4, 3, 90.0, 10.0))
    o = oracle.Oracle(p, _single_env(p, boxes=[(-100, 3, -100, 100, 4, 100)]))
    c = math.cos(math.pi / 4)
    s = np.array([[0, 0, 0, c, 0, 0, c, 0, 0, 0, 0, 0, 0]], float)
    dep, _, _, _, _, _ = o.render(s)
    np.testing.assert_allclose(dep, 3.0, atol=1e-12)


def test_lidar_ranges_against_wall():
    C, Az = 3, 12
    p = synth.params(model="rigid", n_env=1, cam=None, lidar=(C, Az, -15.0, 15.0, 20.0))
    o = oracle.Oracle(p, _single_env(p, boxes=[(5, -100, -100, 6, 100, 100)]))
    s = np.array([[0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0]], float)
    _, lid, _, _, _, _ = o.render(s)
    for ch, el in enumerate((-15.0, 0.0, 15.0)):
        for k in range(Az):
            az = 2 * math.pi * k / Az
            cx = math.cos(math.radians(el)) * math.cos(az)
            exp = 5.0 / cx if cx > 1e-12 and 5.0 / cx < 20.0 else 20.0
            assert lid[0, ch * Az + k] == pytest.approx(exp, abs=1e-12)


def test_lidar_elevations():
    p = synth.params(lidar=(16, 4, -15.0, 15.0, 20.0))
    d = oracle.lidar_dirs(p)
    el = np.degrees(np.arcsin(d[::4, 2]))
    np.testing.assert_allclose(el, np.linspace(-15, 15, 16), atol=1e-12)
    np.testing.assert_allclose(d[1], [0, math.cos(math.radians(-15)), math.sin(math.radians(-15))], atol=1e-15)


def test_pointmass_attitude():
    p = synth.params(model="pm")
    # thrust straight up, velocity EMA along +y: x_B = +y, z_B = +z, y_B = -x
    s = np.zeros(12)
    s[6:9] = [0, 0, 9.81]
    s[9:12] = [0, 2.0, 0.5]
    o, R, f = oracle.pose(p, s)
    np.testing.assert_allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    assert f == 0
    # tilted thrust: z_B along a, x_B orthogonal to z_B in the plane of z_B and the heading
    rng = np.random.default_rng(0)
    for _ in range(50):
        s[6:9] = rng.normal(0, 3, 3) + [0, 0, 9.81]
        s[9:12] = rng.normal(0, 2, 3)
        o, R, f = oracle.pose(p, s)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0)
        np.testing.assert_allclose(R[:, 2], s[6:9] / np.linalg.norm(s[6:9]), atol=1e-14)
        h = np.array([s[9], s[10], 0.0])
        assert R[:, 0] @ h > 0
        assert abs(np.cross(R[:, 2], h) @ R[:, 0]) < 1e-12
    # degenerate: zero thrust and zero heading -> level, facing +x
    o, R, f = oracle.pose(p, np.zeros(12))
    np.testing.assert_allclose(R, np.eye(3), atol=1e-15)
    assert f & 1 and f & 2
