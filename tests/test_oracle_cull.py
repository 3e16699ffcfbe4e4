"""Pins of the oracle's count of the culled ray-casting work (Sec. III-B:
rays are cast only against the primitives a sensor's field of view can
reach).  Hand-placed primitives in front of, behind, beside, above and
beyond a camera and a LiDAR with a known pose fix every branch of the rule;
and the rule must be conservative: every primitive that some ray of the
brute-force cast actually hits has to be among the counted ones."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_10247_b300 import synth


def _one(spheres=(), boxes=(), cam=(16, 9, 90.0, 10.0), lidar=None, model="rigid"):
    """One rigid agent at the origin, identity attitude (camera along +x,
    y left, z up), with the given primitives in its map."""
    p = synth.params(model=model, n_env=1, n_agent=1, horizon=1, cam=cam, lidar=lidar,
                     map_counts=[(len(spheres), len(boxes))])
    inp = synth.make_inputs(p, seed=0)
    inp["spheres"] = np.array(spheres, dtype=float).reshape(-1, 4)
    inp["boxes"] = np.array(boxes, dtype=float).reshape(-1, 6)
    inp["sph_off"] = np.array([0, len(spheres)], np.int32)
    inp["box_off"] = np.array([0, len(boxes)], np.int32)
    o = oracle.Oracle(p, inp)
    s = np.zeros((1, o.D))
    if model == "rigid":
        s[0, 3] = 1.0  # q = (1, 0, 0, 0)
    return o, s


def _kept(spheres=(), boxes=(), **kw):
    o, s = _one(spheres, boxes, **kw)
    c = o.cull_counts(s)
    R = o.Rc + o.Rl
    assert c["rays"] == R and c["ambiguous"] == 0
    return c["sphere_tests"] / max(o.Rc or o.Rl, 1), c["other_tests"] / max(o.Rc or o.Rl, 1)


def test_camera_frustum_cases():
    # straight ahead, behind, beyond range, beside (outside the 45 deg half
    # angle: direction 60 deg off-axis at 5 m, radius 0.5)
    ahead = (5.0, 0.0, 0.0, 0.5)
    behind = (-5.0, 0.0, 0.0, 0.5)
    far = (30.0, 0.0, 0.0, 0.5)
    side = (5 * math.cos(math.radians(60)), 5 * math.sin(math.radians(60)), 0.0, 0.5)
    assert _kept([ahead]) == (1, 0)
    assert _kept([behind]) == (0, 0)
    assert _kept([far]) == (0, 0)
    assert _kept([side]) == (0, 0)
    # the same direction with a radius reaching back across the side plane:
    # the plane is at 45 deg, the centre 15 deg beyond it at 5 m, so its
    # distance to the plane is 5 sin(15 deg) = 1.294 m
    d = 5 * math.sin(math.radians(15))
    assert _kept([side[:3] + (d - 0.01,)]) == (0, 0)
    assert _kept([side[:3] + (d + 0.01,)]) == (1, 0)
    # vertical: the 16x9 image spans atan(tan(45 deg) 9 / 16) = 29.4 deg above the axis
    up = (5 * math.cos(math.radians(40)), 0.0, 5 * math.sin(math.radians(40)), 0.3)
    assert _kept([up]) == (0, 0)
    # a box ahead counts among the other kinds; one behind does not
    assert _kept(boxes=[(4, -1, -1, 6, 1, 1)]) == (0, 1)
    assert _kept(boxes=[(-6, -1, -1, -4, 1, 1)]) == (0, 0)
    assert _kept([ahead, behind, far], [(4, -1, -1, 6, 1, 1)]) == (1, 1)


def test_range_uses_the_longest_unclamped_ray():
    # the corner ray's length at the 10 m z-depth clamp: 10 sqrt(1 + u^2 + v^2)
    th = 1.0
    u, v = (1 - 1 / 16) * th, (1 - 1 / 9) * th * 9 / 16
    L = 10 * math.sqrt(1 + u * u + v * v)
    # a small sphere along the corner direction, just inside / outside that length
    d = np.array([1.0, u, v]) / math.sqrt(1 + u * u + v * v)
    r = 0.1
    inside = tuple((L + r - 0.01) * d) + (r,)
    outside = tuple((L + r + 0.01) * d) + (r,)
    assert _kept([inside]) == (1, 0)
    assert _kept([outside]) == (0, 0)


def test_origin_inside_casts_no_test():
    o, s = _one([(0.0, 0.0, 0.0, 1.0), (5.0, 0.0, 0.0, 0.5)])
    c = o.cull_counts(s)
    assert c["sphere_tests"] == 0 and c["other_tests"] == 0 and c["rays"] == o.Rc
    o, s = _one(boxes=[(-1, -1, -1, 1, 1, 1)], spheres=[(5.0, 0.0, 0.0, 0.5)])
    assert o.cull_counts(s)["sphere_tests"] == 0


def test_lidar_elevation_band():
    lid = (16, 360, -15.0, 15.0, 20.0)
    level = (8.0, 3.0, 0.0, 0.5)                      # elevation 0: kept
    high = (8 * math.cos(math.radians(40)), 0.0, 8 * math.sin(math.radians(40)), 0.5)  # 40 deg up: culled
    # 20 deg up with angular radius asin(r / 8): reaches below 15 deg + 1 mrad iff asin(r/8) > 5 deg - 1 mrad
    edge = math.radians(20)
    r_in = 8 * math.sin(math.radians(5) + 0.002)
    r_out = 8 * math.sin(math.radians(5) - 0.01)
    base = (8 * math.cos(edge), 0.0, 8 * math.sin(edge))
    behind = (-8.0, 0.0, 0.0, 0.5)                    # the LiDAR sees all azimuths: kept
    assert _kept([level], cam=None, lidar=lid) == (1, 0)
    assert _kept([behind], cam=None, lidar=lid) == (1, 0)
    assert _kept([high], cam=None, lidar=lid) == (0, 0)
    assert _kept([base + (r_in,)], cam=None, lidar=lid) == (1, 0)
    assert _kept([base + (r_out,)], cam=None, lidar=lid) == (0, 0)
    assert _kept([(25.0, 0.0, 0.0, 0.5)], cam=None, lidar=lid) == (0, 0)  # beyond 20 m


def test_cull_is_conservative_against_brute_force_hits():
    """Every primitive some ray hits in the brute-force cast is counted."""
    p = synth.preset("rigid_65536env_256obst_depth_lidar", n_env=1, horizon=1)
    p = dict(p, cam=(16, 12, 90.0, 20.0), lidar=(8, 90, -15.0, 15.0, 20.0))
    inp = synth.make_inputs(p, seed=5)
    o = oracle.Oracle(p, inp)
    rng = np.random.default_rng(0)
    for _ in range(40):
        s = np.zeros((1, o.D))
        s[0, :3] = rng.uniform([-15, -15, 1], [15, 15, 9])
        q = rng.standard_normal(4)
        s[0, 3:7] = q / np.linalg.norm(q)
        c = o.cull_counts(s)
        dep, lid, hc, hl, _, _ = o.render(s)
        # hits nearer than the range clamp (the cast records farther ones too)
        hit_cam = set(int(h) for h, z in zip(hc.ravel(), dep.ravel()) if h >= 0 and z < p["cam"][3])
        hit_lid = set(int(h) for h, z in zip(hl.ravel(), lid.ravel()) if h >= 0 and z < p["lidar"][4])
        ns = int(np.diff(inp["sph_off"])[0])
        if c["sphere_tests"] == 0 and c["other_tests"] == 0:
            continue  # origin inside a primitive
        # per sensor kept counts are not separated in the totals; their sum
        # bounds the distinct hits of both sensors from above
        kept_s = c["sphere_tests"]
        kept_o = c["other_tests"]
        need_s = o.Rc * sum(1 for h in hit_cam if h < ns) + o.Rl * sum(1 for h in hit_lid if h < ns)
        need_o = o.Rc * sum(1 for h in hit_cam if h >= ns) + o.Rl * sum(1 for h in hit_lid if h >= ns)
        assert kept_s >= need_s and kept_o >= need_o
