"""Pins of the closed-loop policy-gradient oracle: the policy network's
backward pass and the whole closed-loop gradient (policy -> actions ->
simulator step -> rendered observation -> next action, Eq. 5) against
central finite differences of the oracle's own forward map in FP64, on
tiny screened instances; closed forms of the activations."""
import numpy as np
import pytest

import oracle
from oracle import policy as PO
from paper_2509_10247_b300 import synth


def _tiny(**kw):
    p = synth.preset("rigid_65536env_256obst_depth_lidar", n_env=2, horizon=3, cam=(6, 4, 90.0, 10.0),
                     lidar=(2, 8, -15.0, 15.0, 10.0), map_counts=[(3, 2)], obst_lo=(2.0, -3.0, -1.0),
                     obst_hi=(7.0, 3.0, 3.0), init_lo=(-1.0, -1.0, 0.5), init_hi=(1.0, 1.0, 1.5),
                     bound_lo=(-np.inf,) * 3, bound_hi=(np.inf,) * 3, terminate=0, w_obs=5.0, d_safe=4.0)
    p.update(kw)
    return p


def test_tanh_and_silu_closed_forms():
    P = {"W1": np.zeros((256, 20)), "b1": np.zeros(256), "W2": np.zeros((4, 256)), "b2": np.array([0, 1, -1, 40.0])}
    f = PO.forward(P, np.zeros((3, 20)), rounding=False)
    np.testing.assert_allclose(f["y"][0], np.tanh([0, 1, -1, 40.0]))
    assert (f["h"] == 0).all()  # silu(0) = 0


def test_policy_backward_matches_central_differences():
    p = _tiny()
    rng = np.random.default_rng(3)
    P = PO.split(p, synth.policy_init(p, seed=4, scale=2.0))
    obs = rng.standard_normal((5, PO.n_features(p)))
    gy = rng.standard_normal((5, 4))
    f = PO.forward(P, obs, rounding=False)
    g, g_obs = PO.backward(P, f, gy, rounding=False)
    L = lambda Q, o: float(np.sum(gy * PO.forward(Q, o, rounding=False)["y"]))
    for k, arr in P.items():
        for ix in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(8)]:
            Qp = {kk: v.copy() for kk, v in P.items()}
            Qm = {kk: v.copy() for kk, v in P.items()}
            Qp[k][ix] += 1e-6
            Qm[k][ix] -= 1e-6
            fd = (L(Qp, obs) - L(Qm, obs)) / 2e-6
            assert abs(fd - g[k][ix]) <= 1e-6 * abs(fd) + 1e-9, (k, ix)
    for ix in [tuple(rng.integers(0, s) for s in obs.shape) for _ in range(8)]:
        op, om = obs.copy(), obs.copy()
        op[ix] += 1e-6
        om[ix] -= 1e-6
        fd = (L(P, op) - L(P, om)) / 2e-6
        assert abs(fd - g_obs[ix]) <= 1e-6 * abs(fd) + 1e-9


def test_closed_loop_gradient_matches_central_differences():
    p = _tiny()
    inp = synth.make_inputs(p, seed=7)
    orc = oracle.Oracle(p, inp)
    flat = synth.policy_init(p, seed=8, scale=1.0).astype(np.float64)
    P = PO.split(p, flat)
    g_r = synth.cotangents(p, seed=9)["g_r"]
    L0, grads, rec = PO.closed_loop(orc, P, inp["s0"], g_r, rounding=False)
    assert rec["amb"].sum() == 0
    rng = np.random.default_rng(10)
    gflat = np.concatenate([grads[k].reshape(-1) for k, _ in PO.shapes(p)])
    scale = np.abs(gflat).max()
    idx = np.concatenate([rng.integers(0, flat.size, 24),
                          np.arange(flat.size - 4 - 1024, flat.size)[rng.integers(0, 1028, 16)]])

    def L(v):
        return PO.closed_loop(orc, PO.split(p, v), inp["s0"], g_r, rounding=False)[0]

    checked = 0
    for i in idx:
        d = []
        for h in (1e-6, 2e-6):
            vp, vm = flat.copy(), flat.copy()
            vp[i] += h
            vm[i] -= h
            d.append((L(vp) - L(vm)) / (2 * h))
        if abs(d[0] - d[1]) > 1e-6 * max(abs(d[0]), scale):
            continue  # a branch of the forward map crossed within the step
        assert abs(gflat[i] - d[0]) <= 1e-5 * max(abs(d[0]), scale), (i, gflat[i], d[0])
        checked += 1
    assert checked >= 30
