"""Pins of the surrogate-MLP oracle: bf16 rounding from the IEEE definition
(hand-worked values and the library conversion), SiLU closed forms, the
plain network against an independent library formulation, the backward
pass against central differences, Adam's first steps in closed form, the
statistics and the trained-range test on constructed data."""
import numpy as np
import pytest
import torch

from oracle import surrogate as S


# ------------------------------------------------------------------ bf16
@pytest.mark.parametrize("x,want", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                    # tie: even significand (…0) wins
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),     # tie between …1 and …10: even
    (1.0 + 2.0 ** -8 + 2.0 ** -30, 1.0 + 2.0 ** -7),
    (-2.5, -2.5),
    (np.pi, 3.140625),                          # 1.1001001|0000111... rounds down
    (1.0 / 3.0, 0.333984375),                   # 1.0101010|1010... rounds up
    (2.0 ** -133, 2.0 ** -133),                 # smallest subnormal
    (2.0 ** -134, 0.0),                         # tie with zero: even
    (3 * 2.0 ** -135, 2.0 ** -133),
    ((2 - 2.0 ** -7) * 2.0 ** 127, (2 - 2.0 ** -7) * 2.0 ** 127),  # largest finite
    ((2 - 2.0 ** -8) * 2.0 ** 127, np.inf),      # tie beyond the largest: overflows
    (0.0, 0.0),
    (np.inf, np.inf),
])
def test_bf16_hand_values(x, want):
    got = S.bf16_round(np.array([x, -x]))
    assert got[0] == want and got[1] == -want


def test_bf16_matches_library_conversion_of_float32():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(20000) * np.exp2(rng.integers(-60, 60, 20000)),
        rng.uniform(-1, 1, 2000) * 2.0 ** -128,      # subnormal range
        (1 + rng.integers(0, 2 ** 16, 2000) * 2.0 ** -16) * np.exp2(rng.integers(-20, 20, 2000)),
    ]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(x.astype(np.float64)), ref)


def test_bf16_nan_and_signed_zero():
    r = S.bf16_round(np.array([np.nan, -0.0]))
    assert np.isnan(r[0]) and r[1] == 0 and np.signbit(r[1])


# ------------------------------------------------------------------ SiLU
def test_silu_closed_forms():
    assert S.silu(0.0) == 0.0 and S.dsilu(0.0) == 0.5
    assert abs(S.silu(40.0) - 40.0) < 1e-12 and abs(S.silu(-40.0)) < 1e-15
    assert abs(S.silu(1.0) - 1.0 / (1.0 + np.exp(-1.0))) < 1e-15
    z = np.linspace(-6, 6, 97)
    fd = (S.silu(z + 1e-6) - S.silu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(S.dsilu(z), fd, rtol=1e-8, atol=1e-10)


# ------------------------------------------------------------------ network
def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    P = {}
    for name, (o, i) in (("1", (256, 17)), ("2", (256, 256)), ("3", (13, 256))):
        P["W" + name] = (rng.uniform(-1, 1, (o, i)) * scale / np.sqrt(i)).astype(np.float32).astype(np.float64)
        P["b" + name] = (rng.uniform(-0.1, 0.1, o)).astype(np.float32).astype(np.float64)
    return P


def test_plain_forward_matches_library_layers():
    P = _params(1)
    x = np.random.default_rng(2).standard_normal((5, 17))
    y = S.forward(P, x, rounding=False)["y"]
    t = lambda a: torch.from_numpy(np.asarray(a, np.float64))
    F = torch.nn.functional
    h = F.silu(F.linear(t(x), t(P["W1"]), t(P["b1"])))
    h = F.silu(F.linear(h, t(P["W2"]), t(P["b2"])))
    ref = F.linear(h, t(P["W3"]), t(P["b3"])).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_rounded_forward_is_within_bf16_error_of_plain():
    P = _params(3)
    x = np.random.default_rng(4).standard_normal((64, 17))
    a = S.forward(P, x, rounding=True)["y"]
    b = S.forward(P, x, rounding=False)["y"]
    assert np.abs(a - b).max() <= 2.0 ** -5 * np.abs(b).max()
    assert np.abs(a - b).max() > 0  # the rounding points are live


def test_backward_matches_central_differences():
    P = _params(5, scale=2.0)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((4, 17))
    t = rng.standard_normal((4, 13))
    _, g, _ = S.loss_grads(P, x, t, rounding=False)
    eps = 1e-6
    for name, arr in P.items():
        idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]
        for ix in idx:
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][ix] += eps
            Pm[name][ix] -= eps
            fd = (S.loss_grads(Pp, x, t, rounding=False)[0] - S.loss_grads(Pm, x, t, rounding=False)[0]) / (2 * eps)
            # FD noise: loss rounding ~1e-15 / 2e-6 plus O(eps^2) truncation
            assert abs(fd - g[name][ix]) <= 1e-6 * abs(fd) + 2e-9, (name, ix, fd, g[name][ix])


def test_rounded_backward_is_within_bf16_error_of_plain():
    P = _params(7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((32, 17))
    t = rng.standard_normal((32, 13))
    _, ga, _ = S.loss_grads(P, x, t, rounding=True)
    _, gb, _ = S.loss_grads(P, x, t, rounding=False)
    for k in ga:
        assert np.abs(ga[k] - gb[k]).max() <= 2.0 ** -4 * np.abs(gb[k]).max(), k


# ------------------------------------------------------------------ Adam
def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(9)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    w1, m, v = S.adam_step(w, g, m, v, 1)
    # bias-corrected moments of the first step are g and g^2
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    w2, m, v = S.adam_step(w1, g, m, v, 2)
    np.testing.assert_allclose(w2, w1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.19 * g, rtol=1e-14)
    np.testing.assert_allclose(v, (0.001 + 0.999 * 0.001) * g * g, rtol=1e-14)


# ------------------------------------------------------------------ statistics, range, step
def test_column_stats_closed_forms():
    n = 1001
    k = np.arange(n, dtype=np.float64)
    X = np.stack([k * (j + 1) for j in range(17)], axis=1)
    X[:, 5] = 3.0  # constant column
    D = np.stack([np.where(k % 2 == 0, 1.0, -1.0) * (j + 1) for j in range(13)], axis=1)
    st = S.column_stats(X, D)
    np.testing.assert_allclose(st["mu_x"][0], 500.0)
    np.testing.assert_allclose(st["sd_x"][0], np.sqrt((n * n - 1) / 12.0), rtol=1e-13)
    assert st["rs_x"][5] == 1.0 and st["mu_x"][5] == 3.0
    np.testing.assert_allclose(st["mu_d"][2], 3.0 / n, rtol=1e-12)
    assert st["lo_x"][1] == 0 and st["hi_x"][1] == 2000
    np.testing.assert_allclose(st["sd_d"][0], np.sqrt(1 - 1.0 / n ** 2), rtol=1e-12)


def test_in_range_margin():
    lo, hi = np.zeros(17), np.ones(17)
    x = np.full((4, 17), 0.5)
    x[1, 3] = 1.1     # on the 10% margin: inside
    x[2, 16] = -0.11  # beyond it
    x[3, 0] = 1.0
    np.testing.assert_array_equal(S.in_range(x, lo, hi), [True, True, False, True])


def _stats(mu_d=0.0, sd_d=1.0):
    return dict(mu_x=np.zeros(17, np.float32), rs_x=np.ones(17, np.float32),
                mu_d=np.full(13, mu_d, np.float32), sd_d=np.full(13, sd_d, np.float32),
                lo_x=np.full(17, -1e9), hi_x=np.full(17, 1e9))


def test_step_with_constant_output_is_an_affine_update():
    P = _params(10)
    P["W3"][:] = 0.0
    P["b3"][:] = np.linspace(-0.5, 0.5, 13)
    st = _stats(mu_d=0.25, sd_d=0.5)
    rng = np.random.default_rng(11)
    s = rng.standard_normal((6, 13)).astype(np.float32)
    s[:, 3:7] = [1, 0, 0, 0]
    a = rng.uniform(-1, 1, (6, 4))
    sp = S.step(P, st, s, a)
    want = s.astype(np.float64) + 0.5 * P["b3"] + 0.25
    q = want[:, 3:7] / np.linalg.norm(want[:, 3:7], axis=1, keepdims=True)
    np.testing.assert_allclose(sp[:, :3], want[:, :3], rtol=1e-14)
    np.testing.assert_allclose(sp[:, 7:], want[:, 7:], rtol=1e-14)
    np.testing.assert_allclose(sp[:, 3:7], q, rtol=1e-14)


def test_rollout_falls_back_outside_the_trained_range():
    P = _params(12)
    st = _stats()
    st["lo_x"], st["hi_x"] = np.full(17, 5.0), np.full(17, 6.0)  # nothing is inside
    rng = np.random.default_rng(13)
    s0 = rng.standard_normal((3, 13)).astype(np.float32)
    acts = rng.uniform(-1, 1, (4, 3, 4))
    plain = lambda s, a: s + 0.01 * np.concatenate([a, a, a, a[:, :1]], axis=1)
    states, fb = S.rollout(P, st, s0, acts, plain)
    assert fb.all()
    s = s0.astype(np.float64)
    for t in range(4):
        s = plain(s, acts[t].astype(np.float32).astype(np.float64)).astype(np.float32).astype(np.float64)
        np.testing.assert_array_equal(states[t + 1], s)


def test_in_range_unbounded_features_and_zero_margin():
    lo = np.array([-np.inf, 0.0] + [0.0] * 15)
    hi = np.array([np.inf, 1.0] + [1.0] * 15)
    x = np.full((2, 17), 0.5)
    x[1, 1] = 1.0 + 1e-9
    np.testing.assert_array_equal(S.in_range(x, lo, hi, margin=0.0), [True, False])
    np.testing.assert_array_equal(S.in_range(x, lo, hi, margin=0.1), [True, True])
