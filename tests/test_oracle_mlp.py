"""Pins of the warm-start MLP oracle (oracle/mlp.py) against things other than itself:
central finite differences of the loss, closed forms of silu and of special networks,
the first Adam step, and bfloat16 roundings fixed by the format."""
import numpy as np
import pytest

from oracle import mlp


def small_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    u = {"W1": rng.random((mlp.WIDTH, mlp.N_IN)), "W2": rng.random((mlp.WIDTH, mlp.WIDTH)),
         "W3": rng.random((mlp.WIDTH, mlp.WIDTH)), "w4": rng.random(mlp.WIDTH)}
    P = mlp.init_params(u)
    for k in ("b1", "b2", "b3"):
        P[k] = 0.1 * scale * (rng.random(mlp.WIDTH) - 0.5)
    P["b4"] = np.array([0.3])
    return P


def test_silu_closed_forms():
    assert mlp.silu(0.0) == 0.0
    assert mlp.dsilu(0.0) == 0.5
    assert mlp.silu(40.0) == pytest.approx(40.0, rel=1e-15)
    assert abs(mlp.silu(-40.0)) < 1e-15
    # d/dz silu at z = ln(3): s = 3/4, silu' = 3/4 (1 + ln 3 / 4)
    z = np.log(3.0)
    assert mlp.dsilu(z) == pytest.approx(0.75 * (1.0 + z / 4.0), rel=1e-15)
    zs = np.linspace(-6, 6, 25)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(zs), (mlp.silu(zs + h) - mlp.silu(zs - h)) / (2 * h), rtol=1e-8, atol=1e-10)


def test_bf16_rounding_follows_the_format():
    # 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1)
    assert mlp.to_bf16(1.0 + 2.0**-8) == 1.0
    assert mlp.to_bf16(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6  # tie -> even mantissa
    assert mlp.to_bf16(1.0 + 2.0**-8 + 2.0**-12) == 1.0 + 2.0**-7
    assert mlp.to_bf16(-3.0) == -3.0
    assert mlp.to_bf16(0.1) == pytest.approx(0.1, rel=2.0**-9)
    v = np.random.default_rng(1).normal(size=1000)
    r = mlp.to_bf16(v)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0**-8)
    # idempotent and exact on values with 8 significant bits
    np.testing.assert_array_equal(mlp.to_bf16(r), r)


def test_gradients_match_central_differences():
    P = small_params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(12, mlp.N_IN))
    t = rng.normal(size=12)
    _, g = mlp.loss_and_grads(x, t, P)
    h = 1e-6
    for k, idx in [("W1", (3, 2)), ("W1", (100, 4)), ("b1", (7,)), ("W2", (5, 9)), ("W2", (127, 0)),
                   ("b2", (64,)), ("W3", (1, 120)), ("b3", (33,)), ("w4", (17,)), ("b4", (0,))]:
        Pp = {kk: vv.copy() for kk, vv in P.items()}
        Pm = {kk: vv.copy() for kk, vv in P.items()}
        Pp[k][idx] += h
        Pm[k][idx] -= h
        fd = (mlp.loss_and_grads(x, t, Pp)[0] - mlp.loss_and_grads(x, t, Pm)[0]) / (2 * h)
        assert g[k][idx] == pytest.approx(fd, rel=1e-6, abs=1e-11), (k, idx)


def test_network_with_zero_hidden_weights_is_constant():
    """W2 = W3 = 0: y = silu(b3) . w4 + b4 for every input, and only b3, w4, b4, W3 get
    a gradient (dZ2 = 0 because W3 = 0)."""
    P = small_params(5)
    P["W2"][:] = 0.0
    P["W3"][:] = 0.0
    x = np.random.default_rng(6).normal(size=(9, mlp.N_IN))
    y, _ = mlp.forward(x, P)
    want = float(np.dot(mlp.silu(P["b3"]), P["w4"]) + P["b4"][0])
    np.testing.assert_allclose(y, want, rtol=1e-14)
    t = np.zeros(9)
    _, g = mlp.loss_and_grads(x, t, P)
    assert g["b4"][0] == pytest.approx(2.0 * want, rel=1e-14)  # d mean((y-0)^2)/d b4 = 2 y
    assert np.all(g["W1"] == 0) and np.all(g["b1"] == 0) and np.all(g["W2"] == 0)


def test_first_adam_step_is_lr_times_sign():
    """Step 1: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)."""
    P = {"a": np.array([1.0, -2.0, 0.5]), "b": np.array([0.0])}
    g = {"a": np.array([0.3, -1e-3, 0.0]), "b": np.array([5.0])}
    z = {k: np.zeros_like(v) for k, v in P.items()}
    P1, m1, v1 = mlp.adam_step(P, g, z, z, 1, lr=0.01)
    np.testing.assert_allclose(P1["a"], P["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(P1["b"], [-0.01 * 5.0 / (5.0 + 1e-8)], rtol=1e-15)
    np.testing.assert_allclose(m1["a"], 0.1 * g["a"])
    np.testing.assert_allclose(v1["a"], 0.001 * g["a"] ** 2)


def test_bf16_mode_stays_close_to_fp64():
    """The mixed-precision reading changes the gradient by bfloat16 rounding only
    (a few 2^-8 relative in norm)."""
    P = small_params(7)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(64, mlp.N_IN))
    t = rng.normal(size=64)
    l64, g64 = mlp.loss_and_grads(x, t, P)
    l16, g16 = mlp.loss_and_grads(x, t, P, bf16=True)
    assert l16 == pytest.approx(l64, rel=0.02)
    for k in g64:
        assert np.linalg.norm(g16[k] - g64[k]) <= 0.03 * np.linalg.norm(g64[k]) + 1e-12, k


def test_training_by_the_oracle_fits_a_smooth_profile():
    """A few hundred full-batch Adam steps fit a tanh profile of z/H: the loss drops by
    two orders of magnitude (the network can represent the target family)."""
    rng = np.random.default_rng(9)
    n = 256
    raw = np.column_stack([np.full(n, 0.8), np.full(n, -5.0), np.ones(n), np.full(n, 1.4), rng.random(n),
                           np.full(n, 7.0)])
    t = 1.3 - 1.1 * np.tanh(10.0 * (raw[:, 4] - 0.5))
    x = mlp.normalise(raw)
    P = small_params(10, scale=0.0)
    m = {k: np.zeros_like(v) for k, v in P.items()}
    v = {k: np.zeros_like(v) for k, v in P.items()}
    l0 = mlp.loss_and_grads(x, t, P)[0]
    for it in range(1, 301):
        loss, g = mlp.loss_and_grads(x, t, P)
        P, m, v = mlp.adam_step(P, g, m, v, it, lr=3e-3)
    assert loss < 1e-2 * l0
