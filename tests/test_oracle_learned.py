"""Pins of the FP64 network oracle (learned multigrid correction): finite-difference
gradients, delta-kernel identities, a brute-force loop on a tiny grid, BF16 rounding."""
import itertools

import numpy as np
import pytest

from oracle import learned as N


def small_params(seed=1, ch=3):
    p = N.init_params(seed, ch=ch)
    rng = np.random.default_rng(seed + 10)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    return p


def test_single_layer_equals_brute_force_loops():
    n = 4
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, n, n, n))
    W = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    got = N.conv(a, W, b)
    want = np.zeros((3, n, n, n))
    for o, z, y, x in itertools.product(range(3), range(n), range(n), range(n)):
        acc = b[o]
        for t, (dz, dy, dx) in enumerate(N.TAPS):
            zz, yy, xx = z + dz, y + dy, x + dx
            if 0 <= zz < n and 0 <= yy < n and 0 <= xx < n:
                acc += sum(W[o, t, c] * a[c, zz, yy, xx] for c in range(2))
        want[o, z, y, x] = acc
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_delta_kernels_reduce_the_network_to_relu():
    n, ch = 5, 4
    p = {k: np.zeros_like(v) for k, v in N.init_params(0, ch=ch).items()}
    c = N.TAPS.index((0, 0, 0))
    p["W1"][0, c, 0] = 1.0
    p["W2"][0, c, 0] = 1.0
    p["W3"][0, c, 0] = 2.0
    x = np.random.default_rng(3).standard_normal((n, n, n))
    y, _ = N.forward(p, x)
    np.testing.assert_allclose(y, 2.0 * np.maximum(x, 0.0), atol=0)


def test_zero_padding_on_a_constant_field():
    n = 4
    a = np.ones((1, n, n, n))
    W = np.ones((1, 27, 1))
    out = N.conv(a, W, np.zeros(1))[0]
    # each output counts the in-grid neighbours: 27 inside, 8 at a corner, 12 on an edge
    assert out[1, 1, 1] == 27 and out[0, 0, 0] == 8 and out[0, 0, 1] == 12 and out[0, 1, 1] == 18


def test_input_gradient_is_the_adjoint():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 5, 5, 5))
    g = rng.standard_normal((3, 5, 5, 5))
    W = rng.standard_normal((3, 27, 2))
    lhs = float((g * N.conv(a, W, np.zeros(3))).sum())
    rhs = float((N.conv_input_grad(g, W) * a).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_parameter_gradients_match_central_differences():
    p = small_params()
    rng = np.random.default_rng(7)
    xs = [rng.standard_normal((5, 5, 5)) for _ in range(2)]
    ts = [rng.standard_normal((5, 5, 5)) for _ in range(2)]
    L0, g = N.loss_and_grads(p, xs, ts)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            Lp, _ = N.loss_and_grads(p, xs, ts)
            flat[i] = old - eps
            Lm, _ = N.loss_and_grads(p, xs, ts)
            flat[i] = old
            fd = (Lp - Lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (k, i, fd, an)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, -3.14159265, 1e-30, 0.0])
    r = N.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7      # ties to even
    assert abs(r[3] - (-3.140625)) < 1e-12 and r[5] == 0.0
    assert np.all(np.abs(r - v) <= 2 ** -8 * np.abs(v) + 1e-38)


def test_ahat_on_a_sine_mode_is_its_eigenvalue():
    n, kap = 9, 0.13
    h = 1.0 / (n + 1)
    k = (1, 3, 2)
    i = np.arange(1, n + 1) * h
    v = (np.sin(k[0] * np.pi * i)[:, None, None] * np.sin(k[1] * np.pi * i)[None, :, None]
         * np.sin(k[2] * np.pi * i)[None, None, :])
    lam = 1.0 - 2.0 * kap * sum(np.cos(kk * np.pi * h) for kk in k)
    np.testing.assert_allclose(N.apply_ahat(v, kap), lam * v, atol=1e-13)


def test_ahat_is_symmetric():
    rng = np.random.default_rng(8)
    a, b = rng.standard_normal((2, 6, 6, 6))
    lhs = float((b * N.apply_ahat(a, 0.15)).sum())
    rhs = float((N.apply_ahat(b, 0.15) * a).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_operator_norm_loss_gradients_match_central_differences():
    p = small_params(seed=2)
    rng = np.random.default_rng(9)
    xs = [rng.standard_normal((5, 5, 5)) for _ in range(2)]
    ts = [rng.standard_normal((5, 5, 5)) for _ in range(2)]
    kaps = [0.1, 1.0 / 6.0]
    _, g = N.loss_and_grads(p, xs, ts, kaps)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + eps
            Lp, _ = N.loss_and_grads(p, xs, ts, kaps)
            flat[i] = old - eps
            Lm, _ = N.loss_and_grads(p, xs, ts, kaps)
            flat[i] = old
            fd = (Lp - Lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (k, i, fd, an)


def test_operator_norm_loss_is_the_scaled_residual_after_the_correction():
    # with x = Ahat t the loss equals 0.5 mean((x - Ahat y)^2): the residual left by y
    p = small_params(seed=3)
    rng = np.random.default_rng(10)
    t = rng.standard_normal((5, 5, 5))
    kap = 0.12
    x = N.apply_ahat(t, kap)
    L, _ = N.loss_and_grads(p, [x], [t], [kap])
    y, _ = N.forward(p, x)
    r = x - N.apply_ahat(y, kap)
    assert abs(L - 0.5 * float((r * r).mean())) < 1e-13


@pytest.mark.parametrize("power", [0, 2, 3])
def test_loss_powers_match_central_differences(power):
    p = small_params(seed=4)
    rng = np.random.default_rng(11)
    xs = [rng.standard_normal((5, 5, 5))]
    ts = [rng.standard_normal((5, 5, 5))]
    kaps = [0.14]
    _, g = N.loss_and_grads(p, xs, ts, kaps, power)
    eps = 1e-6
    for k in ("W1", "W2", "b3"):
        flat = p[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + eps
            Lp, _ = N.loss_and_grads(p, xs, ts, kaps, power)
            flat[i] = old - eps
            Lm, _ = N.loss_and_grads(p, xs, ts, kaps, power)
            flat[i] = old
            fd = (Lp - Lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (k, i, fd, an)


def test_loss_power_two_weights_a_mode_by_its_squared_eigenvalue():
    # a single sine mode as the error y - t (y = 0 with zero weights): the loss is
    # 0.5 lambda^(2p) mean(t^2), lambda the mode's eigenvalue of Ahat
    n, kap = 7, 0.15
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1) * h
    k = (5, 6, 7)
    t = (np.sin(k[0] * np.pi * i)[:, None, None] * np.sin(k[1] * np.pi * i)[None, :, None]
         * np.sin(k[2] * np.pi * i)[None, None, :])
    lam = 1.0 - 2.0 * kap * sum(np.cos(kk * np.pi * h) for kk in k)
    p = {kk: np.zeros_like(v) for kk, v in N.init_params(0).items()}
    for power in (0, 1, 2):
        L, _ = N.loss_and_grads(p, [np.zeros_like(t)], [t], [kap], power)
        assert abs(L - 0.5 * lam ** (2 * power) * float((t * t).mean())) < 1e-14
