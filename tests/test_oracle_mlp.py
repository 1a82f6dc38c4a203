"""Pins of the network oracle (oracle/mlp.py) against closed forms and finite
differences, independent of the oracle's own backward pass."""
import math

import numpy as np

from oracle import mlp


def _norm(rng):
    return dict(in_shift=rng.normal(0, 0.1, mlp.N_IN), in_scale=rng.uniform(0.5, 2.0, mlp.N_IN),
                out_shift=rng.normal(0, 1, mlp.N_OUT), out_scale=rng.uniform(0.5, 2.0, mlp.N_OUT))


def _theta(rng, scale=1.0):
    parts = []
    for s in mlp.SHAPES:
        fan_in = s[1] if len(s) == 2 else 1
        parts.append(rng.normal(0, scale / math.sqrt(fan_in), s))
    return mlp.flatten(parts)


def test_bf16_rounding():
    one = 1.0
    assert mlp.bf16_round(np.array([one]))[0] == 1.0
    # spacing of bfloat16 at 1 is 2^-7; halfway cases round to the even mantissa
    assert mlp.bf16_round(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16_round(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    assert mlp.bf16_round(np.array([1 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1 + 2.0 ** -7
    assert mlp.bf16_round(np.array([-1.5]))[0] == -1.5
    x = np.random.default_rng(0).normal(0, 10, 10000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))   # unit roundoff of an 8-bit significand
    assert np.all(r.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


def test_gelu_closed_forms():
    # gelu(x) = x Phi(x): Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) <= 1e-15
    assert abs(mlp.gelu(np.array(-1.0)) + 0.15865525393145707) <= 1e-15
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu_prime(np.array(0.0)) - 0.5) <= 1e-16
    x = np.linspace(-6, 6, 97)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_prime(x))) <= 1e-9
    assert abs(mlp.gelu(np.array(40.0)) - 40.0) <= 1e-12 and abs(mlp.gelu(np.array(-40.0))) <= 1e-12


def test_zero_weights_output_is_bias():
    rng = np.random.default_rng(1)
    th = _theta(rng)
    W = mlp.unflatten(th)
    for k in (0, 2, 4, 6):
        W[k][:] = 0.0
    th = mlp.flatten(W)
    X = rng.normal(0, 1, (7, mlp.N_IN))
    norm = _norm(rng)
    y = mlp.forward(th, X, norm)
    assert np.array_equal(y, np.broadcast_to(W[7], y.shape))
    # closed-form gradient: dW4 = (sum_i r_i) outer gelu(b3); db4 = sum_i r_i
    Y = rng.normal(0, 1, (7, mlp.N_OUT))
    loss, g = mlp.loss_and_grad(th, X, Y, norm)
    G = mlp.unflatten(g)
    t = (Y - norm["out_shift"]) / norm["out_scale"]
    r = (W[7] - t) / (7 * mlp.N_OUT)
    assert np.allclose(G[7], r.sum(axis=0), rtol=1e-13, atol=0)
    a3 = mlp.gelu(W[5])
    assert np.allclose(G[6], np.outer(r.sum(axis=0), a3), rtol=1e-12, atol=1e-300)
    assert abs(loss - np.sum((W[7] - t) ** 2) / (2 * 7 * mlp.N_OUT)) <= 1e-14 * loss


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    th = _theta(rng)
    X = rng.normal(0, 1, (5, mlp.N_IN))
    Y = rng.normal(0, 1, (5, mlp.N_OUT))
    norm = _norm(rng)
    _, g = mlp.loss_and_grad(th, X, Y, norm, bf16=False)
    # sampled entries of every tensor (weights and biases of all four layers)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    idx = np.concatenate([rng.choice(np.arange(offs[k], offs[k + 1]), 6, replace=False) for k in range(8)])
    h = 1e-5
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = mlp.loss_and_grad(tp, X, Y, norm, bf16=False)
        lm, _ = mlp.loss_and_grad(tm, X, Y, norm, bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1e-3, np.abs(g).max()), (i, fd, g[i])


def test_bf16_forward_uses_rounded_weights():
    rng = np.random.default_rng(3)
    th = _theta(rng).astype(np.float32).astype(np.float64)
    W = mlp.unflatten(th)
    Wr = [mlp.bf16_round(w) if k % 2 == 0 else w for k, w in enumerate(W)]
    X = rng.normal(0, 1, (4, mlp.N_IN))
    norm = _norm(rng)
    assert np.array_equal(mlp.forward(th, X, norm, bf16=True), mlp.forward(mlp.flatten(Wr), X, norm, bf16=False))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    th = rng.normal(0, 1, 100)
    g = rng.normal(0, 1, 100)
    m = np.zeros(100)
    v = np.zeros(100)
    th1, m1, v1 = mlp.adam_step(th, g, m, v, 1, 1e-3)
    # with zero moments the bias-corrected step is lr * g / (|g| + eps)
    assert np.allclose(th1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    # second step with the same gradient: mhat = g, vhat = g^2 again
    th2, _, _ = mlp.adam_step(th1, g, m1, v1, 2, 1e-3)
    assert np.allclose(th2, th1 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_param_count():
    # 3 -> 256 -> 256 -> 256 -> 440 with biases
    assert mlp.N_PARAMS == 3 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 440 + 440 == 245688


def test_single_path_network_closed_form():
    # one unit per layer carries input feature 0 through three GELUs to output 0; every
    # other output is its bias; predict() undoes the output normalisation
    rng = np.random.default_rng(5)
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[0][0, 0] = W[2][0, 0] = W[4][0, 0] = W[6][0, 0] = 1.0
    W[7][:] = rng.normal(0, 1, mlp.N_OUT)
    W[7][0] = 0.0
    th = mlp.flatten(W)
    norm = _norm(rng)
    X = rng.normal(0, 1, (3, mlp.N_IN))

    def g(x):
        return x * 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))

    y = mlp.predict(th, X, norm)
    for i in range(3):
        x0 = (X[i, 0] - norm["in_shift"][0]) / norm["in_scale"][0]
        assert abs(y[i, 0] - (g(g(g(x0))) * norm["out_scale"][0] + norm["out_shift"][0])) <= 1e-14 * (1 + abs(y[i, 0]))
        np.testing.assert_allclose(y[i, 1:], W[7][1:] * norm["out_scale"][1:] + norm["out_shift"][1:], rtol=1e-15)
