"""Oracle of the learned warm start's network: forward pass, loss, gradient, Adam step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain FP64 numpy, written from the
definitions, used to check the library's BF16/FP32 training and inference kernels.

The network maps a scenario's features (relative flue-gas flow and CO2-fraction
perturbations and the diameter) to its 220 stage unknowns and 220 row multipliers:
    a0 = (X - in_shift) / in_scale                          (3 features)
    a_l = gelu(a_{l-1} W_l^T + b_l),  l = 1, 2, 3            (width 256)
    yhat = a3 W4^T + b4                                      (440 outputs, normalised)
    loss = sum((yhat - (Y - out_shift) / out_scale)^2) / (2 n 440)
gelu(x) = x Phi(x) with the standard normal CDF Phi (Hendrycks & Gimpel 2016, exact erf
form).  "BF16 weights": the four weight matrices enter every product rounded to
bfloat16 (round to nearest, ties to even, from FP32 master values); biases,
activations and accumulation stay wide (FP32 on the GPU, FP64 here).  Gradients are
taken with respect to the rounded weights and applied to the masters.
Adam is Algorithm 1 of Kingma & Ba (2015) with bias correction.

Parameter order of the flat vector: W1 (256x3, row-major [out][in]), b1, W2 (256x256),
b2, W3 (256x256), b3, W4 (440x256), b4.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 3, 256, 440
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID),
          (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even); returned as float64.
    bfloat16 keeps the top 16 bits of an IEEE float32 (8 exponent, 7 mantissa bits)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unflatten(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def flatten(tensors):
    return np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in tensors])


def phi_cdf(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0)))


def gelu(x):
    return x * phi_cdf(x)


def gelu_prime(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    return phi_cdf(x) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _weights(theta, bf16):
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    if bf16:
        W1, W2, W3, W4 = (bf16_round(W) for W in (W1, W2, W3, W4))
    return [(W1, b1), (W2, b2), (W3, b3), (W4, b4)]


def forward(theta, X, norm, bf16=True, keep=False):
    """Normalised outputs (n, 440); with keep, also the pre-activations and activations."""
    in_shift, in_scale = norm["in_shift"], norm["in_scale"]
    a = (np.asarray(X, dtype=np.float64) - in_shift) / in_scale
    acts, pre = [a], []
    layers = _weights(theta, bf16)
    for W, b in layers[:3]:
        z = a @ W.T + b
        a = gelu(z)
        pre.append(z)
        acts.append(a)
    W4, b4 = layers[3]
    yhat = a @ W4.T + b4
    return (yhat, pre, acts) if keep else yhat


def predict(theta, X, norm, bf16=True):
    """Raw (denormalised) outputs."""
    return forward(theta, X, norm, bf16) * norm["out_scale"] + norm["out_shift"]


def loss_and_grad(theta, X, Y, norm, bf16=True):
    """Loss and its gradient (flat, parameter order) by reverse-mode differentiation of
    the definitions above."""
    yhat, pre, acts = forward(theta, X, norm, bf16, keep=True)
    t = (np.asarray(Y, dtype=np.float64) - norm["out_shift"]) / norm["out_scale"]
    n = yhat.shape[0]
    r = yhat - t
    loss = float(np.sum(r * r) / (2.0 * n * N_OUT))
    layers = _weights(theta, bf16)
    g = r / (n * N_OUT)                       # dloss / dyhat
    grads = [None] * 8
    grads[6] = g.T @ acts[3]                  # dW4
    grads[7] = g.sum(axis=0)                  # db4
    da = g @ layers[3][0]
    for l in (2, 1, 0):
        dz = da * gelu_prime(pre[l])
        grads[2 * l] = dz.T @ acts[l]         # dW_{l+1}
        grads[2 * l + 1] = dz.sum(axis=0)     # db_{l+1}
        if l > 0:
            da = dz @ layers[l][0]
    return loss, flatten(grads)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
