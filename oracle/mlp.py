"""Reference network of the learned stepper: plain numpy, FP64.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU leg may use it; the CUDA library never calls it and shares
nothing with it.

The learned stepper corrects one macro step of the improved ETD scheme
(Algorithm ETDFSSModAlgo) with a small multilayer perceptron; the paper has
no learned component, so this file defines the network the CUDA kernels
must compute:

    x   = (r, v, sin(t/eps), cos(t/eps), dt)                   (5 inputs)
    z1  = W1 x + b1,  h1 = gelu(z1)                             (64)
    z2  = W2 bf16(h1) + b2,  h2 = gelu(z2)                      (64)
    out = W3 bf16(h2) + b3                                      (2: dR, dV)

with gelu(u) = u (1 + erf(u / sqrt 2)) / 2, W1, W2, W3 rounded to bfloat16
(round to nearest even) and everything else in higher precision.  The loss of
a batch of B samples with targets y is sum((out - y)^2) / (2B).  Backward,
with the same rounding points as the forward pass and one more (the
tensor-core GEMMs of the hidden layer take bfloat16 operands):

    dout = (out - y) / B
    dW3  = dout^T bf16(h2),      db3 = sum dout
    dz2  = (dout W3) * gelu'(z2)
    dW2  = bf16(dz2)^T bf16(h1), db2 = sum dz2
    dz1  = (bf16(dz2) W2) * gelu'(z1)
    dW1  = dz1^T x,              db1 = sum dz1

`emulate_bf16=False` drops every rounding: the exact FP64 network, whose
gradients the tests pin against central finite differences of its loss.

Parameters travel as one flat float32 vector (the library's layout):
W1 (64 x 5, row-major) | b1 (64) | W2 (64 x 64) | b2 (64) | W3 (2 x 64) | b3 (2).
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 5, 64, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_SQRT1_2 = 1.0 / math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def unflatten(w) -> dict:
    w = np.asarray(w, dtype=np.float64).ravel()
    assert w.size == N_PARAMS
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = w[k:k + n].reshape(shape)
        k += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    Rounds the FP64 value directly (8 significant bits), so a float32 input
    is rounded exactly as a float32 -> bfloat16 conversion rounds it."""
    x = np.asarray(x, dtype=np.float64)
    b = x.view(np.uint64).copy()
    drop = np.uint64(45)  # 52 - 7 mantissa bits
    lsb = (b >> drop) & np.uint64(1)
    b = b + (np.uint64((1 << 44) - 1) + lsb)  # half an ulp of the result, minus one, plus the kept lsb
    b &= ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


def _erfc(u):
    return np.vectorize(math.erfc, otypes=[np.float64])(u)


def gelu(u):
    # u (1 + erf(u / sqrt 2)) / 2, written with erfc(-u / sqrt 2) = 1 + erf(u / sqrt 2)
    # so that no cancellation occurs for negative u
    return 0.5 * u * _erfc(-u * _SQRT1_2)


def gelu_prime(u):
    return 0.5 * _erfc(-u * _SQRT1_2) + u * _INV_SQRT_2PI * np.exp(-0.5 * u * u)


def _weights(p: dict, emulate_bf16: bool):
    if emulate_bf16:
        return bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    return p["W1"], p["W2"], p["W3"]


def forward(w, X, emulate_bf16: bool = True) -> dict:
    """Activations of a batch X (B x 5)."""
    p = unflatten(w)
    W1, W2, W3 = _weights(p, emulate_bf16)
    r = bf16 if emulate_bf16 else (lambda a: a)
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + p["b1"]
    h1 = gelu(z1)
    h1b = r(h1)
    z2 = h1b @ W2.T + p["b2"]
    h2 = gelu(z2)
    h2b = r(h2)
    out = h2b @ W3.T + p["b3"]
    return dict(z1=z1, h1b=h1b, z2=z2, h2b=h2b, out=out)


def loss_and_grads(w, X, Y, emulate_bf16: bool = True):
    """Loss sum((out - Y)^2) / (2B) and its gradient (flat, library layout)."""
    p = unflatten(w)
    W1, W2, W3 = _weights(p, emulate_bf16)
    r = bf16 if emulate_bf16 else (lambda a: a)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    B = X.shape[0]
    a = forward(w, X, emulate_bf16)
    diff = a["out"] - Y
    loss = float(np.sum(diff * diff)) / (2.0 * B)
    dout = diff / B
    g = {}
    g["W3"] = dout.T @ a["h2b"]
    g["b3"] = dout.sum(axis=0)
    dz2 = (dout @ W3) * gelu_prime(a["z2"])
    dz2b = r(dz2)
    g["W2"] = dz2b.T @ a["h1b"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2b @ W2) * gelu_prime(a["z1"])
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, flatten(g)
