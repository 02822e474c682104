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


# ---------------------------------------------------------------------------
# Interval form: every result a binary32 evaluation of the same network can
# give.
#
# The network is defined with bfloat16 rounding points (above); a binary32
# evaluation (FP32 accumulation, FP32 transcendental functions) may land a
# pre-rounding value on the other side of a bfloat16 rounding boundary than
# the exact value, which moves everything after it by one bfloat16 ulp.  The
# functions below carry each quantity as a midpoint-radius interval (Rump,
# "Fast and parallel interval arithmetic", BIT 39, 1999) that contains the
# exact FP64 value and every value a binary32 evaluation with these error
# bounds can produce:
#
#   * a chain of n fused multiply-adds or additions in binary32 (any order):
#     error <= gamma_n * sum |terms|, gamma_n = n u / (1 - n u), u = 2^-24
#     (Higham, "Accuracy and Stability of Numerical Algorithms", Sec. 3.1);
#   * a bfloat16 x bfloat16 product accumulated by a tensor core: the
#     products are exact in binary32 and each matrix instruction adds its
#     K = 16 products to the accumulator with an error below 2 u of the sum
#     of the magnitudes it adds; TC_UNIT is that bound per instruction, with
#     a factor 4 of margin;
#   * erfc, exp in binary32: within 4 and 2 units in the last place (the
#     CUDA C Programming Guide's table of single-precision function errors),
#     plus the propagated error of their binary32 argument;
#   * a bfloat16 rounding of an interval [lo, hi] is [bf16(lo), bf16(hi)]
#     (rounding to nearest is monotonic).
#
# The width of a result is zero wherever no rounding boundary lies within
# reach, and one bfloat16 ulp (propagated) where one does: a test can then
# require every binary32 result to lie inside the interval, element by
# element, instead of a blanket tolerance.
# ---------------------------------------------------------------------------

U32 = 2.0 ** -24
TC_UNIT = 8.0 * U32  # per 16-deep tensor-core accumulation step (2 u, x4 margin)
_U64 = 2.0 ** -53


def _gamma(n):
    return n * U32 / (1.0 - n * U32)


def _newton(f, df, x):
    for _ in range(60):
        x = x - f(x) / df(x)
    return x


_PHI = lambda z: _INV_SQRT_2PI * math.exp(-0.5 * z * z)  # noqa: E731
# gelu has one minimum (gelu' = 0 near -0.75); gelu' has extrema at +-sqrt(2)
# (gelu'' = phi(z) (2 - z^2))
_GELU_ARGMIN = _newton(lambda z: 0.5 * math.erfc(-z * _SQRT1_2) + z * _PHI(z),
                       lambda z: _PHI(z) * (2.0 - z * z), -0.75)
_GELUP_CRIT = (-math.sqrt(2.0), math.sqrt(2.0))


class Iv:
    """Midpoint-radius interval array: [mid - rad, mid + rad]."""

    __slots__ = ("mid", "rad")

    def __init__(self, mid, rad=None):
        self.mid = np.asarray(mid, np.float64)
        self.rad = np.zeros_like(self.mid) if rad is None else np.asarray(rad, np.float64)

    @staticmethod
    def from_bounds(lo, hi):
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        return Iv(0.5 * (lo + hi), 0.5 * (hi - lo) * (1.0 + 4 * _U64))

    @property
    def lo(self):
        return self.mid - self.rad

    @property
    def hi(self):
        return self.mid + self.rad

    def mag(self):
        return np.abs(self.mid) + self.rad

    def widen(self, r):
        return Iv(self.mid, self.rad + r)

    def __add__(self, o):
        o = o if isinstance(o, Iv) else Iv(o)
        m = self.mid + o.mid
        return Iv(m, self.rad + o.rad + 2 * _U64 * np.abs(m))

    def __sub__(self, o):
        o = o if isinstance(o, Iv) else Iv(o)
        m = self.mid - o.mid
        return Iv(m, self.rad + o.rad + 2 * _U64 * np.abs(m))

    def __mul__(self, o):
        o = o if isinstance(o, Iv) else Iv(o)
        m = self.mid * o.mid
        r = np.abs(self.mid) * o.rad + self.rad * np.abs(o.mid) + self.rad * o.rad
        return Iv(m, r + 2 * _U64 * np.abs(m))

    def matmul(self, o):
        """self @ o (2-D), radius by Rump's midpoint-radius product."""
        o = o if isinstance(o, Iv) else Iv(o)
        m = self.mid @ o.mid
        r = np.abs(self.mid) @ o.rad + self.rad @ (np.abs(o.mid) + o.rad)
        k = self.mid.shape[-1]
        return Iv(m, r + (k + 2) * _U64 * (np.abs(self.mid) @ np.abs(o.mid)))

    def abs_matmul(self, o):
        """An upper bound of sum |a_ik b_kj| over the intervals (for error bounds)."""
        o = o if isinstance(o, Iv) else Iv(o)
        return self.mag() @ o.mag()


def _round_bf16(x: Iv) -> Iv:
    return Iv.from_bounds(bf16(x.lo), bf16(x.hi))


def _gelu_iv(z: Iv) -> Iv:
    lo_v, hi_v = gelu(z.lo), gelu(z.hi)
    lo = np.minimum(lo_v, hi_v)
    hi = np.maximum(lo_v, hi_v)
    inside = (z.lo < _GELU_ARGMIN) & (z.hi > _GELU_ARGMIN)
    lo = np.where(inside, gelu(np.array(_GELU_ARGMIN)), lo)
    return Iv.from_bounds(lo, hi)


def _gelu_prime_iv(z: Iv) -> Iv:
    lo_v, hi_v = gelu_prime(z.lo), gelu_prime(z.hi)
    lo, hi = np.minimum(lo_v, hi_v), np.maximum(lo_v, hi_v)
    for c in _GELUP_CRIT:
        inside = (z.lo < c) & (z.hi > c)
        v = gelu_prime(np.array(c))
        lo = np.where(inside, np.minimum(lo, v), lo)
        hi = np.where(inside, np.maximum(hi, v), hi)
    return Iv.from_bounds(lo, hi)


def _gelu_f32_err(z: Iv, h: Iv):
    """Bound of the binary32 evaluation error of 0.5 z erfc(-z/sqrt2) at z
    (the argument's own error is carried by z): the constant and the product
    -z/sqrt2 (2 u relative on the argument a), erfc within 4 ulp, the final
    product one rounding; the relative effect of the argument error on erfc
    is |a erfc'(a) / erfc(a)| <= 2 a^2 + 1 for a > 0 and <= 1 for a <= 0."""
    a = np.maximum(0.0, -z.lo * _SQRT1_2)
    return (6.0 + 2.0 * (2.0 * a * a + 1.0)) * U32 * h.mag()


def _gelu_prime_f32_err(z: Iv):
    """Bound of the binary32 error of 0.5 erfc(-z/sqrt2) + z phi(z) with phi
    through expf of the binary32 argument -z^2/2 (relative error 2 u, so
    the exponential moves by (z^2/2)(2 u)), the sum one rounding."""
    zm = np.maximum(np.abs(z.lo), np.abs(z.hi))
    a = np.maximum(0.0, -z.lo * _SQRT1_2)
    t1 = 0.5 * _erfc(-z.mid * _SQRT1_2) * (6.0 + 2.0 * (2.0 * a * a + 1.0)) * U32
    t2 = zm * _INV_SQRT_2PI * np.exp(-0.5 * np.minimum(z.lo * z.lo, z.hi * z.hi)) * (6.0 + zm * zm) * U32
    return 2.0 * (t1 + t2) + U32 * np.abs(gelu_prime(z.mid))


def forward_interval(w, X) -> dict:
    """Intervals of the activations and the output of a batch X (B x 5) for
    any binary32 evaluation (layers 1 and 3 as fused multiply-add chains,
    layer 2 on tensor cores) with the bfloat16 rounding points of forward()."""
    p = unflatten(w)
    W1, W2, W3 = bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    X = np.asarray(X, np.float64)
    # layer 1: b1 + sum_i W1 x_i, 5 fused multiply-adds
    z1 = Iv(X @ W1.T + p["b1"])
    z1 = z1.widen(_gamma(6) * (np.abs(X) @ np.abs(W1).T + np.abs(p["b1"])) + 8 * _U64 * np.abs(z1.mid))
    h1 = _gelu_iv(z1)
    h1 = h1.widen(_gelu_f32_err(z1, h1))
    h1b = _round_bf16(h1)
    # layer 2: tensor-core products of bf16 operands (64 deep: 4 steps) + b2
    z2 = h1b.matmul(Iv(W2.T)) + p["b2"]
    z2 = z2.widen(4 * TC_UNIT * h1b.abs_matmul(Iv(np.abs(W2.T))) + 2 * U32 * (z2.mag() + np.abs(p["b2"])))
    h2 = _gelu_iv(z2)
    h2 = h2.widen(_gelu_f32_err(z2, h2))
    h2b = _round_bf16(h2)
    # layer 3: fused multiply-add chains of 16 terms, combined by 2 additions, + b3
    out = h2b.matmul(Iv(W3.T)) + p["b3"]
    out = out.widen(_gamma(19) * (h2b.abs_matmul(Iv(np.abs(W3.T))) + np.abs(p["b3"])))
    return dict(z1=z1, h1b=h1b, z2=z2, h2b=h2b, out=out)


def grads_interval(w, X, Y, n_seq: int) -> tuple:
    """Intervals of the loss and of the gradient (flat, library layout) of
    loss_and_grads() for any binary32 evaluation with the same rounding
    points, where each sum over the batch is evaluated by at most n_seq
    additions in sequence (per-block partial sums and their sum) and the
    bf16 x bf16 weight gradient dW2 on tensor cores."""
    p = unflatten(w)
    W2, W3 = bf16(p["W2"]), bf16(p["W3"])
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    B = X.shape[0]
    a = forward_interval(w, X)
    out, h1b, h2b, z1, z2 = a["out"], a["h1b"], a["h2b"], a["z1"], a["z2"]
    # dout = (out - Y) * fl(1/B): the subtraction and the product round, and
    # 1/B is itself rounded to binary32
    diff = out - Y
    diff = diff.widen(U32 * diff.mag())
    dout = diff * (1.0 / B)
    dout = dout.widen(3 * U32 * dout.mag())
    loss_terms = diff * diff
    loss = Iv(np.sum(loss_terms.mid) / (2.0 * B),
              (np.sum(loss_terms.rad) + _gamma(n_seq + 2) * np.sum(loss_terms.mag())) / (2.0 * B))
    g = {}
    sabs = lambda A, Bm: A.abs_matmul(Bm)  # noqa: E731
    doutT = Iv(dout.mid.T, dout.rad.T)
    g["W3"] = doutT.matmul(h2b).widen(_gamma(n_seq) * sabs(doutT, h2b))
    g["b3"] = Iv(dout.mid.sum(0), dout.rad.sum(0) + _gamma(n_seq) * dout.mag().sum(0))
    # dz2 = (dout W3) gelu'(z2): two products and a fused multiply-add
    dh2 = dout.matmul(Iv(W3))
    dh2 = dh2.widen(_gamma(2) * dout.abs_matmul(Iv(np.abs(W3))))
    gp2 = _gelu_prime_iv(z2).widen(_gelu_prime_f32_err(z2))
    dz2 = dh2 * gp2
    dz2 = dz2.widen(U32 * dz2.mag())
    dz2b = _round_bf16(dz2)
    # dW2 = bf16(dz2)^T h1b on tensor cores (staged tiles of 64 samples), then
    # the per-block partial sums added in sequence
    dz2bT = Iv(dz2b.mid.T, dz2b.rad.T)
    gW2 = dz2bT.matmul(h1b)
    g["W2"] = gW2.widen((n_seq * TC_UNIT + _gamma(n_seq)) * dz2bT.abs_matmul(h1b))
    g["b2"] = Iv(dz2.mid.sum(0), dz2.rad.sum(0) + _gamma(n_seq) * dz2.mag().sum(0))
    # dz1 = (bf16(dz2) W2) gelu'(z1): tensor-core product, then one rounding
    dh1 = dz2b.matmul(Iv(W2))
    dh1 = dh1.widen(4 * TC_UNIT * dz2b.abs_matmul(Iv(np.abs(W2))))
    gp1 = _gelu_prime_iv(z1).widen(_gelu_prime_f32_err(z1))
    dz1 = dh1 * gp1
    dz1 = dz1.widen(U32 * dz1.mag())
    dz1T = Iv(dz1.mid.T, dz1.rad.T)
    gW1 = dz1T.matmul(Iv(X))
    g["W1"] = gW1.widen(_gamma(n_seq) * dz1T.abs_matmul(Iv(np.abs(X))))
    g["b1"] = Iv(dz1.mid.sum(0), dz1.rad.sum(0) + _gamma(n_seq) * dz1.mag().sum(0))
    mid = flatten({k: v.mid for k, v in g.items()})
    rad = flatten({k: v.rad for k, v in g.items()})
    return loss, Iv(mid, rad)
