"""CPU oracle of the learned start-vector network (test infrastructure only).

Not from the paper: a small multilayer perceptron maps the 2L occupation bits
of a basis state (spin-down string in bits 0..L-1, spin-up string in bits
L..2L-1, the combined-integer layout of Sec. III) to (log|psi|, sign logit):

    z1 = W1 x + b1,  a1 = gelu(z1),  z2 = W2 a1 + b2,  a2 = gelu(z2),  out = W3 a2 + b3

with gelu in its tanh form, gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
(Hendrycks & Gimpel, "Gaussian Error Linear Units", 2016).  The GPU stores weights in
bfloat16 and accumulates in float32; this oracle evaluates in float64 with the
same quantities rounded to bfloat16 where the GPU rounds them (weights W1, W2,
W3 and the hidden activation a1 fed to the second matrix product), bfloat16
rounding being round-to-nearest-even of the float32 value.

Loss of a sample with target log-amplitude t, target sign s in {-1, +1} and
weight w (the tests and the training use w = |psi|^2-proportional sampling):
    w * [ (out0 - t)^2 + lam * softplus(-s * out1) ] / sum(w).
"""
from __future__ import annotations

import math

import numpy as np

SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)
GELU_CUBIC = 0.044715


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    nan = np.isnan(f)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(x):
    """The tanh form of GELU (the network's activation)."""
    return 0.5 * x * (1.0 + np.tanh(SQRT_2_OVER_PI * (x + GELU_CUBIC * x ** 3)))


def gelu_grad(x):
    """d gelu / dx of the same form."""
    th = np.tanh(SQRT_2_OVER_PI * (x + GELU_CUBIC * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * SQRT_2_OVER_PI * (1.0 + 3.0 * GELU_CUBIC * x * x)


def bits_of(states: np.ndarray, L: int) -> np.ndarray:
    """Occupation bits of combined integers (up << L) | dn as a (n, 2L) 0/1 array, bit i -> column i."""
    s = np.asarray(states, dtype=np.uint64)
    cols = [((s >> np.uint64(i)) & np.uint64(1)).astype(np.float64) for i in range(2 * L)]
    return np.stack(cols, axis=1)


def unpack(theta: np.ndarray, n_in: int, hidden: int):
    """Flat parameter vector -> (W1 [h,n_in], b1 [h], W2 [h,h], b2 [h], W3 [2,h], b3 [2])."""
    o = 0
    out = []
    for shape in ((hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (2, hidden), (2,)):
        n = int(np.prod(shape))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    return out


def forward(theta, x, n_in, hidden, emulate_bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden)
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    z1 = x @ r(W1).T + b1
    a1 = gelu(z1)
    a1r = r(a1)
    z2 = a1r @ r(W2).T + b2
    a2 = gelu(z2)
    out = a2 @ r(W3).T + b3
    return out, (z1, a1, a1r, z2, a2)


def loss_and_grad(theta, x, t_log, t_sign, w, n_in, hidden, lam=1.0, emulate_bf16=True):
    """Loss and its gradient w.r.t. the flat parameters (straight-through for the bf16 roundings)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden)
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    out, (z1, a1, a1r, z2, a2) = forward(theta, x, n_in, hidden, emulate_bf16)
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    e = out[:, 0] - t_log
    m = -t_sign * out[:, 1]
    sp = np.logaddexp(0.0, m)
    loss = float(np.sum(wn * (e * e + lam * sp)))
    d_out = np.zeros_like(out)
    d_out[:, 0] = wn * 2.0 * e
    d_out[:, 1] = wn * lam * (-t_sign) / (1.0 + np.exp(-m))
    gW3 = d_out.T @ a2
    gb3 = d_out.sum(axis=0)
    d_a2 = d_out @ r(W3)
    d_z2 = d_a2 * gelu_grad(z2)
    gW2 = d_z2.T @ a1r
    gb2 = d_z2.sum(axis=0)
    d_a1 = d_z2 @ r(W2)
    d_z1 = d_a1 * gelu_grad(z1)
    gW1 = d_z1.T @ x
    gb1 = d_z1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
