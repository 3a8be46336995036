"""FP64 oracle of the surrogate network (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU leg may use this
module.  It shares no code with the CUDA kernels.

The surrogate maps run parameters to measured observables of the capillary
model: a fully connected network 6 -> 128 -> 128 -> 128 -> 3 with the exact
(erf) GELU between layers, trained on the mean squared error with Adam.
Parameters are kept in one flat vector in layer order W1, b1, W2, b2, W3, b3,
W4, b4 with W_l stored [in][out] (row-major), so y = x W + b.

``bf16=True`` evaluates the forward and backward products with every GEMM
operand rounded to bfloat16 (round to nearest, ties to even) and exact FP64
sums: the arithmetic the GPU kernels perform, minus their FP32 summation
order.  ``bf16=False`` is the plain FP64 network.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SIZES = (6, 128, 128, 128, 3)


def n_params(sizes=SIZES) -> int:
    return sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))


def unpack(theta: np.ndarray, sizes=SIZES):
    """Views (W_l, b_l) into the flat parameter vector."""
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bias = theta[o:o + b]
        o += b
        out.append((W, bias))
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z: np.ndarray) -> np.ndarray:
    """GELU(z) = z Phi(z) with the exact Gaussian CDF."""
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(seed: int, sizes=SIZES) -> np.ndarray:
    """Uniform(-1/sqrt(in), 1/sqrt(in)) weights, zero biases (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / np.sqrt(a)
        parts.append(rng.uniform(-lim, lim, size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = False):
    """Returns (Y, cache) where cache holds the layer inputs and pre-activations."""
    r = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(np.asarray(theta, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    ins, zs = [], []
    for li, (W, b) in enumerate(layers):
        a = r(h)
        z = a @ r(W) + b
        ins.append(a)
        zs.append(z)
        h = gelu(z) if li < len(layers) - 1 else z
    return h, {"ins": ins, "zs": zs}


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf16: bool = False) -> float:
    Y, _ = forward(theta, X, bf16)
    return float(np.mean((Y - T) ** 2))


def backward(theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf16: bool = False):
    """(loss, gradient) of the mean squared error over batch and outputs."""
    r = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack(np.asarray(theta, dtype=np.float64))
    Y, cache = forward(theta, X, bf16)
    n = X.shape[0]
    dz = 2.0 * (Y - T) / (n * Y.shape[1])
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a = cache["ins"][li]
        gW = a.T @ r(dz)
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            dh = r(dz) @ r(W).T
            dz = dh * gelu_grad(cache["zs"][li - 1])
    grads.reverse()
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return float(np.mean((Y - T) ** 2)), g


def adam(theta, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
