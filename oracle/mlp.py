"""Plain FP64 reference of the warm-start network (numpy): forward pass, loss, backward
pass and Adam step of a fully connected GELU network.

TEST INFRASTRUCTURE ONLY: the test-suite uses it to check the library's BF16 kernels.  It
shares no code with the CUDA library and never imports it.

Network: x (B x d0) -> u_l = a_{l-1} W_l + b_l, a_l = GELU(u_l) for the hidden layers, and
y = a_{L-1} W_L + b_L for the output (no activation); GELU(u) = u Phi(u) with Phi the
standard normal CDF (the exact form, not the tanh approximation).  Loss: masked mean
squared error L = 1 / (2B) sum_b sum_k mask_bk (y_bk - t_bk)^2.

With ``bf16=True`` the values the GPU kernels store in BF16 are rounded to BF16 (round to
nearest, ties to even) at the same points: the weights, the input, every hidden
activation, the output gradient and every pre-activation gradient; everything else stays
FP64.  The comparison with the kernels then differs only by accumulation order.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.  BF16 keeps the
    top 16 bits of the IEEE single: round the float32 bit pattern at bit 16."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def gelu(u: np.ndarray) -> np.ndarray:
    return 0.5 * u * (1.0 + erf(u / SQRT2))


def gelu_grad(u: np.ndarray) -> np.ndarray:
    """d/du [u Phi(u)] = Phi(u) + u phi(u)."""
    return 0.5 * (1.0 + erf(u / SQRT2)) + u * INV_SQRT_2PI * np.exp(-0.5 * u * u)


def init_params(sizes: List[int], seed: int = 0) -> List[Tuple[np.ndarray, np.ndarray]]:
    """He-style normal weights scaled by sqrt(2 / fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((a, b)) * math.sqrt(2.0 / a), np.zeros(b))
            for a, b in zip(sizes[:-1], sizes[1:])]


def forward(params, x: np.ndarray, bf16: bool = False):
    """Returns (y, cache); cache holds the layer inputs and pre-activations for backward."""
    rnd = bf16_round if bf16 else (lambda v: v)
    a = rnd(np.asarray(x, dtype=np.float64))
    inputs, pre = [], []
    for li, (W, b) in enumerate(params):
        inputs.append(a)
        u = a @ rnd(W) + b
        pre.append(u)
        if li < len(params) - 1:
            a = rnd(gelu(u))
        else:
            a = u
    return a, (inputs, pre)


def loss(y: np.ndarray, t: np.ndarray, mask: np.ndarray) -> float:
    return 0.5 * float(np.sum(mask * (y - t) ** 2)) / y.shape[0]


def backward(params, cache, y: np.ndarray, t: np.ndarray, mask: np.ndarray,
             bf16: bool = False):
    """Gradients [(dW_l, db_l)] of the loss for every layer."""
    rnd = bf16_round if bf16 else (lambda v: v)
    inputs, pre = cache
    B = y.shape[0]
    g = rnd(mask * (y - t) / B)                       # dL/du of the output layer
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (inputs[li].T @ g, g.sum(axis=0))
        if li > 0:
            da = g @ rnd(W).T
            g = rnd(da * gelu_grad(pre[li - 1]))
    return grads


def adam(params, grads, state, lr: float, t: int, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step (bias-corrected), in place; state is a list of (m, v) pairs per
    parameter array, created on first use."""
    flat_p = [p for pair in params for p in pair]
    flat_g = [g for pair in grads for g in pair]
    if not state:
        state.extend((np.zeros_like(p), np.zeros_like(p)) for p in flat_p)
    c1, c2 = 1.0 - beta1 ** t, 1.0 - beta2 ** t
    for p, gr, (m, v) in zip(flat_p, flat_g, state):
        m *= beta1
        m += (1.0 - beta1) * gr
        v *= beta2
        v += (1.0 - beta2) * gr * gr
        p -= lr * (m / c1) / (np.sqrt(v / c2) + eps)
