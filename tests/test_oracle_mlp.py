"""Pins of the FP64 reference of the warm-start network (oracle/mlp.py): BF16 rounding,
GELU and its derivative, backward against finite differences and a closed form, the Adam
step.  CPU only."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_bf16_rounding_is_round_to_nearest_even_on_the_top_16_bits():
    ulp = 2.0 ** -7                                   # spacing of BF16 just above 1
    vals = np.array([1.0, 1.0 + ulp / 2, 1.0 + 3 * ulp / 2, 1.0 + ulp / 4, -2.5, 3.0e38])
    # 3e38 is 0x7F61B1E6 as a float32: the low half 0xB1E6 rounds the top half up
    big = float(np.array([0x7F620000], dtype=np.uint32).view(np.float32)[0])
    want = np.array([1.0, 1.0, 1.0 + 2 * ulp, 1.0, -2.5, big])
    got = mlp.bf16_round(vals)
    assert np.array_equal(got, want)
    assert np.isnan(mlp.bf16_round(np.array([np.nan]))[0])


def test_gelu_is_u_times_the_normal_cdf_and_its_derivative():
    u = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(u), u * norm.cdf(u), rtol=1e-13, atol=1e-15)
    assert math.isclose(mlp.gelu(np.array([1.0]))[0], 0.8413447460685429, rel_tol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(u), fd, rtol=1e-7, atol=1e-9)


def _problem(seed=0, B=6, sizes=(5, 7, 6, 4, 3)):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(list(sizes), seed=seed)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((B, sizes[0]))
    t = rng.standard_normal((B, sizes[-1]))
    mask = (rng.random((B, sizes[-1])) < 0.8).astype(float)
    return params, x, t, mask


def test_backward_matches_central_finite_differences():
    params, x, t, mask = _problem()
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t, mask)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.loss(mlp.forward(params, x)[0], t, mask)
                arr[idx] = old - h
                lm = mlp.loss(mlp.forward(params, x)[0], t, mask)
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_output_bias_gradient_closed_form():
    """dL/db_L = (1/B) sum_b mask_b (y_b - t_b), whatever the hidden layers."""
    params, x, t, mask = _problem(seed=3)
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t, mask)
    assert np.allclose(grads[-1][1], (mask * (y - t)).sum(axis=0) / x.shape[0], rtol=1e-14)


def test_first_adam_step_moves_each_weight_by_lr_times_sign_of_its_gradient():
    params, x, t, mask = _problem(seed=4)
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t, mask)
    before = [p.copy() for pair in params for p in pair]
    state = []
    mlp.adam(params, grads, state, lr=1e-3, t=1, eps=0.0)
    after = [p for pair in params for p in pair]
    flat_g = [g for pair in grads for g in pair]
    for p0, p1, g in zip(before, after, flat_g):
        nz = g != 0
        assert np.allclose((p0 - p1)[nz], 1e-3 * np.sign(g[nz]), rtol=1e-12)


def test_bf16_mode_rounds_only_the_stored_values():
    params, x, t, mask = _problem(seed=5)
    y64, _ = mlp.forward(params, x)
    y16, cache = mlp.forward(params, x, bf16=True)
    assert not np.allclose(y64, y16, rtol=1e-6)            # rounding happened
    assert np.allclose(y64, y16, rtol=5e-2, atol=5e-2)      # ... at BF16 precision only
    for a in cache[0]:
        assert np.array_equal(a, mlp.bf16_round(a))        # stored inputs are BF16 values
