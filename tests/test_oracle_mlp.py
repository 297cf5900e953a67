"""Pins for the learned proposal's FP64 network oracle (oracle/mlp.py).

* The hand-written backpropagation equals central finite differences of the
  loss (FP64, no BF16 rounding), parameter by parameter on a sample.
* GELU (tanh form): g(0) = 0, g(x) -> x for large x, g(-x) = g(x) - x; its
  derivative matches finite differences; g'(0) = 1/2 and g''(0) = sqrt(2/pi),
  as for x Phi(x); the x^4 coefficient of its Taylor series,
  k0 (k1 - k0^2 / 3) / 2, pins k1; and it stays within 5e-4 of x Phi(x)
  (scipy's erf) on [-12, 12] (the form's known accuracy, about 4.7e-4).
* bf16 rounding: exact values stay, ties go to even, the relative error is
  at most 2^-8 (7 stored fraction bits: half an ulp).
* The NLL of a standard-normal residual with zero output equals
  sum r^2 / 2 (the log-scale term vanishes), and its minimiser over a
  constant output is the sample mean / log standard deviation.
* Adam's first step moves every parameter by lr * sign(grad) (bias
  correction makes m/sqrt(v) = +-1).
"""
import math

import numpy as np
import pytest

from oracle import mlp


def _data(B=7, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (B, mlp.IN))
    R = rng.normal(0.0, 1.0, (B, 2))
    return X, R


def test_backprop_matches_finite_differences():
    theta = mlp.init_params(1, out_scale=0.5) + 0.01 * np.random.default_rng(2).normal(size=mlp.N_PARAMS)
    X, R = _data()
    _, g = mlp.loss_and_grad(theta, X, R)
    rng = np.random.default_rng(3)
    sample = rng.choice(mlp.N_PARAMS, size=120, replace=False)
    # include every block's first entry (W1, b1, W2, b2, W3, b3)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp._SHAPES])[:-1]
    for k in list(sample) + list(offs):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, X, R)[0] - mlp.loss_and_grad(tm, X, R)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-8), k


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    x = np.linspace(-4, 4, 41)
    assert np.allclose(mlp.gelu(-x), mlp.gelu(x) - x, atol=1e-15)
    assert mlp.gelu(np.array([30.0]))[0] == 30.0
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_gelu_tanh_form_against_x_phi():
    from scipy.special import erf
    k0 = math.sqrt(2.0 / math.pi)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    h = 1e-5  # g''(0) = 2 phi(0) = sqrt(2/pi), the same as x Phi(x)'s
    d2 = (mlp.gelu_grad(np.array([h]))[0] - mlp.gelu_grad(np.array([-h]))[0]) / (2 * h)
    assert d2 == pytest.approx(k0, rel=1e-9)
    # series g = x/2 + k0 x^2/2 + k0 (k1 - k0^2/3) x^4 / 2 + O(x^6) with k1 = 0.044715
    x = 3e-3
    c4 = (mlp.gelu(np.array([x]))[0] - x / 2 - k0 * x * x / 2) / x ** 4
    assert c4 == pytest.approx(0.5 * k0 * (0.044715 - k0 ** 2 / 3), rel=1e-5)
    z = np.linspace(-12.0, 12.0, 240001)
    assert np.max(np.abs(mlp.gelu(z) - 0.5 * z * (1.0 + erf(z / math.sqrt(2.0))))) <= 5e-4


def test_bf16_rounding():
    exact = np.array([1.0, -2.5, 0.15625, 3.0 * 2 ** -20, 0.0])
    assert np.array_equal(mlp.bf16(exact), exact)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    # 1 + 3 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mlp.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(0).normal(0, 10, 10000)
    assert np.max(np.abs(mlp.bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_nll_closed_forms():
    R = np.random.default_rng(4).normal(size=(1000, 2))
    out = np.zeros((1000, 4))
    assert np.allclose(mlp.nll(out, R), 0.5 * np.sum(R ** 2, axis=1))
    # the constant output minimising the mean NLL: mu = mean(R), s = log std(R)
    mu, sd = R.mean(0), R.std(0)
    best = np.tile(np.concatenate([mu, np.log(sd)]), (1000, 1))
    base = mlp.nll(best, R).mean()
    for d in (np.array([0.01, 0, 0, 0]), np.array([0, 0, 0.01, 0]), np.array([0, -0.01, 0, 0.01])):
        assert mlp.nll(best + d, R).mean() > base


def test_adam_first_step_is_lr_times_sign():
    theta = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, -1e-6, 5.0])
    t, m, v = mlp.adam_step(theta, g, np.zeros(5), np.zeros(5), step=1, lr=0.01, eps=1e-12)
    assert np.allclose(t, -0.01 * np.sign(g), rtol=1e-6)


def test_zero_output_layer_gives_the_transition():
    theta = mlp.init_params(5, out_scale=0.0)
    X, _ = _data(B=11)
    out, _ = mlp.forward(theta, X)
    assert np.all(out == 0.0)


def test_patch_rows_mirror_at_edges():
    J = 6
    x = np.arange(2 * J * J, dtype=np.float64)
    rows = mlp.patch_rows(x, J, [0, 14], np.array([0.5, -0.5]))
    v = x[:J * J].reshape(J, J)
    # node 0 = (0, 0): row offsets -2..2 map to rows 1, 0, 0, 1, 2 (mirror about the edge)
    idx = [1, 0, 0, 1, 2]
    assert np.array_equal(rows[0, :25].reshape(5, 5), v[np.ix_(idx, idx)])
    assert rows[0, 50] == 0.5
    # node 14 = (2, 2): an interior 5x5 window
    assert np.array_equal(rows[1, :25].reshape(5, 5), v[0:5, 0:5])
    assert np.array_equal(rows[1, 25:50].reshape(5, 5), x[J * J:].reshape(J, J)[0:5, 0:5])
