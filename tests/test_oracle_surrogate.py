"""Pins of the surrogate network's FP64 reference (oracle/surrogate.py).

The network is not in the paper, so its reference is pinned against mathematics:
BF16 rounding on hand-worked values and an independent conversion, GELU against
its closed-form values and symmetry, the backward pass against central finite
differences of the forward pass, and Adam's first step against its closed form.
"""

import math

import numpy as np
import pytest

import oracle.surrogate as S


def test_bf16_round_worked_values():
    one = 1.0
    u = 2.0 ** -7                      # BF16 spacing at 1 (7 stored mantissa bits)
    cases = [
        (1.0, 1.0),
        (one + u / 2, 1.0),            # tie -> even mantissa (0)
        (one + 1.5 * u, one + 2 * u),  # tie -> even mantissa (2)
        (one + u / 2 + 2.0 ** -20, one + u),
        (one + u / 2 - 2.0 ** -20, 1.0),
        (-(one + 1.5 * u), -(one + 2 * u)),
        (3.0, 3.0),
        (0.0, 0.0),
    ]
    for v, want in cases:
        assert S.bf16_round(np.array([v]))[0] == want, v


def test_bf16_round_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.Generator(np.random.PCG64(5)).standard_normal(20000) * 10.0 ** np.linspace(-8, 8, 20000)
    x32 = x.astype(np.float32)
    mine = S.bf16_round(x32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mine, ref)


def test_gelu_closed_forms():
    # GELU(z) = z Phi(z): Phi(0) = 1/2, Phi(1) = 0.841344746068542948585...
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert abs(S.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    z = np.linspace(-6, 6, 101)
    # Phi(-z) = 1 - Phi(z)  =>  GELU(-z) = GELU(z) - z
    assert np.max(np.abs(S.gelu(-z) - (S.gelu(z) - z))) < 1e-14
    # GELU'(0) = 1/2, and GELU' against central differences
    assert abs(S.gelu_prime(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - S.gelu_prime(z))) < 1e-8


def _tiny(seed=3, D=7, w=5, B=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.standard_normal(S.param_count(D, w)) * 0.5
    X = rng.standard_normal((B, D))
    T = rng.standard_normal((B, D))
    return theta, X, T, D, w


def test_forward_hand_computed_single_path():
    # w = 1, D = 1: f(x) = W4 GELU(W3 GELU(W2 GELU(W1 x + b1) + b2) + b3) + b4
    theta = np.array([0.7, 0.1, -1.3, 0.2, 0.9, -0.4, 1.5, 0.25])
    x = 0.6
    h1 = S.gelu(np.array([0.7 * x + 0.1]))[0]
    h2 = S.gelu(np.array([-1.3 * h1 + 0.2]))[0]
    h3 = S.gelu(np.array([0.9 * h2 - 0.4]))[0]
    want = 1.5 * h3 + 0.25
    Y, _ = S.forward(theta, np.array([[x]]), 1, 1, bf16=False)
    assert abs(Y[0, 0] - want) < 1e-15


def test_backward_matches_finite_differences():
    theta, X, T, D, w = _tiny()
    loss, g = S.loss_and_grad(theta, X, T, D, w, bf16=False)
    h = 1e-6
    for j in range(theta.size):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        lp, _ = S.loss_and_grad(tp, X, T, D, w, bf16=False)
        lm, _ = S.loss_and_grad(tm, X, T, D, w, bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j])), (j, fd, g[j])


def test_weighted_backward_matches_finite_differences():
    theta, X, T, D, w = _tiny(seed=11)
    c = np.random.Generator(np.random.PCG64(12)).uniform(0.0, 3.0, D)
    loss, g = S.loss_and_grad(theta, X, T, D, w, bf16=False, weights=c)
    Y, _ = S.forward(theta, X, D, w, bf16=False)
    assert abs(loss - np.mean(c * (Y - T) ** 2)) < 1e-14 * max(1.0, loss)
    h = 1e-6
    for j in range(0, theta.size, 3):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        fd = (S.loss_and_grad(tp, X, T, D, w, False, c)[0] - S.loss_and_grad(tm, X, T, D, w, False, c)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j])), (j, fd, g[j])


def test_loss_is_mean_square():
    theta, X, T, D, w = _tiny(seed=4)
    Y, _ = S.forward(theta, X, D, w, bf16=False)
    loss, _ = S.loss_and_grad(theta, X, T, D, w, bf16=False)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-15 * max(1.0, loss)


def test_bf16_reference_rounds_inputs_and_weights():
    # with every parameter and input already a BF16 value, rounding changes only
    # the hidden activations: the two modes then agree to BF16 precision
    theta, X, T, D, w = _tiny(seed=6)
    theta = S.bf16_round(theta.astype(np.float32))
    X = S.bf16_round(X.astype(np.float32))
    Y1, _ = S.forward(theta, X, D, w, bf16=True)
    Y0, _ = S.forward(theta, X, D, w, bf16=False)
    rel = np.max(np.abs(Y1 - Y0)) / np.max(np.abs(Y0))
    assert 0 < rel < 2.0 ** -7


def test_adam_first_step_closed_form():
    # from zero moments the bias-corrected first step is -lr g / (|g| + eps)
    rng = np.random.Generator(np.random.PCG64(8))
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m1, m2 = S.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.max(np.abs(new - (th - 1e-3 * g / (np.abs(g) + 1e-8)))) < 1e-15
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_param_count_and_layout():
    D, w = 11, 4
    n = S.param_count(D, w)
    assert n == w * D + w + w * w + w + w * w + w + D * w + D
    parts = S.unpack(np.arange(n, dtype=np.float64), D, w)
    assert parts[0].shape == (w, D) and parts[0][1, 0] == D          # row-major W1
    assert parts[6].shape == (D, w) and parts[7][0] == n - D          # b4 last
    with pytest.raises(AssertionError):
        S.unpack(np.zeros(n + 1), D, w)


def test_gelu_erf_constant():
    # the 1/sqrt(2 pi) factor of phi: integral of GELU'(z) - Phi(z) = z phi(z) over R is 0
    z = np.linspace(-12, 12, 24001)
    v = S.gelu_prime(z) - 0.5 * (1 + np.vectorize(math.erf)(z / math.sqrt(2)))
    assert abs(np.trapezoid(v, z)) < 1e-12
    # and the integral of z^2 phi(z) (second moment) is 1
    assert abs(np.trapezoid(z * v, z) - 1.0) < 1e-9
