"""Pins of the FP64 surrogate-network oracle against closed forms, library
routines and finite differences."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_round_matches_torch_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        # exact ties between two bfloat16 neighbours
                        (np.arange(1, 200) * 2 + 1) * 2.0 ** -8,
                        [0.0, -0.0, 1.0, -3.0, 65504.0, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 241)
    g = M.gelu(x)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # x Phi(x) - (-x) Phi(-x) = x
    assert np.allclose(g - M.gelu(-x), x, atol=1e-15)
    assert abs(M.gelu(np.array([10.0]))[0] - 10.0) < 1e-20
    # Phi(1) = 0.841344746068543 (normal table)
    assert abs(M.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-14
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(x), fd, atol=1e-9)


def test_gelu_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.linspace(-8, 8, 513)
    ref = torch.nn.functional.gelu(torch.tensor(x, dtype=torch.float64)).numpy()
    assert np.allclose(M.gelu(x), ref, atol=1e-15)


def test_backward_matches_finite_differences():
    """Every weight and bias gradient of a small network (3 -> 5 -> 5 -> 2)
    against central differences of the loss."""
    rng = np.random.default_rng(1)
    Wt, b = M.init_params([3, 5, 5, 2], rng)
    b = [rng.standard_normal(v.shape) * 0.1 for v in b]
    x = rng.standard_normal((7, 3))
    t = rng.standard_normal((7, 2))
    wgt = np.array([1.0, 0.5])
    y, cache = M.forward(Wt, b, x)
    gW, gb = M.backward(Wt, b, cache, y, t, weight=wgt)
    h = 1e-6

    def loss():
        return M.mse_loss(M.forward(Wt, b, x)[0], t, weight=wgt)

    for l in range(3):
        for arr, grad in ((Wt[l], gW[l]), (b[l], gb[l])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                i = it.multi_index
                keep = arr[i]
                arr[i] = keep + h
                lp = loss()
                arr[i] = keep - h
                lm = loss()
                arr[i] = keep
                assert abs((lp - lm) / (2 * h) - grad[i]) < 1e-8 * max(1.0, abs(grad[i]))


def test_linear_network_gradient_closed_form():
    """One linear layer: dL/dWt = 2/(B N) (X Wt^T + b - T)^T X."""
    rng = np.random.default_rng(2)
    Wt = [rng.standard_normal((3, 4))]
    b = [rng.standard_normal(3)]
    X, T = rng.standard_normal((6, 4)), rng.standard_normal((6, 3))
    y, cache = M.forward(Wt, b, X)
    gW, gb = M.backward(Wt, b, cache, y, T)
    R = X @ Wt[0].T + b[0] - T
    assert np.allclose(gW[0], 2.0 / R.size * R.T @ X, atol=1e-14)
    assert np.allclose(gb[0], 2.0 / R.size * R.sum(0), atol=1e-14)


def test_adam_first_step_closed_form():
    """After one update the bias-corrected moments are g and g^2, so the
    step is lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p = p0.copy()
    M.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.allclose(p0 - p, 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-18)


def test_bf16_forward_is_the_rounded_fp64_forward():
    """bf16=True changes only the stored operands: with inputs and weights
    already on the bfloat16 grid, the first pre-activation is identical."""
    rng = np.random.default_rng(4)
    Wt, b = M.init_params([7, 16, 4], rng)
    Wt = [M.bf16_round(w) for w in Wt]
    x = M.bf16_round(rng.standard_normal((5, 7)))
    _, (_, z64) = M.forward(Wt, b, x)
    _, (hs, z16) = M.forward(Wt, b, x, bf16=True)
    assert np.array_equal(z64[0], z16[0])
    assert np.array_equal(hs[1], M.bf16_round(M.gelu(z64[0])))


def test_training_reduces_loss_on_a_smooth_target():
    rng = np.random.default_rng(5)
    Wt, b = M.init_params([2, 16, 16, 1], rng)
    X = rng.uniform(-1, 1, (64, 2))
    T = np.sin(2 * X[:, :1]) + X[:, 1:] ** 2
    mW = [np.zeros_like(w) for w in Wt]
    vW = [np.zeros_like(w) for w in Wt]
    mb = [np.zeros_like(v) for v in b]
    vb = [np.zeros_like(v) for v in b]
    l0 = M.mse_loss(M.forward(Wt, b, X)[0], T)
    for t in range(1, 301):
        y, cache = M.forward(Wt, b, X)
        gW, gb = M.backward(Wt, b, cache, y, T)
        for l in range(3):
            M.adam_step(Wt[l], gW[l], mW[l], vW[l], t, 1e-2)
            M.adam_step(b[l], gb[l], mb[l], vb[l], t, 1e-2)
    l1 = M.mse_loss(M.forward(Wt, b, X)[0], T)
    assert l1 < 0.02 * l0
    assert math.isfinite(l1)
