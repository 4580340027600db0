"""Pins of the oracle's MLP (the learned proposal's network): finite
differences for every gradient, the GELU odd-part identity and its erf form,
a one-layer case that reduces to a matrix product, and BF16 rounding against
torch's bfloat16 conversion."""
import math

import numpy as np
import torch
from scipy.special import erf

import oracle

RNG = np.random.default_rng(7)


def init(dims, scale=0.5):
    p = []
    for l in range(1, len(dims)):
        p.append(RNG.normal(0, scale, dims[l] * dims[l - 1]))
        p.append(RNG.normal(0, 0.1, dims[l]))
    return np.concatenate(p)


def test_gradients_match_finite_differences():
    dims = [5, 8, 7, 3]
    P = init(dims)
    X = RNG.normal(size=(6, 5))
    Yt = RNG.normal(size=(6, 3))
    loss, g = oracle.mlp_loss_grad(dims, P, X, Yt)
    eps = 1e-6
    for i in range(P.size):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += eps
        Pm[i] -= eps
        fd = (oracle.mlp_loss_grad(dims, Pp, X, Yt)[0] - oracle.mlp_loss_grad(dims, Pm, X, Yt)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])
    Y = oracle.mlp_forward(dims, P, X)
    assert abs(loss - np.mean((Y - Yt) ** 2)) < 1e-14


def test_gelu_identity_and_erf_form():
    dims = [1, 1, 1]
    # identity weights: y = gelu(x)
    P = np.array([1.0, 0.0, 1.0, 0.0])
    x = np.linspace(-6, 6, 41)[:, None]
    y = oracle.mlp_forward(dims, P, x)[:, 0]
    assert np.allclose(y, 0.5 * x[:, 0] * (1 + erf(x[:, 0] / math.sqrt(2))), atol=1e-15)
    ym = oracle.mlp_forward(dims, P, -x)[:, 0]
    assert np.allclose(y - ym, x[:, 0], atol=1e-14)  # x Phi(x) - (-x) Phi(-x) = x


def test_single_layer_is_a_matrix_product():
    dims = [6, 4]
    P = init(dims)
    X = RNG.normal(size=(9, 6))
    W = P[:24].reshape(4, 6)
    b = P[24:]
    assert np.allclose(oracle.mlp_forward(dims, P, X), X @ W.T + b, atol=1e-13)


def test_bf16_rounding_matches_torch():
    dims = [6, 4]
    P = init(dims) * 3.3
    X = RNG.normal(size=(9, 6)) * 7.1
    W = P[:24].reshape(4, 6)
    b = P[24:]
    r = lambda a: torch.tensor(a, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    ref = r(X) @ r(W).T + b
    assert np.allclose(oracle.mlp_forward(dims, P, X, bf16=True), ref, atol=1e-12)
