"""Pins of the float64 reference of the learned recovery seed (oracle/mlp_ref.py)
against things other than itself: finite differences, hand-built networks
with closed-form outputs, the exact fit, Adam's first step, the published
SplitMix64 sequence and kinematic identities of the features."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_1508_03452_gb300 import workloads as W


def _data(n, seed):
    r = np.random.default_rng(seed)
    X = r.normal(size=(n, M.N_IN))
    X[:, 19] = 1.0
    Y = r.normal(size=(n, M.N_OUT)) * 0.3
    return X, Y


def test_parameter_count_matches_layout():
    assert M.NPARAM == 64 * 20 + 64 + 2 * (64 * 64 + 64) + 4 * 64 + 4 == 9924
    P = np.arange(M.NPARAM, dtype=np.float64)
    assert np.array_equal(M.pack(M.unpack(P)), P)


def test_gradient_matches_central_differences():
    X, Y = _data(7, 1)
    P = W.mlp_init_params(3).astype(np.float64)
    L, g = M.loss_and_grad(P, X, Y)
    assert L == pytest.approx(M.loss(P, X, Y), rel=1e-14)
    r = np.random.default_rng(5)
    # every bias and a random sample of weights of every layer
    o, idx = 0, []
    for name, shape in M.SHAPES:
        n = int(np.prod(shape))
        idx += list(o + (np.arange(n) if name.startswith("b") else r.choice(n, 40, replace=False)))
        o += n
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (M.loss(Pp, X, Y) - M.loss(Pm, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_hand_built_network_closed_form():
    """W1 picks +x0, -x1 and x2 into units 0, 1, 2; W2 is a permutation
    (unit k -> unit k+5 mod 64), W3 the identity; W4 reads units 5, 6, 7.
    Then y0 = relu(x0) + 2 relu(-x1), y1 = 3 relu(x2) + 0.5, y2 = y3 = 0.
    A transposed W2 would route the units elsewhere and fail."""
    d = {name: np.zeros(shape) for name, shape in M.SHAPES}
    d["W1"][0, 0], d["W1"][1, 1], d["W1"][2, 2] = 1.0, -1.0, 1.0
    for k in range(64):
        d["W2"][(k + 5) % 64, k] = 1.0
    d["W3"] = np.eye(64)
    d["W4"][0, 5], d["W4"][0, 6], d["W4"][1, 7] = 1.0, 2.0, 3.0
    d["b4"][1] = 0.5
    P = M.pack(d)
    X, _ = _data(50, 2)
    y = M.forward(P, X)
    assert np.allclose(y[:, 0], np.maximum(X[:, 0], 0) + 2 * np.maximum(-X[:, 1], 0), rtol=0, atol=1e-15)
    assert np.allclose(y[:, 1], 3 * np.maximum(X[:, 2], 0) + 0.5, rtol=0, atol=1e-15)
    assert np.all(y[:, 2:] == 0)


def test_exact_fit_has_zero_loss_and_gradient():
    X, _ = _data(9, 3)
    P = W.mlp_init_params(4).astype(np.float64)
    L, g = M.loss_and_grad(P, X, M.forward(P, X))
    assert L == 0.0 and np.all(g == 0.0)


def test_first_adam_step_closed_form():
    """From zero moments the bias-corrected first step is lr g / (|g| + eps)."""
    r = np.random.default_rng(6)
    P, g = r.normal(size=M.NPARAM), r.normal(size=M.NPARAM)
    P1, m, v = M.adam_step(P, np.zeros_like(P), np.zeros_like(P), g, 1, 1e-3)
    assert np.allclose(P - P1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 0: its first two outputs (state 0, then state
    0 + golden gamma) are 0xE220A8397B1DCDAF and 0x6E789E6AA1B965F4."""
    assert M.splitmix64(0) == 0xE220A8397B1DCDAF
    assert M.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_batch_rows_in_range_and_spread():
    rows = M.batch_rows(7, 3, 4000, 1000)
    assert rows.min() >= 0 and rows.max() < 1000
    counts = np.bincount(rows, minlength=1000)
    assert counts.max() < 20 and (counts > 0).mean() > 0.95


def test_features_kinematic_identities():
    """For N^mu = n U^mu, N^a / N^0 = beta; for dust (p = 0, no fields)
    T^{0a} / T^00 = beta and T^{ab} / T^00 = beta_a beta_b."""
    beta = np.array([0.3, -0.2, 0.1])
    g = 1 / np.sqrt(1 - beta @ beta)
    U = g * np.concatenate([[1.0], beta])
    n, rho = 1.7, 2.3
    T = rho * np.outer(U, U)
    x = M.features(T, n * U, np.zeros(3), np.zeros(3))
    assert np.allclose(x[0:3], beta, rtol=1e-15, atol=0)
    assert np.allclose(x[9:12], beta, rtol=1e-15, atol=0)
    bb = np.outer(beta, beta)
    assert np.allclose(x[3:9], [bb[0, 0], bb[1, 1], bb[2, 2], bb[0, 1], bb[0, 2], bb[1, 2]], rtol=1e-14, atol=0)
    assert x[12] == pytest.approx(n / (rho * g), rel=1e-15) and x[19] == 1.0


def test_bf16_rounding():
    assert M.to_bf16(1.0) == 1.0
    assert M.to_bf16(1.0 + 2 ** -8) == 1.0                # tie, rounds to even
    assert M.to_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie, rounds up to even
    assert M.to_bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7      # representable
    x = np.random.default_rng(1).normal(size=1000)
    assert np.all(np.abs(M.to_bf16(x) - x) <= 2 ** -8 * np.abs(x))  # half an ulp


def test_training_reduces_loss():
    """A few hundred Adam steps on a smooth target lower the loss."""
    r = np.random.default_rng(8)
    X = r.uniform(-1, 1, size=(512, M.N_IN))
    X[:, 19] = 1
    Y = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], np.zeros(512), 0.5 * X[:, 3]], 1)
    data = np.concatenate([X, Y], 1)
    P = W.mlp_init_params(9).astype(np.float64)
    P, m, v, losses = M.train(P, np.zeros_like(P), np.zeros_like(P), data, 300, 64, 3e-3, 11)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()
