"""Pins for the oracle MADE proposal: autoregressive structure, normalisation,
finite-difference gradients, AdamW, bfloat16 rounding and sampling."""
import itertools

import numpy as np
import pytest

from oracle import mlp


def _params(n, H, seed=0):
    return mlp.init_params(n, H, seed)


def test_bf16_round_matches_definition():
    vals = np.array([1.0, 1.00390625, 1.0078125, 1.005859375, -3.14159, 1e-30, 65504.0, 0.0])
    got = mlp.bf16_round(vals)
    for v, g in zip(vals, got):
        # g must be representable with 8 significand bits and be a nearest neighbour
        f = np.float32(v).view(np.uint32)
        lo = np.uint32(f & 0xFFFF0000).view(np.float32)
        hi = np.uint32((f & 0xFFFF0000) + 0x10000).view(np.float32) if v >= 0 else np.uint32(
            (f & 0xFFFF0000) + 0x10000).view(np.float32)
        assert g in (float(lo), float(hi))
        assert abs(g - v) <= abs(float(hi) - float(lo)) / 2 + 1e-300
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert mlp.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


@pytest.mark.parametrize("bf16", [False, True])
def test_autoregressive_structure(bf16):
    """logit_i does not depend on x_j for j >= i."""
    n, H = 7, 24
    p = _params(n, H, 1)
    rng = np.random.default_rng(2)
    X = rng.integers(0, 2, size=(40, n)).astype(float)
    L0, _ = mlp.forward(p, X, bf16)
    for j in range(n):
        X2 = X.copy()
        X2[:, j] = 1 - X2[:, j]
        L1, _ = mlp.forward(p, X2, bf16)
        np.testing.assert_array_equal(L0[:, : j + 1], L1[:, : j + 1])


@pytest.mark.parametrize("bf16", [False, True])
def test_probabilities_normalise(bf16):
    n, H = 6, 16
    p = _params(n, H, 3)
    X = mlp.bits_matrix(np.arange(1 << n, dtype=np.uint64), n)
    total = np.exp(mlp.log_prob(p, X, bf16)).sum()
    assert total == pytest.approx(1.0, abs=1e-12)


def test_gradients_finite_differences():
    n, H = 5, 8
    p = _params(n, H, 4)
    rng = np.random.default_rng(5)
    X = rng.integers(0, 2, size=(12, n)).astype(float)
    _, g = mlp.loss_and_grads(p, X, bf16=False)
    M1, M2, M3 = mlp.masks(n, H)
    mk = {"W1": M1, "W2": M2, "W3": M3}
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            if k in mk and mk[k].reshape(-1)[idx] == 0:
                assert g[k].reshape(-1)[idx] == 0
                continue
            q1 = {kk: vv.copy() for kk, vv in p.items()}
            q2 = {kk: vv.copy() for kk, vv in p.items()}
            q1[k].reshape(-1)[idx] += eps
            q2[k].reshape(-1)[idx] -= eps
            l1, _ = mlp.loss_and_grads(q1, X, bf16=False)
            l2, _ = mlp.loss_and_grads(q2, X, bf16=False)
            fd = (l1 - l2) / (2 * eps)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, abs=1e-7, rel=1e-5), (k, idx)


def test_adamw_first_step_is_signed_lr():
    """With bias correction, the first Adam step moves every parameter by ~lr * sign(grad)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 0.0])}
    out = mlp.adamw(p, g, {}, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(out["a"], [0.99, -1.99, 0.5], atol=1e-9)
    out2 = mlp.adamw(p, g, {}, lr=0.01, eps=1e-12, wd=0.1)
    np.testing.assert_allclose(out2["a"], [0.99 - 0.001, -1.99 + 0.002, 0.5 - 0.0005], atol=1e-9)


def test_sampling_frequencies_match_model():
    n, H = 3, 8
    p = _params(n, H, 6)
    grid = (np.arange(24) + 0.5) / 24
    U = np.array(list(itertools.product(grid, repeat=n)))
    X, lq = mlp.sample(p, U)
    keys = (X * (1 << np.arange(n))).sum(axis=1).astype(int)
    freq = np.bincount(keys, minlength=1 << n) / len(keys)
    allx = mlp.bits_matrix(np.arange(1 << n, dtype=np.uint64), n)
    prob = np.exp(mlp.log_prob(p, allx))
    np.testing.assert_allclose(freq, prob, atol=0.03)
    np.testing.assert_allclose(lq, mlp.log_prob(p, X))


def test_training_reduces_loss():
    n, H = 8, 32
    p = _params(n, H, 7)
    rng = np.random.default_rng(8)
    # a correlated target: x_{i+1} copies x_i with probability 0.9
    X = np.zeros((256, n))
    X[:, 0] = rng.integers(0, 2, 256)
    for i in range(1, n):
        keep = rng.random(256) < 0.9
        X[:, i] = np.where(keep, X[:, i - 1], 1 - X[:, i - 1])
    st = {}
    l0, _ = mlp.loss_and_grads(p, X)
    for _ in range(200):
        _, g = mlp.loss_and_grads(p, X)
        p = mlp.adamw(p, g, st, lr=3e-3)
    l1, _ = mlp.loss_and_grads(p, X)
    assert l1 < 0.6 * l0
