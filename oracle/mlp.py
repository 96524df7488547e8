"""MADE autoregressive proposal network (oracle; test infrastructure only).

The paper's Metropolis chain (Sec. 4.2) proposes single bit flips.  The
learned proposal is an autoregressive Bernoulli model q(x) = prod_i
q(x_i | x_<i) (a masked autoencoder, Germain et al. 2015) with one input
layer n -> H, a hidden layer H -> H and an output layer H -> n:

    degrees   input i = i + 1 (i = 0..n-1), hidden unit k: m(k) = (k mod (n-1)) + 1
    masks     W1[k, i] kept iff m1(k) >= i + 1
              W2[k2, k1] kept iff m2(k2) >= m1(k1)
              W3[i, k] kept iff i + 1 > m2(k)
    forward   Z1 = X W1^T + b1, H1 = relu(Z1); Z2 = H1 W2^T + b2, H2 = relu(Z2);
              logits = H2 W3^T + b3, q(x_i = 1 | x_<i) = sigmoid(logit_i)
    loss      mean over the batch of the Bernoulli negative log-likelihood
    update    AdamW (decoupled weight decay), bias-corrected moments

Precision model of the CUDA kernels, emulated here in FP64: weights are used as
bfloat16 (round to nearest even) copies of FP32 master weights; H1, H2 and the
backward signals dZ3, dZ2, dZ1 are rounded to bfloat16 where they enter a
matrix product; products accumulate exactly (FP64 here, FP32 on the GPU);
biases, logits and gradients are not rounded.  `bf16=False` turns the
rounding off (used for the finite-difference pins).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def degrees(n: int, H: int):
    if n < 2:
        raise ValueError("MADE needs n >= 2")
    d_in = np.arange(1, n + 1)
    m = (np.arange(H) % (n - 1)) + 1
    return d_in, m, m


def masks(n: int, H: int):
    d_in, m1, m2 = degrees(n, H)
    M1 = (m1[:, None] >= d_in[None, :]).astype(np.float64)          # H x n
    M2 = (m2[:, None] >= m1[None, :]).astype(np.float64)            # H x H
    M3 = (d_in[:, None] > m2[None, :]).astype(np.float64)           # n x H
    return M1, M2, M3


def bits_matrix(xs, n: int) -> np.ndarray:
    xs = np.asarray(xs, dtype=np.uint64)
    return ((xs[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)


def _w(params, name, M, bf16):
    W = params[name] * M
    return bf16_round(W) if bf16 else W


def forward(params, X: np.ndarray, bf16: bool = True):
    """Returns (logits, cache).  X: batch x n of 0/1 floats."""
    n = X.shape[1]
    H = params["b1"].shape[0]
    M1, M2, M3 = masks(n, H)
    r = bf16_round if bf16 else (lambda a: a)
    W1, W2, W3 = _w(params, "W1", M1, bf16), _w(params, "W2", M2, bf16), _w(params, "W3", M3, bf16)
    Z1 = X @ W1.T + params["b1"]
    H1 = r(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + params["b2"]
    H2 = r(np.maximum(Z2, 0.0))
    logits = H2 @ W3.T + params["b3"]
    return logits, dict(X=X, W1=W1, W2=W2, W3=W3, H1=H1, H2=H2, M=(M1, M2, M3))


def _softplus(z):
    return np.logaddexp(0.0, z)


def nll(logits, X):
    """Per-row negative log-likelihood -log q(x)."""
    return np.sum(_softplus(logits) - X * logits, axis=1)


def log_prob(params, X, bf16: bool = True):
    logits, _ = forward(params, X, bf16)
    return -nll(logits, X)


def loss_and_grads(params, X, bf16: bool = True):
    """Mean NLL over the batch and its gradients (masked), backward in the order
    dZ3 -> (dW3, db3, dH2) -> dZ2 -> (dW2, db2, dH1) -> dZ1 -> (dW1, db1)."""
    r = bf16_round if bf16 else (lambda a: a)
    logits, c = forward(params, X, bf16)
    Mb = X.shape[0]
    loss = float(np.mean(nll(logits, X)))
    sig = 1.0 / (1.0 + np.exp(-logits))
    dZ3 = (sig - X) / Mb
    d3 = r(dZ3)
    M1, M2, M3 = c["M"]
    g = {}
    g["W3"] = (d3.T @ c["H2"]) * M3
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (d3 @ c["W3"]) * (c["H2"] > 0)
    d2 = r(dZ2)
    g["W2"] = (d2.T @ c["H1"]) * M2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (d2 @ c["W2"]) * (c["H1"] > 0)
    d1 = r(dZ1)
    g["W1"] = (d1.T @ X) * M1
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def adamw(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step; state holds m, v per tensor and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for k, p in params.items():
        m = state.setdefault("m_" + k, np.zeros_like(p))
        v = state.setdefault("v_" + k, np.zeros_like(p))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        out[k] = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return out


def sample(params, uniforms: np.ndarray, bf16: bool = True):
    """Autoregressive sampling: bit i = [u_i < q(x_i = 1 | x_<i)], i = 0..n-1.

    uniforms: batch x n.  Returns (X, log q(X)).
    """
    Bn, n = uniforms.shape
    X = np.zeros((Bn, n))
    for i in range(n):
        logits, _ = forward(params, X, bf16)
        p = 1.0 / (1.0 + np.exp(-logits[:, i]))
        X[:, i] = (uniforms[:, i] < p).astype(np.float64)
    return X, log_prob(params, X, bf16)


def init_params(n: int, H: int, seed: int):
    """FP32-representable initial weights (uniform fan-in scaling)."""
    rng = np.random.default_rng(seed)

    def u(shape, fan_in):
        lim = 1.0 / np.sqrt(fan_in)
        return rng.uniform(-lim, lim, size=shape).astype(np.float32).astype(np.float64)

    return {"W1": u((H, n), n), "b1": u((H,), n), "W2": u((H, H), H), "b2": u((H,), H),
            "W3": u((n, H), H), "b3": u((n,), H)}
