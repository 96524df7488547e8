"""Helpers for the GPU parity tests: oracle runs (optionally in a spawn pool)
and comparisons of exported CUDA terms with oracle CH-forms."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import decomp
from oracle import estimators as E

_POOL = None


def pool():
    """Process pool for oracle work, started with spawn (safe after CUDA init)."""
    global _POOL
    if _POOL is None:
        _POOL = cf.ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)),
                                       mp_context=mp.get_context("spawn"))
    return _POOL


def _build_terms(args):
    n, ops, chi, mode, seed, ccz_mode, alphas = args
    terms, coefs, chs = decomp.build_decomposition(n, ops, chi=chi, mode=mode, seed=seed,
                                                   ccz_mode=ccz_mode, alphas=alphas)
    return terms, coefs, chs


def oracle_terms(n, ops, chi, mode, seed=0, ccz_mode="proj", alphas=None, parallel=False):
    """Oracle CH-forms, coefficients and choices of the given term indices."""
    alphas = list(range(chi)) if alphas is None else list(alphas)
    if not parallel or len(alphas) < 8:
        return _build_terms((n, ops, chi, mode, seed, ccz_mode, alphas))
    k = max(1, min(64, len(alphas) // 2))
    chunks = [alphas[i::k] for i in range(k)]
    res = list(pool().map(_build_terms, [(n, ops, chi, mode, seed, ccz_mode, c) for c in chunks]))
    order = {}
    for c, (t, b, ch) in zip(chunks, res):
        for i, a in enumerate(c):
            order[a] = (t[i], b[i], ch[i])
    return ([order[a][0] for a in alphas], [order[a][1] for a in alphas],
            [order[a][2] for a in alphas])


def _eta_job(args):
    terms, coefs, n, seed, ls = args
    return [E.overlap_A(terms, coefs, E.draw_A(n, seed, l)) for l in ls]


def oracle_overlaps(terms, coefs, n, seed, L, parallel=False):
    """<phi_A_l|psi> for l < L (complex)."""
    ls = list(range(L))
    if not parallel:
        return np.array(_eta_job((terms, coefs, n, seed, ls)))
    k = min(L, 32)
    chunks = [ls[i::k] for i in range(k)]
    res = list(pool().map(_eta_job, [(terms, coefs, n, seed, c) for c in chunks]))
    out = np.zeros(L, complex)
    for c, r in zip(chunks, res):
        out[c] = r
    return out


def compare_term(ex, i, ch, label=""):
    """Bit-exact comparison of exported GPU term i with oracle CHForm ch."""
    n = ch.n
    assert [int(w) for w in ex["F"][i]] == ch.F, f"{label} F differs"
    assert [int(w) for w in ex["G"][i]] == ch.G, f"{label} G differs"
    assert [int(w) for w in ex["M"][i]] == ch.M, f"{label} M differs"
    assert [int(g) for g in ex["gamma"][i]] == ch.gamma, f"{label} gamma differs"
    assert int(ex["v"][i]) == ch.v, f"{label} v differs"
    assert int(ex["s"][i]) == ch.s, f"{label} s differs"
    om = int(ex["omega"][i])
    assert bool((om >> 3) & 1) == ch.zero, f"{label} zero flag differs"
    if not ch.zero:
        assert om & 7 == ch.k % 8, f"{label} omega phase differs"
        assert om >> 8 == ch.h, f"{label} omega magnitude differs"
    assert n == ex["F"].shape[1]


def amp_tol(want, n, norm=1.0):
    """|a_gpu - a| <= 1e-5 max(|a|, ||psi|| 2^{-n/2})."""
    return 1e-5 * np.maximum(np.abs(want), norm * 2.0 ** (-n / 2))


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
