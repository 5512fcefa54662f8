"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random matrices; it holds none of the reduction's arithmetic.
The paper measures on random matrices with entries uniform in (0, 1) (Section 4); the
workloads below follow the configured shapes and distributions: Gaussian N(0, 1)
entries (symmetrised for the symmetric case), a symmetric matrix with a known spectrum
that is log-uniform in [1e-6, 1] with random signs, and batches of uneven sizes.  The
generator is NumPy's PCG64 with an explicit seed, in FP64, column-major.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sym_gaussian(n: int, seed: int = 0) -> np.ndarray:
    """G ~ N(0,1) n x n, A = (G + G^T)/2, column-major."""
    G = rng(seed).standard_normal((n, n))
    return np.asfortranarray((G + G.T) * 0.5)


def gen_gaussian(m: int, n: int, seed: int = 0) -> np.ndarray:
    """m x n with iid N(0,1) entries, column-major."""
    return np.asfortranarray(rng(seed).standard_normal((m, n)))


def sym_uniform(n: int, seed: int = 0) -> np.ndarray:
    """Paper-shaped symmetric input: entries uniform in (0,1), symmetrised."""
    G = rng(seed).random((n, n))
    return np.asfortranarray((G + G.T) * 0.5)


def sym_known_spectrum(n: int, seed_q: int = 0, seed_lam: int = 1):
    """A = Q diag(lam) Q^T with Q from the QR factorisation of a Gaussian matrix and
    lam_i = s_i * 10^{U(-6, 0)}, s_i = +-1 at random.  Returns (A, lam sorted)."""
    G = rng(seed_q).standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    r = rng(seed_lam)
    lam = np.power(10.0, r.uniform(-6.0, 0.0, n)) * np.where(r.random(n) < 0.5, -1.0, 1.0)
    A = (Q * lam) @ Q.T
    A = (A + A.T) * 0.5
    return np.asfortranarray(A), np.sort(lam)


def gen_known_singular(m: int, n: int, seed: int = 0):
    """A = U diag(sig) V^T with Haar-like U (m x n), V (n x n) and sig log-uniform in
    [1e-6, 1].  Returns (A, sig sorted descending)."""
    r = rng(seed)
    U, _ = np.linalg.qr(r.standard_normal((m, n)))
    V, _ = np.linalg.qr(r.standard_normal((n, n)))
    sig = np.power(10.0, r.uniform(-6.0, 0.0, n))
    A = (U * sig) @ V.T
    return np.asfortranarray(A), np.sort(sig)[::-1]


def batched_mix(count_sym: int = 1000, count_gen: int = 1000, nmin: int = 64, nmax: int = 1024,
                seed: int = 0, widths=(16, 32)):
    """Shapes of the batched workload: count_sym symmetric with n ~ U[nmin, nmax] and
    count_gen general m x n with n ~ U[nmin, nmax], m ~ U[n, 2n]; w drawn from widths.
    Returns two lists of (n, w) and (m, n, w); matrices are drawn by ``batched_matrix``."""
    r = rng(seed)
    sym = [(int(r.integers(nmin, nmax + 1)), int(r.choice(widths))) for _ in range(count_sym)]
    gen = []
    for _ in range(count_gen):
        n = int(r.integers(nmin, nmax + 1))
        m = int(r.integers(n, 2 * n + 1))
        gen.append((m, n, int(r.choice(widths))))
    return sym, gen


def batched_matrix(kind: str, index: int, shape, seed: int = 0) -> np.ndarray:
    """The index-th matrix of a batch: N(0,1) entries, symmetrised for kind == 'sym'."""
    s = seed * 1_000_003 + (0 if kind == "sym" else 500_000) + index + 17
    if kind == "sym":
        return sym_gaussian(shape[0], s)
    return gen_gaussian(shape[0], shape[1], s)
