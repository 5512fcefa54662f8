"""The seeded input generators (workloads.py) produce the stated recipes: exact known
spectra and singular values, the stated distributions and the batched shape ranges.
CPU only."""
import numpy as np
import pytest

import workloads


def test_known_spectrum_is_exact_and_log_uniform_with_both_signs():
    A, lam = workloads.sym_known_spectrum(240, 0, 1)
    assert A.flags.f_contiguous and np.array_equal(A, A.T)
    assert np.max(np.abs(np.linalg.eigvalsh(A) - lam)) <= 1e-14 * 240
    mag = np.abs(lam)
    assert mag.min() >= 1e-6 and mag.max() <= 1.0
    assert (lam > 0).any() and (lam < 0).any()
    # log10 |lam| uniform on [-6, 0]: mean -3, variance 3
    lg = np.log10(mag)
    assert abs(lg.mean() + 3.0) < 0.4 and abs(lg.var() - 3.0) < 0.8


def test_known_singular_values_are_exact():
    A, sig = workloads.gen_known_singular(300, 200, 5)
    assert A.shape == (300, 200) and A.flags.f_contiguous
    assert np.max(np.abs(np.linalg.svd(A, compute_uv=False) - sig)) <= 1e-14 * 300
    assert np.all(np.diff(sig) <= 0) and sig.min() >= 1e-6 and sig.max() <= 1.0


def test_gaussian_inputs_have_the_stated_moments():
    A = workloads.sym_gaussian(400, 3)
    assert A.flags.f_contiguous and np.array_equal(A, A.T)
    off = A[np.triu_indices(400, 1)]
    assert abs(off.mean()) < 0.01 and abs(off.var() - 0.5) < 0.02   # (G + G^T)/2
    assert abs(np.diag(A).var() - 1.0) < 0.2
    G = workloads.gen_gaussian(300, 200, 4)
    assert abs(G.mean()) < 0.01 and abs(G.var() - 1.0) < 0.02
    U = workloads.sym_uniform(300, 2)
    assert np.array_equal(U, U.T) and U.min() > 0.0 and U.max() < 1.0


def test_seeds_reproduce_and_differ():
    assert np.array_equal(workloads.sym_gaussian(50, 7), workloads.sym_gaussian(50, 7))
    assert not np.array_equal(workloads.sym_gaussian(50, 7), workloads.sym_gaussian(50, 8))


@pytest.mark.parametrize("seed", [0, 1])
def test_batched_mix_shapes(seed):
    sym, gen = workloads.batched_mix(1000, 1000, seed=seed)
    assert len(sym) == 1000 and len(gen) == 1000
    assert all(64 <= n <= 1024 and w in (16, 32) for n, w in sym)
    assert all(64 <= n <= 1024 and n <= m <= 2 * n and w in (16, 32) for m, n, w in gen)
    ns = np.array([n for n, _ in sym])
    assert abs(ns.mean() - 544) < 25            # U[64, 1024]
    assert 0.4 < np.mean([w == 16 for _, w in sym]) < 0.6
    assert workloads.batched_mix(1000, 1000, seed=seed) == (sym, gen)
    B = workloads.batched_matrix("sym", 3, (sym[3][0],), seed)
    assert B.shape == (sym[3][0],) * 2 and np.array_equal(B, B.T)
    m, n, _ = gen[5]
    assert workloads.batched_matrix("gen", 5, (m, n), seed).shape == (m, n)
