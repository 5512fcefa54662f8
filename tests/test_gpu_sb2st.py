"""Second stage on the GPU against the oracle: band -> tridiagonal (bulge chasing,
bandred_sb2st) and the tridiagonal's eigenvalues (bisection, bandred_sterf).

The oracle (oracle.sb2st / oracle.tridiag_eig, pinned on the CPU) takes the same
reflectors in the same order, so d and e are compared elementwise (the sums are formed
in another order, so to 1e-11 ||B||_F); the eigenvalues of the GPU tridiagonal are
compared with LAPACK's eigenvalues of the band, and the bisection with the oracle's
bisection.  The last tests run the whole eigenvalue path (sy2sb, sb2st, sterf) on the
known-spectrum workload.
"""
import time

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def band_of(n, w, seed):
    A = workloads.sym_gaussian(n, seed)
    i, j = np.indices((n, n))
    A[np.abs(i - j) > w] = 0.0
    return A


@pytest.mark.parametrize("n,w", [(50, 4), (200, 16), (300, 32), (513, 64), (260, 128), (40, 1), (3, 2), (2, 5),
                                 (1, 3), (97, 2), (400, 63)])
def test_sb2st_matches_oracle(br, n, w):
    A = band_of(n, w, 7 * n + w)
    dA = to_dev(np.tril(A))
    d, e, st = br.sb2st(dA, w)
    assert int(st.item()) == 0
    d, e = d.cpu().numpy(), e.cpu().numpy()
    do, eo = oracle.sb2st(np.tril(A), w)
    fa = np.linalg.norm(A)
    assert np.max(np.abs(d - do), initial=0.0) <= 1e-11 * fa
    assert np.max(np.abs(e - eo), initial=0.0) <= 1e-11 * fa
    if n > 1:
        la = np.linalg.eigvalsh(A)
        lt = sl.eigvalsh_tridiagonal(d, e)
        assert np.max(np.abs(lt - la)) <= 1e-13 * max(n, 10) * np.abs(la).max()
    # the input is not written
    assert np.array_equal(to_host(dA), np.tril(A))


@pytest.mark.parametrize("n,w", [(3000, 64), (3001, 17), (1200, 2)])
def test_sb2st_repeatable_and_matches_oracle(br, n, w):
    """Sweeps run concurrently, each waiting on the one before through a progress counter:
    the same input must give the same bits on every run (a missed dependency shows up as
    run-to-run differences), the eigenvalues of the band (an orthogonal similarity: also
    its trace and Frobenius norm), and for w >= 16 the oracle's d and e elementwise.  For
    small w and long chases the tridiagonal itself is ill-conditioned: the oracle moves by
    7e-12 ||A||_F at n = 1200, w = 2 when each input entry moves by one ulp, so rounding
    in another order is not held to 1e-11 there."""
    A = band_of(n, w, 5 * n + w)
    dA = to_dev(np.tril(A))
    runs = []
    for _ in range(4):
        d, e, st = br.sb2st(dA, w)
        assert int(st.item()) == 0
        runs.append((d.cpu().numpy(), e.cpu().numpy()))
    for d, e in runs[1:]:
        assert np.array_equal(d, runs[0][0]) and np.array_equal(e, runs[0][1])
    d, e = runs[0]
    fa = np.linalg.norm(A)
    la = np.linalg.eigvalsh(A)
    lt = sl.eigvalsh_tridiagonal(d, e)
    assert np.max(np.abs(lt - la)) <= 1e-13 * n * np.abs(la).max()
    assert abs(d.sum() - np.trace(A)) <= 1e-13 * n * fa
    assert abs((d @ d + 2 * e @ e) - fa * fa) <= 1e-13 * n * fa * fa
    if w >= 16:
        do, eo = oracle.sb2st(np.tril(A), w)
        assert np.max(np.abs(d - do)) <= 1e-11 * fa
        assert np.max(np.abs(e - eo)) <= 1e-11 * fa


def test_sb2st_on_sy2sb_output(br):
    """The packed sy2sb output (reflectors below the band) goes in unchanged."""
    n, w = 600, 24
    A = workloads.sym_gaussian(n, 21)
    dA = to_dev(A)
    _, _, st = br.sy2sb(dA, w, br.make_opts(b=8, precision="fp64"))
    assert int(st.item()) == 0
    d, e, st = br.sb2st(dA, w)
    assert int(st.item()) == 0
    lam = br.sterf(d, e).cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [1, 2, 17, 1000])
def test_sterf_matches_oracle(br, n):
    import torch

    rng = np.random.default_rng(n)
    d, e = rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))
    lam = br.sterf(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()).cpu().numpy()
    lo = oracle.tridiag_eig(d, e)
    scale = max(np.abs(lo).max(), 1.0)
    assert np.max(np.abs(lam - lo)) <= 1e-13 * scale
    if n > 1:
        assert np.max(np.abs(lam - sl.eigvalsh_tridiagonal(d, e))) <= 1e-13 * scale


def test_sterf_closed_form(br):
    import torch

    n = 513
    lam = br.sterf(torch.full((n,), 2.0, dtype=torch.float64, device="cuda"),
                   torch.full((n - 1,), -1.0, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = 2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.max(np.abs(lam - ref)) <= 1e-14


@pytest.mark.parametrize("n,w,precision", [(2048, 64, "ozaki"), (8192, 64, "ozaki")])
def test_eigenvalue_path_known_spectrum(br, n, w, precision):
    """sy2sb + sb2st + sterf on A = Q diag(lambda) Q^T: the eigenvalues within the
    backward error of the path (|lambda| spans 1e-6 .. 1)."""
    import torch

    A, lam_true = workloads.sym_known_spectrum(n, 0, 1)
    dA = to_dev(A)
    del A
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, st = br.sy2sb(dA, w, br.make_opts(b=w, precision=precision))
    assert int(st.item()) == 0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    d, e, st = br.sb2st(dA, w)
    assert int(st.item()) == 0
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    lam = br.sterf(d, e).cpu().numpy()
    t3 = time.perf_counter()
    print(f"\nn={n} w={w}: sy2sb {1e3 * (t1 - t0):.1f} ms, sb2st {1e3 * (t2 - t1):.1f} ms, "
          f"sterf {1e3 * (t3 - t2):.1f} ms")
    err = np.max(np.abs(lam - np.sort(lam_true)))
    assert err <= 1e-12 * np.abs(lam_true).max(), err


@pytest.mark.parametrize("n,w", [(300, 32), (260, 100)])
def test_sb2st_tiny_entries(br, n, w):
    """A band scaled by 2^-1000 (every reflector's vector below 2^-900), through the
    shared-memory kernel (w = 32) and the L2 one (w = 100): tiny vectors are scaled by exact
    powers of two, so d and e are 2^-1000 times the unscaled oracle's."""
    A = band_of(n, w, 13 * n + w)
    d, e, st = br.sb2st(to_dev(np.tril(A) * 2.0 ** -1000), w)
    assert int(st.item()) == 0
    d, e = d.cpu().numpy() * 2.0 ** 1000, e.cpu().numpy() * 2.0 ** 1000
    do, eo = oracle.sb2st(np.tril(A), w)
    fa = np.linalg.norm(A)
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
    assert np.max(np.abs(d - do)) <= 1e-11 * fa
    assert np.max(np.abs(e - eo)) <= 1e-11 * fa
