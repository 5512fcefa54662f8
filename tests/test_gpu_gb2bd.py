"""SVD second stage on the GPU against the oracle: upper band -> upper bidiagonal (bulge
chasing, bandred_gb2bd) and the bidiagonal's singular values (bandred_bdsv).

The oracle (oracle.gb2bd / oracle.bd_singular_values, pinned on the CPU) takes the same
reflectors in the same order, so d and e are compared elementwise (the sums are formed in
another order: to 1e-11 ||A||_F, where a one-ulp perturbation of the input moves the
oracle's own d and e by at most 3e-13 ||A||_F for these shapes); the singular values of
the GPU bidiagonal are compared with LAPACK's singular values of the band.  The last tests
run the whole SVD path (ge2gb, gb2bd, bdsv) on a dense matrix.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import to_dev

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


def upper_band(n, w, seed):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.standard_normal((n, n)))
    return np.triu(A) - np.triu(A, w + 1)


def bidiag(d, e):
    return np.diag(d) + np.diag(e, 1)


@pytest.mark.parametrize("n,w", [(50, 4), (200, 16), (300, 32), (513, 64), (260, 128), (40, 1), (3, 2), (2, 5),
                                 (1, 3), (97, 2), (400, 63)])
def test_gb2bd_matches_oracle(br, n, w):
    A = upper_band(n, w, 7 * n + w)
    dA = to_dev(A)
    d, e, st = br.gb2bd(dA, w)
    assert int(st.item()) == 0
    d, e = d.cpu().numpy(), e.cpu().numpy()
    do, eo = oracle.gb2bd(A, w)
    fa = np.linalg.norm(A)
    assert np.max(np.abs(d - do), initial=0.0) <= 1e-11 * fa
    assert np.max(np.abs(e - eo), initial=0.0) <= 1e-11 * fa
    if n > 1:
        sa = np.linalg.svd(A, compute_uv=False)
        sb = np.linalg.svd(bidiag(d, e), compute_uv=False)
        assert np.max(np.abs(sb - sa)) <= 1e-13 * max(n, 10) * sa.max()
    # the input is not written
    assert np.array_equal(dA.cpu().numpy(), A)


@pytest.mark.parametrize("n,w", [(2000, 64), (2001, 17)])
def test_gb2bd_repeatable_and_matches_oracle(br, n, w):
    """Sweeps run concurrently, each waiting on the one before through a progress counter:
    the same input must give the same bits on every run, and the oracle's result."""
    A = upper_band(n, w, 5 * n + w)
    dA = to_dev(A)
    runs = []
    for _ in range(4):
        d, e, st = br.gb2bd(dA, w)
        assert int(st.item()) == 0
        runs.append((d.cpu().numpy(), e.cpu().numpy()))
    for d, e in runs[1:]:
        assert np.array_equal(d, runs[0][0]) and np.array_equal(e, runs[0][1])
    d, e = runs[0]
    do, eo = oracle.gb2bd(A, w)
    fa = np.linalg.norm(A)
    assert np.max(np.abs(d - do)) <= 1e-11 * fa
    assert np.max(np.abs(e - eo)) <= 1e-11 * fa
    assert abs((d @ d + e @ e) - fa * fa) <= 1e-13 * n * fa * fa


@pytest.mark.parametrize("n", [1, 2, 17, 1000])
def test_bdsv_matches_oracle(br, n):
    import torch

    rng = np.random.default_rng(n)
    d, e = rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))
    s = br.bdsv(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()).cpu().numpy()
    so = oracle.bd_singular_values(d, e)
    ref = np.linalg.svd(bidiag(d, e), compute_uv=False)
    scale = max(ref.max(), 1.0)
    assert np.max(np.abs(s - so)) <= 1e-13 * scale
    assert np.max(np.abs(s - ref)) <= 1e-13 * scale


def test_bdsv_closed_form(br):
    import torch

    n = 513
    s = br.bdsv(torch.ones(n, dtype=torch.float64, device="cuda"),
                torch.ones(n - 1, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (2 * n + 1))
    assert np.max(np.abs(s - ref)) <= 1e-14


@pytest.mark.parametrize("m,n,w,precision", [(1024, 1024, 32, "fp64"), (1536, 1024, 64, "ozaki")])
def test_svd_path_on_ge2gb_output(br, m, n, w, precision):
    """ge2gb + gb2bd + bdsv: the singular values of A within the backward error of the path.
    The packed ge2gb result (reflectors below the band) goes into gb2bd unchanged."""
    A = workloads.gen_gaussian(m, n, 3)
    dA = to_dev(A)
    _, _, _, st = br.ge2gb(dA, w, br.make_opts(b=min(w, 32), precision=precision))
    assert int(st.item()) == 0
    d, e, st = br.gb2bd(dA, w)
    assert int(st.item()) == 0
    s = br.bdsv(d, e).cpu().numpy()
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - ref)) <= 1e-12 * ref.max()


def test_gb2bd_tiny_entries(br):
    """A band scaled by 2^-1000 (every reflector's vector below 2^-900): the chase scales
    tiny vectors by exact powers of two, so d and e are 2^-1000 times the unscaled
    oracle's."""
    n, w = 300, 32
    A = upper_band(n, w, 11)
    d, e, st = br.gb2bd(to_dev(A * 2.0 ** -1000), w)
    assert int(st.item()) == 0
    d, e = d.cpu().numpy() * 2.0 ** 1000, e.cpu().numpy() * 2.0 ** 1000
    do, eo = oracle.gb2bd(A, w)
    fa = np.linalg.norm(A)
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e))
    assert np.max(np.abs(d - do)) <= 1e-11 * fa
    assert np.max(np.abs(e - eo)) <= 1e-11 * fa
