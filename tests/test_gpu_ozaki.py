"""The Ozaki-scheme precision (BANDRED_OZAKI): FP64-class products on the BF16 tensor
cores, and the reductions built on them, against the FP64 oracle with the tolerances of
the plain FP64 path.

Engine bound: each row of an operand is scaled by a power of two above its largest entry
and cut into 7 signed 8-bit digits (56 bits); digit pairs are summed exactly, so an entry
of C = op(A) B errs by the dropped pairs and the final rounding, far below
1e-13 * sum_k |a_ik| |b_kj| (asserted; the RMS over entries must be near the unit
roundoff).  Reductions: the same elementwise parity with the oracle as the FP64 path
(band entries within 1e-12 ||A||_F, reflectors and tau within 1e-10) and backward error,
orthogonality and spectrum error below 1e-13.
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import gen_report, sym_report
from gpu_util import lower_band_and_v, to_dev, to_host

pytestmark = pytest.mark.gpu

B_TOL = 1e-12
V_TOL = 1e-10


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def rel_errors(C, Cref, absprod):
    e = np.abs(C - Cref) / np.maximum(absprod, 1e-300)
    return e.max(), np.sqrt(np.mean(e ** 2))


@pytest.mark.parametrize("m,n,k,trans", [(128, 64, 32, 0), (300, 64, 1000, 0), (257, 33, 700, 1),
                                         (1000, 128, 4100, 0), (64, 64, 8000, 1), (5, 16, 3, 0), (130, 7, 129, 1)])
def test_gemm_ozaki(br, m, n, k, trans):
    import torch

    rng = np.random.Generator(np.random.PCG64(m + n + k + 11))
    A = rng.standard_normal((k, m) if trans else (m, k))
    B = rng.standard_normal((k, n))
    dC = to_dev(np.full((m, n), np.nan))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_gemm_split(to_dev(A), to_dev(B), dC, "ozaki", transA=bool(trans), dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Aop = A.T if trans else A
    mx, rms = rel_errors(to_host(dC), Aop @ B, np.abs(Aop) @ np.abs(B))
    assert mx <= 1e-13 and rms <= 1e-15, (mx, rms)


def test_gemm_ozaki_wide_dynamic_range(br):
    """Rows and columns scaled by powers of two from 2^-300 to 2^300 (far outside the
    bf16 split modes' range): the per-row and per-column scaling keeps every entry's
    relative accuracy."""
    import torch

    rng = np.random.Generator(np.random.PCG64(5))
    m, n, k = 200, 40, 300
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-300, 300, size=(m, 1)))
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-300, 300, size=(1, n)))
    dC = to_dev(np.zeros((m, n)))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_gemm_split(to_dev(A), to_dev(B), dC, "ozaki", dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    mx, rms = rel_errors(to_host(dC), A @ B, np.abs(A) @ np.abs(B))
    assert mx <= 1e-13, (mx, rms)


@pytest.mark.parametrize("n,kb", [(128, 64), (300, 64), (513, 32), (77, 5)])
def test_syr2k_ozaki(br, n, kb):
    import torch

    rng = np.random.Generator(np.random.PCG64(n + kb))
    X, Y = rng.standard_normal((n, kb)), rng.standard_normal((n, kb))
    C0 = rng.standard_normal((n, n))
    dC = to_dev(C0)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_syr2k_split(to_dev(X), to_dev(Y), dC, "ozaki", dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    C = to_host(dC)
    ref = C0 + X @ Y.T + Y @ X.T
    low = np.tril(np.ones((n, n), dtype=bool))
    absprod = np.abs(C0) + np.abs(X) @ np.abs(Y).T + np.abs(Y) @ np.abs(X).T
    mx, _ = rel_errors(C[low], ref[low], absprod[low])
    assert mx <= 1e-13
    assert np.array_equal(C[~low], C0[~low])  # strictly upper triangle untouched


@pytest.mark.parametrize("n,w,b,la", [(512, 32, 32, -1), (300, 20, 16, 0), (257, 16, 5, -1), (130, 64, 64, 0),
                                      (400, 64, 32, -1)])
def test_sy2sb_ozaki_parity(br, n, w, b, la):
    A = workloads.sym_gaussian(n, seed=n + w + b + 1)
    dA = to_dev(A)
    _, tau, st = br.sy2sb(dA, w, br.make_opts(b=b, lookahead=la, precision="ozaki"))
    assert int(st.item()) == 0
    Aout, tau = to_host(dA), tau.cpu().numpy()
    Ao, to = oracle.sy2sb(A, w)
    fa = np.linalg.norm(A)
    bg, vg = lower_band_and_v(Aout, w)
    bo, vo = lower_band_and_v(Ao, w)
    assert np.max(np.abs(bg - bo), initial=0.0) <= B_TOL * fa
    assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tau - to), initial=0.0) <= V_TOL
    r = sym_report(A, Aout, tau, w)
    assert r["backward"] < 1e-13 and r["orth"] < 1e-13 and r["eig"] < 1e-13, r


@pytest.mark.parametrize("m,n,w,b,la", [(200, 200, 8, 8, 0), (300, 170, 10, 4, -1), (129, 100, 24, 8, -1),
                                        (90, 90, 30, 30, 0)])
def test_ge2gb_ozaki_parity(br, m, n, w, b, la):
    A = workloads.gen_gaussian(m, n, seed=m + n + w + 2)
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(b=b, lookahead=la, precision="ozaki"))
    assert int(st.item()) == 0
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    Ao, tqo, tpo = oracle.ge2gb(A, w)
    fa = np.linalg.norm(A)
    i, j = np.indices((m, n))
    band = (j - i >= 0) & (j - i <= w)
    assert np.max(np.abs(Aout[band] - Ao[band])) <= B_TOL * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= V_TOL
    assert np.max(np.abs(tq - tqo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tp - tpo), initial=0.0) <= V_TOL
    r = gen_report(A, Aout, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r
