"""Rectangular m < n on the GPU against the oracle (lower band form, A = Q B P^T).

Section 3.1 assumes m >= n; for a wide matrix the library reduces A^T (tall) with the
same kernels and writes the result back transposed, which the oracle defines the same way
(oracle.ge2gb_wide, pinned on the CPU by reconstruction and LAPACK singular values).
FP64 and Ozaki: elementwise at the FP64 parity tolerances; bf16x6: the singular values
of the band at its stated tolerance.
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import wide_band, wide_report
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


SHAPES = [(300, 520, 16, 8), (600, 1100, 32, 32), (64, 200, 8, 8), (10, 40, 12, 4), (257, 700, 40, 16)]


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("m,n,w,b", SHAPES)
def test_wide_matches_oracle(br, m, n, w, b, precision):
    A = workloads.gen_gaussian(m, n, 11 * m + n)
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(b=b, precision=precision))
    assert int(st.item()) == 0
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    Ao, tqo, tpo = oracle.ge2gb_wide(A, w)
    assert tq.shape == tqo.shape and tp.shape == tpo.shape
    i, j = np.indices((m, n))
    band = (i - j >= 0) & (i - j <= w)
    fa = np.linalg.norm(A)
    assert np.max(np.abs(Aout[band] - Ao[band])) <= 1e-12 * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= 1e-10
    assert np.max(np.abs(tq - tqo), initial=0.0) <= 1e-10
    assert np.max(np.abs(tp - tpo), initial=0.0) <= 1e-10
    r = wide_report(A, Aout, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r


def test_wide_split_precision_singular_values(br):
    m, n, w = 400, 900, 32
    A = workloads.gen_gaussian(m, n, 5)
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(precision="bf16x6"))
    assert int(st.item()) == 0
    s_b = np.linalg.svd(wide_band(to_host(dA), w), compute_uv=False)
    s_a = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s_b - s_a)) <= 2e-5 * s_a[0]
