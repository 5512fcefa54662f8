"""Equal-bandwidth band form (Section 3.3) on the GPU against the oracle, A = U B V^T with
B(i, j) = 0 for |i - j| > w.

The oracle (oracle.ge2bb, pinned on the CPU by reconstruction, LAPACK singular values, the
w = 1 tridiagonal case and planted mistakes) takes the same reflectors in the same order,
so FP64 and Ozaki results are compared elementwise: the band at 1e-12 ||A||_F, the
reflector vectors and the tau at 1e-10.  bf16x6 is checked through the singular values of
the band at its stated tolerance.  Shapes cover tall, wide and square matrices, b < w and
b = w, ragged last blocks, and the degenerate cases where only one side (or neither) has
reflectors, each without look-ahead and with it (Variant V1 for 2b <= w: the next panels
inside B1 and C1; Variant V2 otherwise, asked for with lookahead = 2: inside the first
t = 2b - w columns and rows of D).
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import bb_band, bb_form_uv, bb_report
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


SHAPES = [(300, 260, 16, 8), (260, 300, 16, 16), (256, 256, 32, 8), (100, 40, 12, 4), (40, 100, 12, 5),
          (20, 10, 12, 4), (10, 20, 12, 4), (8, 8, 12, 4), (700, 650, 48, 16), (520, 700, 64, 64),
          (400, 380, 24, 16), (90, 300, 10, 10)]


def run(br, A, w, **kw):
    dA = to_dev(A)
    _, tq, tp, st = br.ge2bb(dA, w, br.make_opts(**kw))
    assert int(st.item()) == 0
    return dA, tq, tp


@pytest.mark.parametrize("lookahead", [0, -1, 2])
@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("m,n,w,b", SHAPES)
def test_ge2bb_matches_oracle(br, m, n, w, b, precision, lookahead):
    A = workloads.gen_gaussian(m, n, 13 * m + n)
    dA, tq, tp = run(br, A, w, b=b, precision=precision, lookahead=lookahead)
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    Ao, tqo, tpo = oracle.ge2bb(A, w)
    assert tq.shape == tqo.shape and tp.shape == tpo.shape
    i, j = np.indices((m, n))
    band = np.abs(i - j) <= w
    fa = np.linalg.norm(A)
    assert np.max(np.abs(Aout[band] - Ao[band]), initial=0.0) <= 1e-12 * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= 1e-10
    assert np.max(np.abs(tq - tqo), initial=0.0) <= 1e-10
    assert np.max(np.abs(tp - tpo), initial=0.0) <= 1e-10
    r = bb_report(A, Aout, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r


@pytest.mark.parametrize("b", [16, 32])
def test_ge2bb_split_precision_singular_values(br, b):
    m, n, w = 700, 600, 32
    A = workloads.gen_gaussian(m, n, 9)
    dA, _, _ = run(br, A, w, b=b, precision="bf16x6")
    s_b = np.linalg.svd(bb_band(to_host(dA), w), compute_uv=False)
    s_a = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s_b - s_a)) <= 2e-5 * s_a[0]


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("m,n,w,b", [(400, 330, 24, 8), (200, 260, 16, 16)])
def test_ge2bb_form_u_v(br, m, n, w, b, precision):
    A = workloads.gen_gaussian(m, n, 29 * m + n)
    dA, tq, tp = run(br, A, w, b=b, precision=precision)
    o = br.make_opts(precision=precision)
    Ud, _ = br.ge2bb_form(dA, w, tq, 0, o)
    Vd, _ = br.ge2bb_form(dA, w, tp, 1, o)
    U, V, Aout = to_host(Ud), to_host(Vd), to_host(dA)
    Ur, Vr = bb_form_uv(Aout, tq.cpu().numpy(), tp.cpu().numpy(), w)
    assert np.max(np.abs(U - Ur)) <= 1e-12 and np.max(np.abs(V - Vr)) <= 1e-12
    assert np.linalg.norm(A - U @ bb_band(Aout, w) @ V.T) <= 1e-13 * np.linalg.norm(A)
