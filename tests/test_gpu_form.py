"""Forming Q, U and V on the GPU from the packed reflectors of a finished reduction.

The reference is NumPy's explicit product of the same packed reflectors (tests/checks.py,
one reflector at a time, FP64): the GPU's blocked formation (compact WY in groups, last
group first, FP64 or Ozaki-scheme products) must give the same matrix to rounding, an
orthogonal one, and reconstruct A with the band: A = Q B Q^T (Section 2.1), A = U B V^T
(Section 3.1), A = Q B P^T for m < n.
"""
import numpy as np
import pytest

import workloads
from checks import gen_band, gen_form_uv, sym_band, sym_form_q, wide_band, wide_form_qp
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-12  # entries of an orthogonal matrix are at most 1


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def orth_err(Q):
    return np.linalg.norm(Q.T @ Q - np.eye(Q.shape[0]))


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("n,w,b,fb", [(700, 32, 32, 0), (300, 20, 8, 16), (130, 64, 64, 0), (97, 7, 3, 5)])
def test_sy2sb_form_q(br, n, w, b, fb, precision):
    A = workloads.sym_gaussian(n, 17 * n + w)
    dA = to_dev(A)
    _, tau, st = br.sy2sb(dA, w, br.make_opts(b=b, precision=precision))
    assert int(st.item()) == 0
    Qd, st2 = br.sy2sb_form_q(dA, w, tau, br.make_opts(b=fb, precision=precision))
    assert int(st2.item()) == 0
    Q = to_host(Qd)
    Aout, t = to_host(dA), tau.cpu().numpy()
    Qr = sym_form_q(Aout, t, w)
    assert np.max(np.abs(Q - Qr)) <= TOL
    assert orth_err(Q) <= 1e-13 * np.sqrt(n)
    B = sym_band(Aout, w)
    assert np.linalg.norm(A - Q @ B @ Q.T) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("m,n,w,b", [(640, 600, 24, 8), (300, 170, 10, 4), (90, 90, 30, 30)])
def test_ge2gb_form_u_v(br, m, n, w, b, precision):
    A = workloads.gen_gaussian(m, n, 19 * m + n)
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(b=b, precision=precision))
    assert int(st.item()) == 0
    o = br.make_opts(precision=precision)
    Ud, _ = br.ge2gb_form(dA, w, tq, 0, o)
    Vd, _ = br.ge2gb_form(dA, w, tp, 1, o)
    U, V = to_host(Ud), to_host(Vd)
    Aout = to_host(dA)
    Ur, Vr = gen_form_uv(Aout, tq.cpu().numpy(), tp.cpu().numpy(), w)
    assert np.max(np.abs(U - Ur)) <= TOL and np.max(np.abs(V - Vr)) <= TOL
    assert orth_err(U) <= 1e-13 * np.sqrt(m) and orth_err(V) <= 1e-13 * np.sqrt(n)
    assert np.linalg.norm(A - U @ gen_band(Aout, w) @ V.T) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_wide_form_q_p(br, precision):
    m, n, w = 300, 520, 16
    A = workloads.gen_gaussian(m, n, 23)
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(b=8, precision=precision))
    assert int(st.item()) == 0
    o = br.make_opts(precision=precision)
    Qd, _ = br.ge2gb_form(dA, w, tq, 0, o)
    Pd, _ = br.ge2gb_form(dA, w, tp, 1, o)
    Q, P = to_host(Qd), to_host(Pd)
    Aout = to_host(dA)
    Qr, Pr = wide_form_qp(Aout, tq.cpu().numpy(), tp.cpu().numpy(), w)
    assert np.max(np.abs(Q - Qr)) <= TOL and np.max(np.abs(P - Pr)) <= TOL
    assert np.linalg.norm(A - Q @ wide_band(Aout, w) @ P.T) <= 1e-13 * np.linalg.norm(A)


def test_form_q_at_n4096_on_device(br):
    """n = 4096, w = b = 64, Ozaki reduction and formation; checked on the device (test
    code): ||Q^T Q - I||_F and ||A - Q B Q^T||_F / ||A||_F."""
    import torch

    n, w = 4096, 64
    A = workloads.sym_gaussian(n, 3)
    dA = to_dev(A)
    o = br.make_opts(b=w, precision="ozaki")
    _, tau, st = br.sy2sb(dA, w, o)
    assert int(st.item()) == 0
    Q, st2 = br.sy2sb_form_q(dA, w, tau, o)
    assert int(st2.item()) == 0
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    orth = torch.linalg.norm(Q.t() @ Q - I).item()
    Bl = torch.tril(dA) - torch.tril(dA, -w - 1)
    B = Bl + torch.tril(Bl, -1).t()
    At = torch.from_numpy(A).cuda()
    bwd = (torch.linalg.norm(At - Q @ B @ Q.t()) / torch.linalg.norm(At)).item()
    print(f"\nn=4096 formed Q: orthogonality {orth:.2e}, backward {bwd:.2e}")
    assert orth <= 1e-13 * np.sqrt(n) and bwd <= 1e-13
