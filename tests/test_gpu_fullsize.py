"""Full-size parity: the benchmark's workloads in the benchmark's launch configuration.

sy2sb n = 8192, w = b = 64 on the known-spectrum matrix (look-ahead auto, as bench.py
times it): the oracle runs the whole reduction once on the host cores (about a minute),
and the FP64 and Ozaki GPU paths must match it elementwise.  The split (bf16x6) path must
meet its stated backward error and the invariants of an orthogonal similarity: the band's
Frobenius norm and trace equal those of A (sqrt(sum lam^2) and sum lam, known exactly).

Tolerances at this size: entries of the band differ from the oracle's by rounding in a
different summation order, which grows with n: below 1e-11 ||A||_F (n u ~ 1e-12, ten
times margin; measured 8e-16).  A reflector is determined only to about
u ||A|| / ||x2|| by its column, and this spectrum reaches down to 1e-6 ||A||, so the late
reflectors' entries and tau are compared to 1e-7 (measured 1.5e-8).  The split path's
invariants are relative to ||A||_F with the bf16x6 backward-error tolerance.
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import gen_probe_backward, sym_probe_backward
from gpu_util import lower_band_and_v, to_dev, to_host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, W = 8192, 64
B_TOL = 1e-11
V_TOL = 1e-7
SPLIT_TOL = 3e-5


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


@pytest.fixture(scope="module")
def config2():
    A, lam = workloads.sym_known_spectrum(N, 0, 1)
    oracle.set_threads(0)
    Ao, to = oracle.sy2sb(A, W)
    return A, lam, Ao, to


def band_invariants(Aout, w):
    d = np.diagonal(Aout).copy()
    off = sum(np.sum(np.diagonal(Aout, -k) ** 2) for k in range(1, w + 1))
    return np.sqrt(np.sum(d * d) + 2.0 * off), np.sum(d)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_sy2sb_config2_matches_oracle(br, config2, precision):
    A, lam, Ao, to = config2
    dA = to_dev(A)
    _, tau, st = br.sy2sb(dA, W, br.make_opts(b=W, lookahead=-1, precision=precision))
    assert int(st.item()) == 0
    Aout, tau = to_host(dA), tau.cpu().numpy()
    fa = np.sqrt(np.sum(lam * lam))
    bg, vg = lower_band_and_v(Aout, W)
    bo, vo = lower_band_and_v(Ao, W)
    db = np.max(np.abs(bg - bo))
    dv = np.max(np.abs(vg - vo))
    dt = np.max(np.abs(tau - to))
    print(f"\n{precision}: band {db / fa:.2e} ||A||_F, v {dv:.2e}, tau {dt:.2e}")
    assert db <= B_TOL * fa and dv <= V_TOL and dt <= V_TOL
    assert sym_probe_backward(A, Aout, tau, W, probes=4) < 1e-13


def test_sy2sb_config2_split_path(br, config2):
    A, lam, _, _ = config2
    dA = to_dev(A)
    _, tau, st = br.sy2sb(dA, W, br.make_opts(b=W, lookahead=-1, precision="bf16x6"))
    assert int(st.item()) == 0
    Aout, tau = to_host(dA), tau.cpu().numpy()
    fa, tr = np.sqrt(np.sum(lam * lam)), np.sum(lam)
    fb, tb = band_invariants(Aout, W)
    bwd = sym_probe_backward(A, Aout, tau, W, probes=4)
    print(f"\nbf16x6: backward {bwd:.2e}, |dF|/F {abs(fb - fa) / fa:.2e}, |dtrace|/F {abs(tb - tr) / fa:.2e}")
    assert bwd <= SPLIT_TOL
    assert abs(fb - fa) <= SPLIT_TOL * fa and abs(tb - tr) <= SPLIT_TOL * fa


def test_ge2gb_config3_split_and_ozaki(br):
    """m = n = 8192, w = b = 64, N(0,1): backward error through the reflectors and the
    Frobenius norm of the band (= that of A) for bf16x6 and the Ozaki path."""
    A = workloads.gen_gaussian(N, N, 0)
    fa = np.linalg.norm(A)
    for precision, tol, ftol in (("bf16x6", SPLIT_TOL, SPLIT_TOL), ("ozaki", 1e-13, 1e-12)):
        dA = to_dev(A)
        _, tq, tp, st = br.ge2gb(dA, W, br.make_opts(b=W, lookahead=-1, precision=precision))
        assert int(st.item()) == 0
        Aout = to_host(dA)
        i, j = np.indices((N, N))
        band = (j - i >= 0) & (j - i <= W)
        fb = np.sqrt(np.sum(Aout[band] ** 2))
        bwd = gen_probe_backward(A, Aout, tq.cpu().numpy(), tp.cpu().numpy(), W, probes=4)
        print(f"\nge2gb {precision}: backward {bwd:.2e}, |dF|/F {abs(fb - fa) / fa:.2e}")
        assert bwd <= tol and abs(fb - fa) <= ftol * fa


def test_sy2sb_config4_invariants_on_device(br):
    """n = 32768, w = b = 128 (8.6 GB, drawn and checked on the device): Frobenius norm and
    trace of the band against those of A, relative to ||A||_F."""
    import torch

    n, w = 32768, 128
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    G = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    A = ((G + G.t()) * 0.5).t().contiguous().t()
    del G
    fa = torch.linalg.norm(A).item()
    tr = torch.trace(A).item()
    _, tau, st = br.sy2sb(A, w, br.make_opts(b=w, lookahead=-1, precision="bf16x6"))
    assert int(st.item()) == 0
    d = torch.diagonal(A)
    off = sum(torch.sum(torch.diagonal(A, -k) ** 2).item() for k in range(1, w + 1))
    fb = float(np.sqrt(torch.sum(d * d).item() + 2.0 * off))
    tb = torch.sum(d).item()
    print(f"\nn=32768: |dF|/F {abs(fb - fa) / fa:.2e}, |dtrace|/F {abs(tb - tr) / fa:.2e}")
    assert abs(fb - fa) <= SPLIT_TOL * fa and abs(tb - tr) <= SPLIT_TOL * fa
    assert torch.all(torch.isfinite(tau)).item()
