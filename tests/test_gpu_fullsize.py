"""Full-size parity: the benchmark's workloads in the benchmark's launch configuration.

The batched workload (2000 uneven matrices) runs whole, with sampled matrices checked
against the oracle.  sy2sb n = 8192, w = b = 64 on the known-spectrum matrix (look-ahead
auto, as bench.py times it): the oracle runs the whole reduction once on the host cores (about a minute),
and the FP64 and Ozaki GPU paths must match it elementwise.  The split (bf16x6) path must
meet its stated backward error and the invariants of an orthogonal similarity: the band's
Frobenius norm and trace equal those of A (sqrt(sum lam^2) and sum lam, known exactly).

ge2gb m = n = 8192, w = b = 64 on N(0,1) runs against the oracle in the same way, and
the singular values of its band are compared with those of the oracle's band and of A.
sy2sb n = 32768, w = b = 128 is checked on the device: a 16-probe backward error with Q
applied through the reflectors, and the band's Frobenius norm and trace.

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


@pytest.fixture(scope="module")
def config3():
    A = workloads.gen_gaussian(N, N, 0)
    oracle.set_threads(0)
    Ao, tqo, tpo = oracle.ge2gb(A, W)
    return A, Ao, tqo, tpo


def svdvals_on_device(M):
    """Singular values of a host matrix, by the GPU's dense SVD (test-side check only)."""
    import torch

    return torch.linalg.svdvals(torch.from_numpy(np.ascontiguousarray(M)).cuda()).cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_ge2gb_config3_matches_oracle(br, config3, precision):
    """m = n = 8192, w = b = 64, N(0,1), look-ahead as bench.py runs it: the band, the
    reflectors and tau elementwise against the oracle, and the singular values of the band
    against those of the oracle's band and of A (the reduction is an orthogonal
    equivalence, so all three agree to rounding relative to sigma_max)."""
    A, Ao, tqo, tpo = config3
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, W, br.make_opts(b=W, lookahead=-1, precision=precision))
    assert int(st.item()) == 0
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    fa = np.linalg.norm(A)
    i, j = np.indices((N, N))
    band = (j - i >= 0) & (j - i <= W)
    db = np.max(np.abs(Aout[band] - Ao[band]))
    dv = np.max(np.abs(Aout[~band] - Ao[~band]))
    dq, dp = np.max(np.abs(tq - tqo)), np.max(np.abs(tp - tpo))
    Bg, Bo = np.where(band, Aout, 0.0), np.where(band, Ao, 0.0)
    sg, so, sa = svdvals_on_device(Bg), svdvals_on_device(Bo), svdvals_on_device(A)
    e_go, e_ga = np.max(np.abs(sg - so)) / sa[0], np.max(np.abs(sg - sa)) / sa[0]
    print(f"\nge2gb {precision}: band {db / fa:.2e} ||A||_F, v {dv:.2e}, tauq {dq:.2e}, taup {dp:.2e}, "
          f"sigma vs oracle band {e_go:.2e}, vs A {e_ga:.2e} (of sigma_max)")
    assert db <= B_TOL * fa and dv <= 1e-8 and dq <= 1e-8 and dp <= 1e-8
    assert e_go <= 1e-11 and e_ga <= 1e-11
    assert gen_probe_backward(A, Aout, tq, tp, W, probes=4) < 1e-13


def apply_reflectors_on_device(Aout, tau, w, X, transpose):
    """Q^T X (transpose) or Q X through the packed reflectors of a sy2sb result held on the
    device: H_c = I - tau_c v_c v_c^T on rows c+w.., v_c = [1; Aout(c+w+1:, c)]."""
    import torch

    X = X.clone()
    order = range(tau.numel()) if transpose else reversed(range(tau.numel()))
    taus = tau.cpu().numpy()
    one = torch.ones(1, dtype=X.dtype, device=X.device)
    for c in order:
        t = float(taus[c])
        if t == 0.0:
            continue
        r0 = c + w
        v = torch.cat((one, Aout[r0 + 1:, c]))
        X[r0:] -= t * torch.outer(v, v @ X[r0:])
    return X


def sym_band_times_on_device(Aout, w, Y):
    """B Y with B the symmetric band held in the lower band of Aout."""
    import torch

    BY = torch.diagonal(Aout)[:, None] * Y
    for d in range(1, w + 1):
        dg = torch.diagonal(Aout, -d)[:, None]  # B(i + d, i)
        BY[d:] += dg * Y[:-d]
        BY[:-d] += dg * Y[d:]
    return BY


@pytest.mark.parametrize("precision,tol", [("bf16x6", SPLIT_TOL), ("ozaki", 1e-13)])
def test_sy2sb_config4_probe_backward_on_device(br, precision, tol):
    """n = 32768, w = b = 128 (8.6 GB, drawn and checked on the device): with 16 Gaussian
    probes X, ||A X - Q B Q^T X||_F / ||A X||_F, Q applied through the reflectors on the
    device (test code, torch); also the Frobenius norm and trace of the band against
    those of A."""
    import torch

    n, w, probes = 32768, 128, 16
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    G = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    A = ((G + G.t()) * 0.5).t().contiguous().t()
    del G
    X = torch.randn((n, probes), dtype=torch.float64, device="cuda", generator=g)
    AX = A @ X
    fa = torch.linalg.norm(A).item()
    tr = torch.trace(A).item()
    _, tau, st = br.sy2sb(A, w, br.make_opts(b=w, lookahead=-1, precision=precision))
    assert int(st.item()) == 0
    assert torch.all(torch.isfinite(tau)).item()
    QtX = apply_reflectors_on_device(A, tau, w, X, transpose=True)
    QBQtX = apply_reflectors_on_device(A, tau, w, sym_band_times_on_device(A, w, QtX), transpose=False)
    bwd = (torch.linalg.norm(AX - QBQtX) / torch.linalg.norm(AX)).item()
    d = torch.diagonal(A)
    off = sum(torch.sum(torch.diagonal(A, -k) ** 2).item() for k in range(1, w + 1))
    fb = float(np.sqrt(torch.sum(d * d).item() + 2.0 * off))
    tb = torch.sum(d).item()
    print(f"\nn=32768 {precision}: probe backward {bwd:.2e}, |dF|/F {abs(fb - fa) / fa:.2e}, "
          f"|dtrace|/F {abs(tb - tr) / fa:.2e}")
    assert bwd <= tol
    assert abs(fb - fa) <= max(tol, 1e-12) * fa and abs(tb - tr) <= max(tol, 1e-12) * fa


def test_batched_config5_sampled_against_oracle(br):
    """The whole batched workload (1000 sy2sb n ~ U[64,1024] and 1000 ge2gb m ~ U[n,2n],
    w in {16,32}, as bench.py runs it: both kinds planned, then run), with six matrices of
    each kind (the largest, the smallest and four more) checked against the oracle: the
    bf16x6 backward error, FP64 orthogonality, and the spectrum of the band."""
    import torch

    from checks import gen_band, gen_report, sym_band, sym_report

    sym, gen = workloads.batched_mix(1000, 1000, seed=0)
    mats_s = [workloads.batched_matrix("sym", q, (n,)) for q, (n, _) in enumerate(sym)]
    mats_g = [workloads.batched_matrix("gen", q, (m, n)) for q, (m, n, _) in enumerate(gen)]
    dS = [to_dev(a) for a in mats_s]
    dG = [to_dev(a) for a in mats_g]
    taus = [torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda") for n, w in sym]
    tqs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _, n, _ in gen]
    tps = [torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda") for _, n, w in gen]
    opts = br.make_opts(precision="bf16x6")
    sb = br.SyBatch(dS, [w for _, w in sym], taus, opts)
    gb = br.GeBatch(dG, [w for _, _, w in gen], tqs, tps, opts)
    ws = torch.empty(sb.workspace(), dtype=torch.uint8, device="cuda")
    wg = torch.empty(gb.workspace(), dtype=torch.uint8, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert sb.plan(ws) == 0 and gb.plan(wg) == 0, br.bandred_last_error()
    assert sb.run(ws, st[0:1]) == 0 and gb.run(wg, st[1:2]) == 0
    torch.cuda.synchronize()
    assert int(st.sum().item()) == 0
    pick = lambda sizes: sorted({int(np.argmax(sizes)), int(np.argmax([0] + sizes[1:])), int(np.argmin(sizes)), 1, 250,
                                 500, 999})
    # ||Q^T Q - I||_F of a product of Householder reflectors grows like m u; these reach m = 2048
    orth_tol = lambda m: max(1e-13, m * 1.2e-16)
    for q in pick([n for n, _ in sym]):
        (n, w), A = sym[q], mats_s[q]
        Aout, tau = to_host(dS[q]), taus[q].cpu().numpy()
        r = sym_report(A, Aout, tau, w)
        assert r["backward"] <= SPLIT_TOL and r["orth"] <= orth_tol(n), (q, n, w, r)
        Ao, _ = oracle.sy2sb(A, w)
        lg, lo = np.linalg.eigvalsh(sym_band(Aout, w)), np.linalg.eigvalsh(sym_band(Ao, w))
        assert np.max(np.abs(lg - lo)) <= 2e-5 * np.linalg.norm(A, 2), (q, n, w)
    for q in pick([n for _, n, _ in gen]):
        (m, n, w), A = gen[q], mats_g[q]
        Aout = to_host(dG[q])
        r = gen_report(A, Aout, tqs[q].cpu().numpy(), tps[q].cpu().numpy(), w)
        assert r["backward"] <= SPLIT_TOL and r["orth_u"] <= orth_tol(m) and r["orth_v"] <= orth_tol(n), (q, m, n, w, r)
        Ao, _, _ = oracle.ge2gb(A, w)
        sg = np.linalg.svd(gen_band(Aout, w), compute_uv=False)
        so = np.linalg.svd(gen_band(Ao, w), compute_uv=False)
        assert np.max(np.abs(sg - so)) <= 2e-5 * so[0], (q, m, n, w)
