"""Parity of the FP64 GPU path with the FP64 oracle (elementwise), through the C ABI.

Section 2.1 (sy2sb) and Section 3.1 (ge2gb).  Tolerances: the oracle and the GPU apply
the same reflectors in a different order (blocked WY vs one at a time), so entries agree
to a small multiple of the unit roundoff times the matrix norm:
  band entries     |B_gpu - B_oracle| <= 1e-12 ||A||_F
  reflector v, tau |dv|, |dtau| <= 1e-10 (v entries are at most 1 in magnitude)
and the independent checks give backward error, orthogonality and spectrum error below
1e-13 (the FP64 tolerance of the reduction).
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import gen_band, gen_report, sym_report
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


def run_sy2sb(br, A, w, **kw):
    dA = to_dev(A)
    _, tau, _ = br.sy2sb(dA, w, br.make_opts(**kw))
    return to_host(dA), tau.cpu().numpy()


def check_sy2sb_parity(A, Aout, tau, w):
    Ao, to = oracle.sy2sb(A, w)
    fa = np.linalg.norm(A)
    bg, vg = lower_band_and_v(Aout, w)
    bo, vo = lower_band_and_v(Ao, w)
    assert np.max(np.abs(bg - bo), initial=0.0) <= B_TOL * fa
    assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tau - to), initial=0.0) <= V_TOL


@pytest.mark.parametrize("n,w,b", [(512, 32, 32), (300, 20, 16), (300, 20, 8), (97, 7, 3), (130, 64, 64),
                                   (257, 16, 5), (64, 1, 1)])
def test_sy2sb_fp64_parity(br, n, w, b):
    A = workloads.sym_gaussian(n, seed=0 if n == 512 else n + w + b)
    Aout, tau = run_sy2sb(br, A, w, b=b, lookahead=0)
    check_sy2sb_parity(A, Aout, tau, w)
    r = sym_report(A, Aout, tau, w)
    assert r["backward"] < 1e-13 and r["orth"] < 1e-13 and r["eig"] < 1e-13, r


def test_sy2sb_upper_triangle_untouched(br):
    n, w = 150, 12
    A = workloads.sym_gaussian(n, 3)
    Au = A.copy()
    Au[np.triu_indices(n, 1)] = np.nan
    Aout, tau = run_sy2sb(br, Au, w, b=8)
    assert np.all(np.isnan(Aout[np.triu_indices(n, 1)]))
    assert not np.any(np.isnan(np.tril(Aout)))
    check_sy2sb_parity(A, Aout, tau, w)


@pytest.mark.parametrize("n,w", [(0, 3), (1, 1), (5, 4), (6, 4), (7, 5), (3, 1)])
def test_sy2sb_trivial_and_tiny(br, n, w):
    import torch

    A = workloads.sym_gaussian(n, 9) if n else np.zeros((0, 0))
    if n == 0:
        dA = torch.zeros((0, 0), dtype=torch.float64, device="cuda")
        _, tau, _ = br.sy2sb(dA, w)
        assert tau.numel() == 0
        return
    Aout, tau = run_sy2sb(br, A, w)
    check_sy2sb_parity(A, Aout, tau, w)


@pytest.mark.parametrize("m,n,w,b", [(200, 200, 8, 8), (300, 170, 10, 4), (64, 64, 1, 1), (129, 100, 24, 8),
                                     (90, 90, 30, 30), (40, 33, 40, 16)])
def test_ge2gb_fp64_parity(br, m, n, w, b):
    A = workloads.gen_gaussian(m, n, seed=m + n + w)
    dA = to_dev(A)
    _, tq, tp, _ = br.ge2gb(dA, w, br.make_opts(b=b, lookahead=0))
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    Ao, tqo, tpo = oracle.ge2gb(A, w)
    fa = np.linalg.norm(A)
    band = gen_band(Ao, w) != 0
    i, j = np.indices((m, n))
    band = (j - i >= 0) & (j - i <= w)
    assert np.max(np.abs(Aout[band] - Ao[band])) <= B_TOL * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= V_TOL
    assert np.max(np.abs(tq - tqo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tp - tpo), initial=0.0) <= V_TOL
    r = gen_report(A, Aout, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r


def test_bounded_wait_reports_timeout(br):
    """A device wait that can never be satisfied ends after its limit with a status."""
    import torch

    n, w = 200, 16
    A = to_dev(workloads.sym_gaussian(n, 1))
    o = br.make_opts(b=16, timeout_ms=50, debug=1)
    tau = torch.zeros(n - w, dtype=torch.float64, device="cuda")
    work = torch.empty(br.bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = br.bandred_sy2sb_ex(A, w, tau, o, work, status)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 1  # BANDRED_DEV_TIMEOUT
    # the context is still usable afterwards
    A2 = workloads.sym_gaussian(64, 2)
    Aout, tau2 = run_sy2sb(br, A2, 4)
    check_sy2sb_parity(A2, Aout, tau2, 4)


def test_workspace_too_small_is_rejected(br):
    import torch

    n, w = 100, 8
    A = to_dev(workloads.sym_gaussian(n, 1))
    o = br.make_opts()
    need = br.bandred_sy2sb_workspace(n, w, o)
    tau = torch.zeros(n - w, dtype=torch.float64, device="cuda")
    work = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    assert br.bandred_sy2sb_ex(A, w, tau, o, work) == -8


def test_short_form_allocates_and_matches(br):
    import torch

    n, w = 180, 10
    A = workloads.sym_gaussian(n, 4)
    dA = to_dev(A)
    tau = torch.zeros(n - w, dtype=torch.float64, device="cuda")
    assert br.bandred_sy2sb(dA, w, tau) == 0
    check_sy2sb_parity(A, to_host(dA), tau.cpu().numpy(), w)


# Panels of the single-matrix reductions run on the cooperative grid kernel, which takes
# its reflectors either in pairs or in groups of four per grid-wide reduction (option
# panel_group); both must give the oracle's reflectors.  Orthogonality of
# the Q formed from them is bounded by 3e-16 n (the oracle's own reaches about 8e-17 n).
@pytest.mark.parametrize("group", [2, 4])
@pytest.mark.parametrize("n,w,b,la", [(1200, 64, 64, 0), (1100, 40, 16, -1), (1030, 21, 5, 0), (1100, 64, 32, -1)])
def test_sy2sb_grid_panel_parity(br, n, w, b, la, group):
    A = workloads.sym_gaussian(n, seed=n + b + group)
    Aout, tau = run_sy2sb(br, A, w, b=b, lookahead=la, panel_group=group)
    check_sy2sb_parity(A, Aout, tau, w)
    r = sym_report(A, Aout, tau, w)
    assert r["backward"] < 1e-13 and r["orth"] < 3e-16 * n and r["eig"] < 1e-13, r


@pytest.mark.parametrize("group", [2, 4])
def test_ge2gb_grid_panel_parity(br, group):
    m, n, w, b = 1100, 900, 24, 8
    A = workloads.gen_gaussian(m, n, seed=7 + group)
    dA = to_dev(A)
    _, tq, tp, _ = br.ge2gb(dA, w, br.make_opts(b=b, lookahead=-1, panel_group=group))
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


@pytest.mark.parametrize("group", [2, 4])
def test_sy2sb_rank_deficient_grid_panels(br, group):
    """A symmetric matrix of rank 30: the trailing panels' columns become dependent, the
    grouped reflectors hit their cancellation guard and fall back to fewer per reduction.
    The reflectors of a rank-deficient panel are set by rounding, so the checks are the
    invariants: backward error, orthogonality and the spectrum."""
    n, w, b = 1100, 32, 32
    rng = np.random.Generator(np.random.PCG64(41))
    U, _ = np.linalg.qr(rng.standard_normal((n, 30)))
    A = (U * rng.uniform(0.5, 2.0, 30)) @ U.T
    A = np.asfortranarray((A + A.T) / 2)
    Aout, tau = run_sy2sb(br, A, w, b=b, lookahead=0, panel_group=group)
    r = sym_report(A, Aout, tau, w)
    assert r["backward"] < 1e-13 and r["orth"] < 3e-16 * n and r["eig"] < 1e-13, r
