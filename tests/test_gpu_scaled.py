"""GPU parity on inputs near the ends of the FP64 range (FP64 and Ozaki precisions).

The reflector of Section 2.1 / 3.1 needs ||x2||, and the panel kernels form it, with the
dot products that give the coefficients of the in-panel update, from plain sums over the
unnormalised column.  Those sums overflow for entries near 2^600 and underflow near
2^-600, so the kernels take a rare path: the column is scaled by a power of two near
1/max|x2| (exact) and the norm and every dot product are summed again.  These tests run
that path against the oracle, whose norm is scaled the same way (its own pins are in
test_oracle_scaling.py):

* A scaled by 2^600 or 2^-600: every reflector takes the rare path.
* A scaled by 2^497: a column's sum of squares, about len * 2^993, crosses the 2^1000
  threshold at a length near 128, so the long columns of the early panels take the rare
  path and the short ones do not (checked from the oracle's output).
* A scaled by 2^-451: a column's largest entry crosses the 2^-450 threshold, which long
  columns usually exceed and short ones usually do not.

Tolerances are the FP64 parity ones relative to the scaled matrix: band entries within
1e-12 ||A||_F, reflector entries and tau within 1e-10; the backward error, orthogonality
and spectrum of the result scaled back by the same power of two stay below 1e-13.
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


def fro(A, s):
    """||A||_F of 2^s A without overflow (A holds the unscaled entries)."""
    return float(np.linalg.norm(A)) * 2.0 ** s


def sym_case(br, n, w, s, precision, **kw):
    A = workloads.sym_gaussian(n, 40 + n + w)
    As = np.ldexp(A, s)
    dA = to_dev(As)
    _, tau, st = br.sy2sb(dA, w, br.make_opts(precision=precision, **kw))
    assert int(st.item()) == 0
    Aout, tau = to_host(dA), tau.cpu().numpy()
    Ao, to = oracle.sy2sb(As, w)
    bg, vg = lower_band_and_v(Aout, w)
    bo, vo = lower_band_and_v(Ao, w)
    fa = fro(A, s)
    assert np.all(np.isfinite(Aout[np.tril_indices(n)])) and np.all(np.isfinite(tau))
    assert np.max(np.abs(bg - bo)) <= B_TOL * fa
    assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tau - to), initial=0.0) <= V_TOL
    # the band scaled back by 2^-s is exact, so the report runs in the ordinary range
    i, j = np.indices((n, n))
    back = np.where((i - j >= 0) & (i - j <= w), np.ldexp(Aout, -s), Aout)
    r = sym_report(A, back, tau, w)
    assert r["backward"] < 1e-13 and r["orth"] < 1e-13 and r["eig"] < 1e-13, r
    return Ao, to


def gen_case(br, m, n, w, s, precision, **kw):
    A = workloads.gen_gaussian(m, n, 50 + m + w)
    As = np.ldexp(A, s)
    dA = to_dev(As)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(precision=precision, **kw))
    assert int(st.item()) == 0
    Aout, tq, tp = to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()
    Ao, tqo, tpo = oracle.ge2gb(As, w)
    i, j = np.indices((m, n))
    band = (j - i >= 0) & (j - i <= w)
    fa = fro(A, s)
    assert np.all(np.isfinite(Aout)) and np.all(np.isfinite(tq)) and np.all(np.isfinite(tp))
    assert np.max(np.abs(Aout[band] - Ao[band])) <= B_TOL * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= V_TOL
    assert np.max(np.abs(tq - tqo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tp - tpo), initial=0.0) <= V_TOL
    back = np.where(band, np.ldexp(Aout, -s), Aout)
    r = gen_report(A, back, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r


# (n, w, b): the first panels of n = 700 have more than 512 rows, the later ones fewer
# (fewer CTAs of the grid panel); b < w adds the A1 update and the V1 look-ahead
SYM = [(700, 32, 32), (300, 20, 8)]


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("s", [600, -600])
@pytest.mark.parametrize("n,w,b", SYM)
def test_sy2sb_scaled_by_power_of_two(br, n, w, b, s, precision):
    sym_case(br, n, w, s, precision, b=b)


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("s", [600, -600])
def test_ge2gb_scaled_by_power_of_two(br, s, precision):
    gen_case(br, 640, 600, 24, s, precision, b=8)


@pytest.mark.parametrize("s", [600, -600])
def test_sy2sb_scaled_cluster_panels(br, s):
    # panel_group = 1: panels of at most 512 rows on one thread-block cluster (the batched
    # path's panel), so its rare path runs too
    sym_case(br, 700, 32, s, "fp64", b=32, panel_group=1)
    sym_case(br, 300, 20, s, "ozaki", b=8, panel_group=1)


def test_sy2sb_scaled_four_reflector_panel(br):
    sym_case(br, 700, 32, 600, "fp64", b=32, panel_group=4, lookahead=0)
    sym_case(br, 700, 32, -600, "fp64", b=32, panel_group=4, lookahead=0)


def _log2_abs(x):
    return np.log2(np.abs(x[x != 0.0]))


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_sy2sb_overflow_threshold_crossed_midway(br, precision):
    n, w, s = 700, 32, 497
    Ao, to = sym_case(br, n, w, s, precision, b=32)
    # ||x|| = |beta| of each reflector: beta^2 >= 2^1000 on the long columns only
    beta = np.array([Ao[c + w, c] for c in range(n - w - 1)])
    lb = 2.0 * _log2_abs(beta)
    assert np.sum(lb > 1001.0) >= 20 and np.sum(lb < 999.0) >= 20


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_sy2sb_underflow_threshold_crossed_midway(br, precision):
    n, w, s = 700, 32, -451
    Ao, to = sym_case(br, n, w, s, precision, b=32)
    # max|x2| = max|v2| tau |beta| (x2 = v2 (alpha - beta), alpha - beta = -tau beta)
    amax = []
    for c in range(n - w - 2):
        v2 = Ao[c + w + 1:, c]
        if to[c] != 0.0:
            amax.append(np.log2(np.max(np.abs(v2)) * to[c]) + np.log2(abs(Ao[c + w, c])))
    amax = np.array(amax)
    assert np.sum(amax > -449.95) >= 10 and np.sum(amax < -450.05) >= 10


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
def test_ge2gb_overflow_threshold_crossed_midway(br, precision):
    gen_case(br, 640, 600, 24, 497, precision, b=8)
