"""The panel kernels' Newton-Raphson reciprocal square root and reciprocal, on their own.

The panel kernels form a Householder reflector (Section 2.1, Eq. updateA0) with
h = q / sqrt(q), tau = 1 + |alpha| / h and 1 / (alpha - beta) from an FP32 estimate
refined by two Newton-Raphson steps in FP64 (bandred_newton_eval evaluates the same
device functions).  Each step roughly doubles the correct bits of the 22-bit estimate,
so the results must lie within a few units in the last place of the exact values.  The
reference here is exact: Python's decimal arithmetic at 60 digits on the exact binary
value of each input.  The inputs cover every exponent of the stated ranges (both parities
of the exponent, which the reciprocal square root treats differently) and their ends.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
REL_BOUND = 4 * U  # "a few units in the last place"


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def _inputs(e_lo, e_hi, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    es = np.arange(e_lo, e_hi + 1)
    m = r.uniform(1.0, 2.0, es.size)
    x = np.ldexp(m, es)
    ends = [np.ldexp(1.0, e_lo), np.nextafter(np.ldexp(1.0, e_lo), np.inf), np.ldexp(1.0, e_hi),
            np.nextafter(np.ldexp(1.0, e_hi + 1), 0.0), 1.0, 2.0, 3.0, 4.0, np.nextafter(4.0, 0.0)]
    return np.concatenate([x, np.array(ends)])


def _rel_err(got, exact):
    return [abs((Decimal(float(g)) - t) / t) for g, t in zip(got, exact)]


def _eval(br, x):
    import torch

    dx = torch.from_numpy(x).cuda()
    rs = torch.empty_like(dx)
    rc = torch.empty_like(dx)
    assert br.bandred_newton_eval(dx, rs, rc) == 0
    torch.cuda.synchronize()
    return rs.cpu().numpy(), rc.cpu().numpy()


def test_rsqrt_within_a_few_ulps_over_the_normal_range(br):
    getcontext().prec = 60
    x = _inputs(-1022, 1022, 1)
    rs, _ = _eval(br, x)
    exact = [Decimal(1) / Decimal(float(v)).sqrt() for v in x]
    err = _rel_err(rs, exact)
    assert max(err) <= REL_BOUND, (max(err), x[int(np.argmax(err))])
    # and against the correctly rounded sqrt followed by a division (at most 1.5 ulps off)
    np.testing.assert_allclose(rs, 1.0 / np.sqrt(x), rtol=6 * U, atol=0)


def test_rcp_within_a_few_ulps_over_its_range(br):
    getcontext().prec = 60
    x = _inputs(-1021, 1020, 2)
    _, rc = _eval(br, x)
    exact = [Decimal(1) / Decimal(float(v)) for v in x]
    err = _rel_err(rc, exact)
    assert max(err) <= REL_BOUND, (max(err), x[int(np.argmax(err))])
    np.testing.assert_allclose(rc, 1.0 / x, rtol=5 * U, atol=0)


def test_both_exponent_parities_at_every_mantissa_bucket(br):
    # q = m 2^(2k) and m 2^(2k+1) for m across [1, 2): the rsqrt splits the exponent into an
    # even part and a parity bit that moves into the mantissa
    getcontext().prec = 60
    m = np.linspace(1.0, 2.0, 257)[:-1]
    x = np.concatenate([np.ldexp(m, 2 * 37), np.ldexp(m, 2 * 37 + 1), np.ldexp(m, -2 * 300), np.ldexp(m, -2 * 300 + 1)])
    rs, rc = _eval(br, x)
    err = _rel_err(rs, [Decimal(1) / Decimal(float(v)).sqrt() for v in x])
    assert max(err) <= REL_BOUND
    err = _rel_err(rc, [Decimal(1) / Decimal(float(v)) for v in x])
    assert max(err) <= REL_BOUND
