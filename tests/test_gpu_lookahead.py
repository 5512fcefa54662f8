"""Look-ahead schedules of Section 2.2 against the oracle (FP64 parity tolerances).

* Depth 2 (Variant V1 with 3b <= w): the panel two iterations ahead is factored on the
  panel stream after the one-sided updates of the two iterations before it, while the
  caller's stream runs the trailing update.  Same reflectors as the basic loop.
* Variant V2 with the Ozaki precision: the next panel and the rest of the rank-2k update
  hold disjoint sets of SMs; the split of the SMs (panel_ctas) must not change the result.
* Depth 2 asked where it is not open (3b > w, or V2) falls back to depth 1.
"""
import numpy as np
import pytest

import oracle
import workloads
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


def check(br, n, w, **kw):
    A = workloads.sym_gaussian(n, 3 * n + w)
    dA = to_dev(A)
    _, tau, st = br.sy2sb(dA, w, br.make_opts(**kw))
    assert int(st.item()) == 0
    Aout, tau = to_host(dA), tau.cpu().numpy()
    Ao, to = oracle.sy2sb(A, w)
    bg, vg = lower_band_and_v(Aout, w)
    bo, vo = lower_band_and_v(Ao, w)
    assert np.max(np.abs(bg - bo)) <= B_TOL * np.linalg.norm(A)
    assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
    assert np.max(np.abs(tau - to), initial=0.0) <= V_TOL


# (n, w, b): 3b <= w; n = 1100 has tall panels (more than 512 rows) and short ones
@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("n,w,b", [(600, 48, 16), (1100, 96, 32), (1100, 100, 33), (260, 64, 8)])
def test_depth2_v1_matches_oracle(br, n, w, b, precision):
    check(br, n, w, b=b, lookahead=1, depth=2, precision=precision)


@pytest.mark.parametrize("n,w,b,la", [(600, 40, 16, 1), (600, 32, 32, 2)])
def test_depth2_where_not_open_falls_back(br, n, w, b, la):
    check(br, n, w, b=b, lookahead=la, depth=2, precision="fp64")


@pytest.mark.parametrize("panel_ctas", [16, 38, 114, 151])
def test_v2_sm_split_matches_oracle(br, panel_ctas):
    check(br, 1100, 32, b=32, lookahead=2, precision="ozaki", panel_ctas=panel_ctas)
