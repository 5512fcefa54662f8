"""The device trace, and what it shows about the look-ahead of Section 2.2 (Variant V2).

With b = w the next panel is factored on the high-priority stream while the rest of the
rank-2k update (A2^R) runs on the caller's stream; with the Ozaki precision the two
kernels hold disjoint sets of SMs.  The trace records, per launch, the earliest CTA start
and the latest CTA end (globaltimer), so the test can check the record layout and that
panel k+1 and A2^R of iteration k really run at the same time, while the result still
matches the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import lower_band_and_v, to_dev, to_host

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


def traced_sy2sb(br, A, w, **kw):
    import torch

    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    dA = to_dev(A)
    assert br.bandred_trace_begin(buf) == 0
    _, tau, st = br.sy2sb(dA, w, br.make_opts(**kw))
    recs = br.bandred_trace_end()
    assert int(st.item()) == 0
    return recs, to_host(dA), tau.cpu().numpy()


def overlap(a, b):
    return max(0, min(a["t1_ns"], b["t1_ns"]) - max(a["t0_ns"], b["t0_ns"]))


def test_trace_records_and_lookahead_overlap(br):
    n, w = 4096, 64
    A = workloads.sym_gaussian(n, 77)
    recs, Aout, tau = traced_sy2sb(br, A, w, b=w, precision="ozaki")
    # parity first: the traced run computes the same reduction
    Ao, to = oracle.sy2sb(A, w)
    bg, _ = lower_band_and_v(Aout, w)
    bo, _ = lower_band_and_v(Ao, w)
    assert np.max(np.abs(bg - bo)) <= 1e-12 * np.linalg.norm(A)
    assert np.max(np.abs(tau - to)) <= 1e-10
    panels = {r["iteration"]: r for r in recs if r["kind"] == "panel"}
    rest = {r["iteration"]: r for r in recs if r["kind"] == "rank_rest"}
    sym = [r for r in recs if r["kind"] == "x1_product"]
    ks = list(range(0, n - w - 1, w))
    assert sorted(panels) == ks and len(sym) == len(ks)
    assert all(r["t1_ns"] > r["t0_ns"] > 0 for r in recs)
    # look-ahead: panel k+w runs while A2^R of iteration k does, on other SMs; measured as
    # the share of the shorter of the two that runs concurrently with the other
    dur = lambda r: r["t1_ns"] - r["t0_ns"]
    ov = [overlap(panels[k + w], rest[k]) / min(dur(panels[k + w]), dur(rest[k]))
          for k in ks if k + w in panels and k in rest]
    print("\noverlap of the shorter launch:", np.round(ov, 2).tolist())
    assert len(ov) >= len(ks) // 2
    # the early iterations, where the rank-2k update is long, run the two side by side
    early = np.array(ov[: max(4, len(ov) // 4)])
    assert np.median(early) > 0.3 and np.max(early) > 0.5, ov
    # and X1 of iteration k + w starts only after both have ended (it reads all of A2 and W)
    for k in ks:
        if k + w in panels and k in rest:
            nxt = [r for r in sym if r["iteration"] == k + w][0]
            assert nxt["t0_ns"] >= max(panels[k + w]["t1_ns"], rest[k]["t1_ns"])


def test_trace_without_lookahead_has_no_overlap(br):
    n, w = 1024, 32
    A = workloads.sym_gaussian(n, 78)
    recs, _, _ = traced_sy2sb(br, A, w, b=w, precision="ozaki", lookahead=0)
    panels = {r["iteration"]: r for r in recs if r["kind"] == "panel"}
    rest = {r["iteration"]: r for r in recs if r["kind"] == "rank_rest"}
    for k, r in rest.items():
        if k + w in panels:
            assert overlap(panels[k + w], r) == 0
