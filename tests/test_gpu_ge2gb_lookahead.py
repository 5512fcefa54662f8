"""ge2gb with both look-ahead overlaps of Section 3.2's third case (w >= 3b), against the
oracle at the FP64 parity tolerances.

The left update of iteration k and the pending right update of iteration k-1 commute; the
schedule forms both from products of the state before either (Z = W_U^T E, P = D W_V,
Z V = Z + (Z W_V) Y_V^T) and applies A + P Y_V^T + Y_U (Z V) in three pieces (the row block
that the row panel needs, the next column panel's columns, the rest) on two streams.  The
result must be the same reduction: same band, same reflectors.  The device trace checks
that row panel k runs while the right update of iteration k - b does.
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import gen_band, gen_report
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


def run(br, A, w, **kw):
    dA = to_dev(A)
    _, tq, tp, st = br.ge2gb(dA, w, br.make_opts(**kw))
    assert int(st.item()) == 0
    return to_host(dA), tq.cpu().numpy(), tp.cpu().numpy()


# (m, n, w, b) with 3b <= w: square and tall, tall panels and short ones (few rows per
# CTA), w a multiple of b and not, the last iterations narrower than b
SHAPES = [(640, 600, 24, 8), (700, 700, 96, 32), (300, 170, 10, 3), (1100, 900, 100, 33), (200, 200, 48, 16)]


@pytest.mark.parametrize("precision", ["fp64", "ozaki"])
@pytest.mark.parametrize("m,n,w,b", SHAPES)
def test_second_overlap_matches_oracle(br, m, n, w, b, precision):
    A = workloads.gen_gaussian(m, n, 7 * m + n + w)
    Aout, tq, tp = run(br, A, w, b=b, lookahead=2, precision=precision)
    Ao, tqo, tpo = oracle.ge2gb(A, w)
    i, j = np.indices((m, n))
    band = (j - i >= 0) & (j - i <= w)
    fa = np.linalg.norm(A)
    assert np.max(np.abs(Aout[band] - Ao[band])) <= 1e-12 * fa
    assert np.max(np.abs(Aout[~band] - Ao[~band]), initial=0.0) <= 1e-10
    assert np.max(np.abs(tq - tqo), initial=0.0) <= 1e-10
    assert np.max(np.abs(tp - tpo), initial=0.0) <= 1e-10
    r = gen_report(A, Aout, tq, tp, w)
    assert r["backward"] < 1e-13 and r["sv"] < 1e-13, r


def test_second_overlap_split_precision(br):
    m, n, w, b = 700, 700, 96, 32
    A = workloads.gen_gaussian(m, n, 3)
    Aout, tq, tp = run(br, A, w, b=b, lookahead=2, precision="bf16x6")
    r = gen_report(A, Aout, tq, tp, w)
    assert r["backward"] < 3e-5 and r["orth_u"] < 1e-12 and r["orth_v"] < 1e-12, r
    s_b = np.linalg.svd(gen_band(Aout, w), compute_uv=False)
    s_a = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s_b - s_a)) <= 2e-5 * s_a[0]


def test_row_panel_overlaps_previous_right_update(br):
    import torch

    m = n = 2048
    w, b = 96, 32
    A = workloads.gen_gaussian(m, n, 5)
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    assert br.bandred_trace_begin(buf) == 0
    Aout, tq, tp = run(br, A, w, b=b, lookahead=2, precision="ozaki")
    recs = br.bandred_trace_end()
    rows = {r["iteration"]: r for r in recs if r["kind"] == "row_panel"}
    right = {r["iteration"]: r for r in recs if r["kind"] == "right_update"}
    ov = []
    for kp in sorted(right):
        r, rp = right[kp], rows.get(kp + b)
        if rp is not None:
            o = max(0, min(rp["t1_ns"], r["t1_ns"]) - max(rp["t0_ns"], r["t0_ns"]))
            ov.append(o / min(rp["t1_ns"] - rp["t0_ns"], r["t1_ns"] - r["t0_ns"]))
    print("\nrow panel k vs right update of k - b, overlap of the shorter:", np.round(ov, 2).tolist())
    # the early iterations, where the right update is long, run the two side by side (late
    # ones finish the short update before the panel stream's own row-block updates end)
    early = np.array(ov[: max(10, len(ov) // 4)])
    assert len(ov) >= 10 and np.median(early) > 0.5 and np.max(early) > 0.9, ov
    Ao, _, _ = oracle.ge2gb(A, w)
    i, j = np.indices((m, n))
    band = (j - i >= 0) & (j - i <= w)
    assert np.max(np.abs(Aout[band] - Ao[band])) <= 1e-12 * np.linalg.norm(A)
