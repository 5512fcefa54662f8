"""The autotuner on the GPU: live tuning of a small size class into the plan cache, and
the gain of the learned cost model on the recorded sweep of this GPU type.

Gain protocol (leave one size class out): for every size class of the committed sweep
(paper_1709_00302_gb300/tuning/sweep_bf16x6_gb300.json, timings of every candidate
configuration), the cost model is trained on the other classes' timings with the
library's CUDA kernels and ranks the held-out class's candidates; the tuner then times
only its top k.  Regret = time of the best timed candidate / best time of the class - 1.
The model must beat (1) timing k candidates drawn at random (exact expectation) and
(2) the library's default configuration, averaged over the classes.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SWEEP = os.path.join(ROOT, "paper_1709_00302_gb300", "tuning", "sweep_bf16x6_gb300.json")


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def by_class(records):
    from paper_1709_00302_gb300 import tune

    out = {}
    for r in records:
        out.setdefault(tune.size_class(r["op"], r["m"], r["n"], r["w"], r["precision"]), []).append(r)
    return out


def expected_min_of_random_k(times, k):
    """E[min of k distinct draws] = sum_i t_(i) C(N-i-1, k-1) / C(N, k), t sorted ascending."""
    t = sorted(times)
    N = len(t)
    if k >= N:
        return t[0]
    return sum(t[i] * math.comb(N - i - 1, k - 1) for i in range(N)) / math.comb(N, k)


def test_expected_min_formula_against_enumeration():
    t = [5.0, 1.0, 3.0, 2.0, 8.0]
    for k in (1, 2, 3):
        brute = np.mean([min(c) for c in itertools.combinations(t, k)])
        assert math.isclose(expected_min_of_random_k(t, k), brute)


def test_cost_model_beats_random_and_default(br):
    from paper_1709_00302_gb300 import tune

    with open(SWEEP) as f:
        records = json.load(f)["records"]
    classes = by_class(records)
    assert len(classes) >= 10
    k = 2
    reg_model, reg_rand, reg_def, rho = [], [], [], []
    for key, recs in classes.items():
        train = [r for kk, rs in classes.items() if kk != key for r in rs]
        X, ms = tune.records_to_arrays(train)
        model = tune.CostModel(hidden=32, seed=0)
        losses = model.fit(X, ms, steps=1500, lr=3e-3)
        assert losses[-1] < 0.5 * losses[0]
        Xc, msc = tune.records_to_arrays(recs)
        pred = model.predict_ms(Xc)
        best = float(np.min(msc))
        top = np.argsort(pred, kind="stable")[:k]
        reg_model.append(float(np.min(msc[top])) / best - 1.0)
        reg_rand.append(expected_min_of_random_k(list(msc), k) / best - 1.0)
        r0 = recs[0]
        d = tune.default_config(r0["op"], r0["m"], r0["n"], r0["w"])
        dm = [r["ms"] for r in recs if (r["b"], r["lookahead"], r["panel_ctas"]) == (d.b, d.lookahead, d.panel_ctas)]
        reg_def.append(dm[0] / best - 1.0 if dm else float(np.max(msc)) / best - 1.0)
        # Spearman rank correlation of prediction and measurement within the class
        rp = np.argsort(np.argsort(pred))
        rm = np.argsort(np.argsort(msc))
        rho.append(float(np.corrcoef(rp, rm)[0, 1]))
    m_model, m_rand, m_def = np.mean(reg_model), np.mean(reg_rand), np.mean(reg_def)
    print(f"\nmean regret: model top-{k} {m_model:.3f}, random {k} {m_rand:.3f}, default {m_def:.3f}; "
          f"mean rank correlation {np.mean(rho):.2f} over {len(classes)} classes")
    assert m_model < m_rand
    assert m_model <= m_def
    assert np.mean(rho) > 0.3


def test_live_tuning_of_a_small_class(br, tmp_path):
    import workloads
    from checks import sym_report
    from gpu_util import to_dev, to_host
    from paper_1709_00302_gb300 import tune

    n, w = 192, 16
    t = tune.Tuner(str(tmp_path / "plans.json"))
    best = t.tune("sy2sb", n, n, w, "bf16x6", reps=2)
    timed = [r for r in t.records if r["n"] == n]
    assert len(timed) == len(tune.candidates("sy2sb", n, n, w))
    assert min(r["ms"] for r in timed) == t.plans[tune.size_class("sy2sb", n, n, w, "bf16x6")]["ms"]
    t.save()
    t2 = tune.Tuner(str(tmp_path / "plans.json"))
    assert t2.lookup("sy2sb", n, n, w, "bf16x6") == best
    # the tuned options compute a valid reduction
    A = workloads.sym_gaussian(n, 3)
    Ad = to_dev(A)
    o = t2.opts("sy2sb", n, n, w, "bf16x6")
    _, tau, st = br.sy2sb(Ad, w, o)
    rep = sym_report(A, to_host(Ad), tau.cpu().numpy(), w)
    assert int(st.item()) == 0
    assert rep["backward"] <= 3e-5 and rep["eig"] <= 2e-5 and rep["orth"] < 1e-10
