"""Host logic of the autotuner (paper_1709_00302_gb300.tune): candidate sets, size-class
keys, model features, model-guided selection and the JSON plan cache.  CPU only."""
import json
import math

import numpy as np
import pytest

from paper_1709_00302_gb300 import tune


@pytest.mark.parametrize("op,m,n,w", [("sy2sb", 8192, 8192, 64), ("sy2sb", 100, 100, 32), ("ge2gb", 3000, 2000, 128),
                                      ("sy2sb", 40, 40, 16), ("ge2gb", 64, 64, 8)])
def test_candidates_are_valid_and_contain_the_default(op, m, n, w):
    c = tune.candidates(op, m, n, w)
    assert len(c) == len(set(c)) > 0
    for cfg in c:
        assert 1 <= cfg.b <= w and cfg.panel_ctas >= 0
        # depth 2 only as Variant V1 of sy2sb with 3b <= w; otherwise none or auto, depth 1
        if cfg.depth == 2:
            assert op == "sy2sb" and cfg.lookahead == 1 and 3 * cfg.b <= w
        else:
            assert cfg.depth == 1 and cfg.lookahead in (0, -1)
    d = tune.default_config(op, m, n, w)
    if d.b >= 8 and d.b < n - w:
        assert d in c


def test_size_class_rounds_up_to_powers_of_two():
    assert tune.size_class("sy2sb", 8192, 8192, 64, "bf16x6") == "sy2sb/bf16x6/m8192/n8192/w64"
    assert tune.size_class("sy2sb", 5000, 5000, 64, "fp64") == "sy2sb/fp64/m8192/n8192/w64"
    assert tune.size_class("ge2gb", 1025, 1000, 32, "bf16x6") == "ge2gb/bf16x6/m2048/n1024/w32"


def test_features_are_finite_order_one_and_distinguish_configs():
    seen = set()
    for op in tune.OPS:
        for n in (256, 8192, 32768):
            for w in (16, 64, 128):
                for cfg in tune.candidates(op, n, n, w):
                    f = tune.features(op, n, n, w, cfg, "bf16x6")
                    assert f.shape == (tune.N_FEATURES,) and f.dtype == np.float32
                    assert np.all(np.isfinite(f)) and np.max(np.abs(f)) <= 2.0
                    seen.add(tuple(f.tolist()))
    n_cfg = sum(len(tune.candidates(op, n, n, w)) for op in tune.OPS for n in (256, 8192, 32768) for w in (16, 64, 128))
    assert len(seen) == n_cfg  # no two configurations share a feature vector


def test_pick_without_model_times_everything_and_with_model_the_top_k():
    c = tune.candidates("sy2sb", 4096, 4096, 64)
    assert tune.pick(c, {}) == c
    pred = np.arange(len(c), 0, -1, dtype=np.float64)  # last candidate predicted fastest
    top = tune.pick(c, {}, pred, 3)
    assert top == [c[-1], c[-2], c[-3]]
    assert tune.pick(c, {}, pred, 100) == c
    ties = np.ones(len(c))
    assert tune.pick(c, {}, ties, 2) == c[:2]


def test_records_to_arrays_and_plan_cache_round_trip(tmp_path):
    path = str(tmp_path / "plans.json")
    t = tune.Tuner(path)
    assert t.lookup("sy2sb", 4096, 4096, 48, "bf16x6") is None
    key = tune.size_class("sy2sb", 4096, 4096, 48, "bf16x6")
    t.plans[key] = {"b": 32, "lookahead": -1, "panel_ctas": 76, "ms": 12.5}
    t.records.append(dict(op="sy2sb", precision="bf16x6", m=4096, n=4096, w=48, b=32, lookahead=-1, panel_ctas=76,
                          ms=12.5))
    t.save()
    with open(path) as f:
        assert json.load(f)["plans"][key]["b"] == 32
    t2 = tune.Tuner(path)
    assert t2.lookup("sy2sb", 4000, 4000, 48, "bf16x6") == tune.Config(32, -1, 76)
    X, ms = tune.records_to_arrays(t2.records)
    assert X.shape == (1, tune.N_FEATURES) and ms[0] == 12.5


def test_plan_cache_options(tmp_path):
    import paper_1709_00302_gb300 as br

    br.build()
    t = tune.Tuner(str(tmp_path / "p.json"))
    o = t.opts("sy2sb", 1000, 1000, 48, "bf16x6")  # a class the packaged sweep lacks: defaults
    assert (o.b, o.lookahead, o.panel_ctas, o.precision) == (48, -1, 0, 2)
    t.plans[tune.size_class("sy2sb", 1000, 1000, 32, "bf16x6")] = {"b": 16, "lookahead": 0, "panel_ctas": 0, "ms": 1}
    o = t.opts("sy2sb", 1000, 1000, 32, "bf16x6")
    assert (o.b, o.lookahead) == (16, 0)


def regret(records_by_class, chooser):
    """Mean over classes of (time of the chosen config / best time) - 1."""
    out = []
    for recs in records_by_class.values():
        best = min(r["ms"] for r in recs)
        out.append(chooser(recs) / best - 1.0)
    return float(np.mean(out))


def test_regret_helper_on_a_toy_table():
    recs = {"a": [{"ms": 1.0}, {"ms": 2.0}], "b": [{"ms": 4.0}, {"ms": 3.0}]}
    assert math.isclose(regret(recs, lambda rs: rs[0]["ms"]), (0.0 + 1 / 3) / 2)


def test_packaged_sweep_is_consistent():
    """The shipped sweep: every record is a candidate of its class, and each plan is the
    fastest record of its class."""
    with open(tune.PACKAGED) as f:
        d = json.load(f)
    plans, recs = d["plans"], d["records"]
    assert len(plans) >= 20 and len(recs) >= 300
    best = {}
    for r in recs:
        key = tune.size_class(r["op"], r["m"], r["n"], r["w"], r["precision"])
        assert tune.Config(r["b"], r["lookahead"], r["panel_ctas"]) in tune.candidates(r["op"], r["m"], r["n"], r["w"])
        if key not in best or r["ms"] < best[key]["ms"]:
            best[key] = r
    assert set(best) == set(plans)
    for key, p in plans.items():
        assert p["ms"] == best[key]["ms"] and p["b"] == best[key]["b"]
    t = tune.Tuner("/nonexistent/plans.json")
    assert t.lookup("sy2sb", 8192, 8192, 128, "bf16x6") == tune.Config(**{k: plans["sy2sb/bf16x6/m8192/n8192/w128"][k]
                                                                          for k in ("b", "lookahead", "panel_ctas")})
