"""Autotuner of the band reductions, with a learned cost model that ranks configurations.

Section 4.2 of the paper shows that the best algorithmic block size b depends on the
problem dimension, the bandwidth w and the parallelism, and the paper tunes b by timing
for every (n, w).  This module does the same search on the GPU: for a size class it
enumerates candidate configurations (b, look-ahead variant, panel CTA count), times them
through the ``bandred_*_ex`` entry points with CUDA events, and keeps the fastest in a
JSON plan cache.

The cost model (``CostModel``; kernels in ``csrc/mlp.cu``, C ABI in
``include/bandred_tune.h``) is a small perceptron that predicts log run time from a
configuration's features.  Trained on the timings of other size classes, it ranks the
candidates of a new class so that only the best-ranked few need to be timed
(``Tuner.tune(..., budget=k, model=...)``).  It never changes a result: every candidate
computes the same reduction.

Command line (on a GPU):
    python -m paper_1709_00302_gb300.tune sweep --out sweep.json     # time every candidate
    python -m paper_1709_00302_gb300.tune tune --op sy2sb --n 8192 --w 64
"""
from __future__ import annotations

import argparse
import json
import math
import os
from dataclasses import asdict, dataclass

import numpy as np

OPS = ("sy2sb", "ge2gb")
PRECISION_IDS = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "ozaki": 3}
N_FEATURES = 9


@dataclass(frozen=True)
class Config:
    b: int
    lookahead: int  # -1 = the variant that b and w allow (Section 2.2 / 3.2), 0 = none
    panel_ctas: int  # 0 = the library's choice (all SMs for a large panel)
    depth: int = 1  # look-ahead depth (2: V1 with 3b <= w, the panel two iterations ahead)


def default_config(op: str, m: int, n: int, w: int) -> Config:
    """What the library does when no option is given: b = min(w, 64), look-ahead auto."""
    return Config(min(w, 64), -1, 0)


def candidates(op: str, m: int, n: int, w: int, sms: int = 152) -> list[Config]:
    """Candidate configurations of one size class: b from powers of two up to w (and w
    itself), with and without look-ahead, all SMs or half of them for the panel, and for
    sy2sb with 3b <= w look-ahead depth 2 (Variant V1)."""
    bs = sorted({b for b in (8, 16, 32, 64, 128, w) if 8 <= b <= w and b < max(n - w, 2)} or {min(w, max(1, n))})
    out = []
    for b in bs:
        for la in (0, -1):
            for pc in (0, sms // 2):
                out.append(Config(b, la, pc))
        if op == "sy2sb" and 3 * b <= w:
            for pc in (0, sms // 2):
                out.append(Config(b, 1, pc, 2))
    return out


def size_class(op: str, m: int, n: int, w: int, precision: str) -> str:
    """Plan-cache key: the operation, precision, w and m, n rounded up to powers of two."""
    p2 = lambda x: 1 << max(0, math.ceil(math.log2(max(x, 1))))
    return f"{op}/{precision}/m{p2(m)}/n{p2(n)}/w{w}"


def features(op: str, m: int, n: int, w: int, cfg: Config, precision: str, sms: int = 152) -> np.ndarray:
    """Inputs of the cost model, each of order one: log sizes, log w and b, b/w, the
    look-ahead flag, the panel's share of the SMs, the operation and the precision."""
    pc = cfg.panel_ctas if cfg.panel_ctas > 0 else sms
    return np.array([
        math.log2(max(n, 1)) / 8.0 - 1.0,
        math.log2(max(m, 1)) / 8.0 - 1.0,
        math.log2(w) / 4.0 - 1.0,
        math.log2(cfg.b) / 4.0 - 1.0,
        cfg.b / w,
        float(cfg.depth) if cfg.lookahead != 0 else 0.0,
        pc / sms,
        1.0 if op == "ge2gb" else 0.0,
        PRECISION_IDS.get(precision, 2) / 2.0,
    ], dtype=np.float32)


# ------------------------------------------------------------------ cost model
class CostModel:
    """Perceptron (two tanh layers of ``hidden`` units) predicting standardised log run
    time; trained with full-batch Adam, all arithmetic in the library's CUDA kernels."""

    def __init__(self, hidden: int = 32, seed: int = 0):
        self.D, self.H, self.seed = N_FEATURES, hidden, seed
        self.params = None
        self.mu, self.sigma = 0.0, 1.0

    def _init(self):
        import torch

        from . import bandred_mlp_param_count

        P = bandred_mlp_param_count(self.D, self.H)
        r = np.random.Generator(np.random.PCG64(self.seed))
        p = np.zeros(P, dtype=np.float32)
        o = 0
        for fan_in, fan_out in ((self.D, self.H), (None, self.H), (self.H, self.H), (None, self.H), (self.H, 1),
                                (None, 1)):
            cnt = (fan_in or 1) * fan_out
            if fan_in is not None:
                p[o:o + cnt] = r.standard_normal(cnt) * math.sqrt(1.0 / fan_in)
            o += cnt
        self.params = torch.from_numpy(p).cuda()

    def fit(self, X: np.ndarray, ms: np.ndarray, steps: int = 1500, lr: float = 3e-3) -> list:
        """Fits log(ms); returns the loss at the first and last step."""
        import torch

        from . import BandredError, bandred_mlp_adam, bandred_mlp_loss_grad, bandred_mlp_workspace

        y = np.log(np.asarray(ms, dtype=np.float64))
        self.mu, self.sigma = float(y.mean()), float(y.std() or 1.0)
        t = torch.from_numpy(((y - self.mu) / self.sigma).astype(np.float32)).cuda()
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        rows = Xd.shape[0]
        self._init()
        P = self.params.numel()
        m = torch.zeros(P, dtype=torch.float32, device="cuda")
        v = torch.zeros_like(m)
        g = torch.zeros_like(m)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        work = torch.empty(bandred_mlp_workspace(self.D, self.H, rows), dtype=torch.uint8, device="cuda")
        out = []
        for k in range(1, steps + 1):
            rc = bandred_mlp_loss_grad(self.D, self.H, self.params, Xd, t, rows, g, loss, work)
            if rc != 0:
                raise BandredError(rc, "bandred_mlp_loss_grad")
            if k == 1:
                out.append(float(loss.item()))
            rc = bandred_mlp_adam(P, self.params, g, m, v, k, lr)
            if rc != 0:
                raise BandredError(rc, "bandred_mlp_adam")
        rc = bandred_mlp_loss_grad(self.D, self.H, self.params, Xd, t, rows, g, loss, work)
        out.append(float(loss.item()))
        return out

    def predict_ms(self, X: np.ndarray) -> np.ndarray:
        import torch

        from . import BandredError, bandred_mlp_forward

        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        y = torch.zeros(Xd.shape[0], dtype=torch.float32, device="cuda")
        rc = bandred_mlp_forward(self.D, self.H, self.params, Xd, Xd.shape[0], y)
        if rc != 0:
            raise BandredError(rc, "bandred_mlp_forward")
        return np.exp(y.cpu().numpy().astype(np.float64) * self.sigma + self.mu)

    def state(self) -> dict:
        return {"D": self.D, "H": self.H, "mu": self.mu, "sigma": self.sigma,
                "params": self.params.cpu().numpy().tolist()}


# ------------------------------------------------------------------ selection (host logic)
def pick(cands: list[Config], timed_ms: dict, predicted_ms=None, budget: int | None = None) -> list[Config]:
    """The candidates to time: all of them without a model or budget, else the `budget`
    best-ranked by the model (ties keep candidate order)."""
    if predicted_ms is None or budget is None or budget >= len(cands):
        return list(cands)
    order = sorted(range(len(cands)), key=lambda i: (predicted_ms[i], i))
    return [cands[i] for i in order[:max(1, budget)]]


def records_to_arrays(records: list[dict]):
    X = np.stack([features(r["op"], r["m"], r["n"], r["w"],
                           Config(r["b"], r["lookahead"], r["panel_ctas"], r.get("depth", 1)), r["precision"])
                  for r in records])
    return X, np.array([r["ms"] for r in records], dtype=np.float64)


# ------------------------------------------------------------------ timing on the GPU
def time_config(op: str, m: int, n: int, w: int, cfg: Config, precision: str, A0, reps: int = 3) -> float:
    """Median CUDA-event time (ms) of one reduction with configuration cfg; A0 (device,
    column-major) is restored before every run outside the timed region."""
    import torch

    from . import (BandredError, bandred_ge2gb_ex, bandred_ge2gb_workspace, bandred_sy2sb_ex,
                   bandred_sy2sb_workspace, make_opts)

    dev = A0.device
    o = make_opts(b=cfg.b, lookahead=cfg.lookahead, precision=precision, panel_ctas=cfg.panel_ctas,
                  depth=cfg.depth)
    A = torch.empty_like(A0)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    if op == "sy2sb":
        tau = torch.zeros(max(n - w, 1), dtype=torch.float64, device=dev)
        work = torch.empty(bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device=dev)
        call = lambda: bandred_sy2sb_ex(A, w, tau, o, work, st, s)
    else:
        tq = torch.zeros(n, dtype=torch.float64, device=dev)
        tp = torch.zeros(max(n - w, 1), dtype=torch.float64, device=dev)
        work = torch.empty(bandred_ge2gb_workspace(m, n, w, o), dtype=torch.uint8, device=dev)
        call = lambda: bandred_ge2gb_ex(A, w, tq, tp, o, work, st, s)
    times = []
    for k in range(reps + 1):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        rc = call()
        e1.record(s)
        if rc != 0:
            raise BandredError(rc, f"{op} {cfg}")
        torch.cuda.synchronize(dev)
        if k > 0:
            times.append(e0.elapsed_time(e1))
    if int(st.item()) != 0:
        raise BandredError(int(st.item()), f"{op} {cfg} device status")
    return float(np.median(times))


def make_input(op: str, m: int, n: int, seed: int = 0):
    """Seeded N(0,1) test matrix on the device (symmetrised for sy2sb), column-major."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    if op == "sy2sb":
        G = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
        return ((G + G.t()) * 0.5).t().contiguous().t()
    return torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g).t()


PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "sweep_bf16x6_gb300.json")
_packaged = None


def packaged_plans() -> dict:
    """Plans of the sweep shipped with the package (every candidate of 27 size classes
    timed on a GB300: ``python -m paper_1709_00302_gb300.tune sweep``)."""
    global _packaged
    if _packaged is None:
        _packaged = {}
        if os.path.exists(PACKAGED):
            with open(PACKAGED) as f:
                _packaged = json.load(f).get("plans", {})
    return _packaged


class Tuner:
    """Plan cache (JSON) of the fastest configuration per size class, filled by timing."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("BANDRED_PLAN_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "paper_1709_00302_gb300", "plans.json")
        self.plans, self.records = {}, []
        if os.path.exists(self.path):
            with open(self.path) as f:
                d = json.load(f)
            self.plans, self.records = d.get("plans", {}), d.get("records", [])

    def save(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"plans": self.plans, "records": self.records}, f, indent=1)
        os.replace(tmp, self.path)

    def lookup(self, op: str, m: int, n: int, w: int, precision: str) -> Config | None:
        """The cached plan of the size class, else the packaged plan measured on GB300."""
        key = size_class(op, m, n, w, precision)
        p = self.plans.get(key) or packaged_plans().get(key)
        return None if p is None else Config(p["b"], p["lookahead"], p["panel_ctas"], p.get("depth", 1))

    def opts(self, op: str, m: int, n: int, w: int, precision: str):
        """bandred_opts of the cached plan (the library defaults when the class is untuned)."""
        from . import make_opts

        c = self.lookup(op, m, n, w, precision) or default_config(op, m, n, w)
        return make_opts(b=c.b, lookahead=c.lookahead, precision=precision, panel_ctas=c.panel_ctas, depth=c.depth)

    def tune(self, op: str, m: int, n: int, w: int, precision: str = "bf16x6", model: CostModel | None = None,
             budget: int | None = None, reps: int = 3, seed: int = 0) -> Config:
        cands = candidates(op, m, n, w)
        pred = None
        if model is not None and budget is not None:
            pred = model.predict_ms(np.stack([features(op, m, n, w, c, precision) for c in cands]))
        chosen = pick(cands, {}, pred, budget)
        A0 = make_input(op, m, n, seed)
        best, best_ms = None, float("inf")
        for c in chosen:
            ms = time_config(op, m, n, w, c, precision, A0, reps)
            self.records.append(dict(op=op, precision=precision, m=m, n=n, w=w, ms=ms, **asdict(c)))
            if ms < best_ms:
                best, best_ms = c, ms
        self.plans[size_class(op, m, n, w, precision)] = dict(ms=best_ms, **asdict(best))
        return best


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1709_00302_gb300.tune")
    sub = ap.add_subparsers(dest="cmd", required=True)
    sw = sub.add_parser("sweep", help="time every candidate of a grid of size classes")
    sw.add_argument("--out", required=True)
    sw.add_argument("--precision", default="bf16x6")
    sw.add_argument("--sy-n", default="512,1024,2048,4096,8192")
    sw.add_argument("--ge-n", default="512,1024,2048,4096")
    sw.add_argument("--w", default="32,64,128")
    sw.add_argument("--reps", type=int, default=3)
    tu = sub.add_parser("tune", help="tune one size class into the plan cache")
    tu.add_argument("--op", default="sy2sb", choices=OPS)
    tu.add_argument("--m", type=int, default=0)
    tu.add_argument("--n", type=int, required=True)
    tu.add_argument("--w", type=int, required=True)
    tu.add_argument("--precision", default="bf16x6")
    tu.add_argument("--cache", default=None)
    a = ap.parse_args(argv)
    from . import build, lib

    build()
    lib()
    if a.cmd == "sweep":
        t = Tuner(a.out)
        ws = [int(x) for x in a.w.split(",")]
        for op, ns in (("sy2sb", a.sy_n), ("ge2gb", a.ge_n)):
            for n in [int(x) for x in ns.split(",") if x]:
                for w in ws:
                    if w >= n // 2:
                        continue
                    best = t.tune(op, n, n, w, a.precision, reps=a.reps)
                    print(op, n, w, best, flush=True)
                    t.save()
        return 0
    t = Tuner(a.cache)
    best = t.tune(a.op, a.m or a.n, a.n, a.w, a.precision)
    t.save()
    print(best)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
