"""Panel-width autotuning and CUDA-graph replay for hps_condense.

Both are host-side helpers around the C ABI: the autotuner times the
candidate LU panel widths of a plan with the library's own kernel timing
(hps_set_blocking + hps_set_timing / hps_phase_times) and keeps the fastest,
optionally remembering it in a JSON cache keyed by (orders present,
precision, m); autotune_orders times them per order (each order's leaves
alone, cached per (p, precision, m)) and sets the fused plan's width from
the per-order times.  CondenseGraph captures one hps_condense call (a
memset and one kernel) into a CUDA graph and replays it: the library does
not capture by itself, capture is the caller's, and after one eager call
with the same plan, precision and m the call allocates nothing and can be
captured (hps_set_blocking documents this).
"""

import json
import os

import numpy as np

from . import hps

CANDIDATES = {"fp64": (16, 8, 4), "fp32": (32, 16, 8)}


def cache_key(plan, prec, m):
    orders = sorted(set(int(v) for v in np.asarray(plan.layout.p)))
    return f"p={','.join(map(str, orders))};prec={prec};m={int(m)}"


def autotune(plan, coef, f, m, prec="fp32", tol=1e-12, kmax=6, reps=2, cache_path=None, out=None):
    """Pick the fastest panel width for this plan and precision; returns
    (width, {width: ms}).  Widths that do not fit an SM are skipped.  The
    choice stays set on the plan."""
    import torch
    key = cache_key(plan, prec, m)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    if key in cache:
        plan.set_blocking(prec, int(cache[key]["nb"]))
        return int(cache[key]["nb"]), {int(k): v for k, v in cache[key]["ms"].items()}
    times = {}
    for nb in CANDIDATES[prec]:
        plan.set_blocking(prec, nb)
        try:
            o = plan.condense(coef, f, m=m, prec=prec, tol=tol, kmax=kmax, out=out)   # warm-up
        except hps.HpsError:
            continue
        out = o
        torch.cuda.synchronize()
        plan.set_timing(True)
        for _ in range(reps):
            plan.condense(coef, f, m=m, prec=prec, tol=tol, kmax=kmax, out=out)
        t = plan.phase_times()
        plan.set_timing(False)
        times[nb] = t[0] / t[1]
    if not times:
        plan.set_blocking(prec, 0)
        raise hps.HpsError(hps.HPS_ERR_ARG, "autotune: no panel width fits")
    best = min(times, key=times.get)
    plan.set_blocking(prec, best)
    if cache_path:
        cache[key] = {"nb": best, "ms": {str(k): v for k, v in times.items()}}
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return best, times


def order_key(p, prec, m):
    return f"p={int(p)};prec={prec};m={int(m)}"


def _order_subsets(plan, coef, f, m):
    """Per order present: (p, leaf indices, coefficients, loads) of that
    order's leaves, gathered from the plan's packed arrays."""
    import torch
    lay = plan.layout
    out = []
    for p in sorted(set(int(v) for v in np.asarray(lay.p))):
        idx = np.flatnonzero(np.asarray(lay.p) == p)
        gx = np.concatenate([np.arange(6 * int(lay.o_p2[l]), 6 * int(lay.o_p2[l + 1])) for l in idx])
        c = coef[torch.from_numpy(gx).to(coef.device)]
        fs = None
        if f is not None and m > 0:
            gf = np.concatenate([np.arange(int(lay.o_p2[l]) * m, int(lay.o_p2[l + 1]) * m) for l in idx])
            fs = f[torch.from_numpy(gf).to(f.device)]
        out.append((p, idx, c, fs))
    return out


def autotune_orders(plan, boxes, kappa, coef, f, m, prec="fp32", tol=1e-12, kmax=6, reps=2, cache_path=None):
    """Per-order tuning for a plan of mixed orders.  Every candidate panel
    width is timed on each order's leaves alone (a sub-plan per order, the
    library's own kernel timing), and the result is cached per (p, prec, m);
    the fused plan then gets the width whose per-order times, summed over
    the orders present, are least (the orders share one launch and its
    shared-memory layout).  Returns (width, {p: {width: ms}})."""
    import torch
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    per = {}
    for p, idx, c, fs in _order_subsets(plan, coef, f, m):
        key = order_key(p, prec, m)
        if key in cache:
            per[p] = {int(k): v for k, v in cache[key].items()}
            continue
        sub = hps.Plan(np.full(len(idx), p, dtype=np.int32), np.asarray(boxes)[idx], kappa)
        times, out = {}, None
        for nb in CANDIDATES[prec]:
            sub.set_blocking(prec, nb)
            try:
                out = sub.condense(c, fs, m=m, prec=prec, tol=tol, kmax=kmax, out=out)
            except hps.HpsError:
                continue
            torch.cuda.synchronize()
            sub.set_timing(True)
            for _ in range(reps):
                sub.condense(c, fs, m=m, prec=prec, tol=tol, kmax=kmax, out=out)
            t = sub.phase_times()
            sub.set_timing(False)
            times[nb] = t[0] / t[1]
        sub.close()
        per[p] = times
        cache[key] = {str(k): v for k, v in times.items()}
    common = set.intersection(*(set(t) for t in per.values())) if per else set()
    if not common:
        raise hps.HpsError(hps.HPS_ERR_ARG, "autotune_orders: no panel width fits every order")
    best = min(common, key=lambda nb: sum(per[p][nb] for p in per))
    plan.set_blocking(prec, best)
    if cache_path:
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return best, per


class CondenseGraph:
    """One hps_condense call captured into a CUDA graph.

    The first (eager) call sizes the plan's workspace so the captured call
    allocates nothing; replay() re-runs the condensation on whatever the
    captured input and output tensors hold at that time."""

    def __init__(self, plan, coef, f, m, prec="fp32", tol=1e-12, kmax=6, out=None):
        import torch
        self.plan = plan
        self.out = plan.condense(coef, f, m=m, prec=prec, tol=tol, kmax=kmax, out=out)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            plan.condense(coef, f, m=m, prec=prec, tol=tol, kmax=kmax, out=self.out)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
        return self.out
