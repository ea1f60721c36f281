"""Panel-width autotuning and CUDA-graph replay for hps_condense.

Both are host-side helpers around the C ABI: the autotuner times the
candidate LU panel widths of a plan with the library's own kernel timing
(hps_set_blocking + hps_set_timing / hps_phase_times) and keeps the fastest,
optionally remembering it in a JSON cache keyed by (orders present,
precision, m); CondenseGraph captures one hps_condense call (a memset and
one kernel) into a CUDA graph and replays it.
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
