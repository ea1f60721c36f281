"""The benchmark's exact setting asserted against the oracle.

bench.py times the full bumps_p20 launch (64 x 64 leaves, p = 20) and the
bumps_p30 launch (32 x 32 leaves, p = 30) with the refinement settings
bench.REFINE_TOL / bench.REFINE_KMAX and the FP64 fallback on (the plan
default).  Here the same launches are checked leaf by leaf against the FP64
oracle on 64 leaves each: the 16 worst-conditioned leaves of the workload
(tests/golden/worst_cond_leaves.json, written by make_worst_cond.py from the
oracle alone), the first and the last leaf of the library's work queue
(largest order first, index order within an order), and seeded random
leaves.  Bars per leaf and output (S, T, W, h): 1e-12 on the FP64 path,
1e-10 on the mixed path, the cond term only for near-resonant leaves
(gpu_cases.leaf_bar).
"""

import json
import os

import numpy as np
import pytest
import torch

import bench
from gpu_cases import assert_within, compare_leaves, gpu_inputs, oracle_pool
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-10}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worst_cond_leaves.json")


@pytest.fixture(scope="module")
def pool():
    p = oracle_pool()
    yield p
    p.close()
    p.join()


def chosen_leaves(w, name, n=64, n_worst=16):
    with open(GOLDEN) as fh:
        worst = [int(l) for l, _ in json.load(fh)[name]["worst"][:n_worst]]
    queue = np.argsort(-np.asarray(w.p), kind="stable")
    pick = set(worst) | {int(queue[0]), int(queue[-1])}
    rng = np.random.default_rng(2024)
    while len(pick) < n:
        pick.add(int(rng.integers(0, w.n_leaves)))
    return sorted(pick), worst


@pytest.mark.parametrize("name", ["bumps_p20", "bumps_p30"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bench_setting_full_launch(name, prec, pool):
    w = getattr(WL, name)()
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=w.m, prec=prec, tol=bench.REFINE_TOL, kmax=bench.REFINE_KMAX)
    torch.cuda.synchronize()
    info = out["info"].cpu().numpy()
    assert (info == 0).all(), np.unique(info, return_counts=True)
    if prec == "fp32":
        print(f"{name}: {plan.fallback_count()} of {w.n_leaves} leaves re-condensed in FP64")
    leaves, worst = chosen_leaves(w, name)
    assert len(leaves) >= 64 and set(worst) <= set(leaves)
    recs = compare_leaves(w, plan, out, leaves, TOL[prec], pool=pool)
    assert_within(recs)
    for k in ("S", "T", "h", "W"):
        assert torch.isfinite(out[k]).all(), k
    plan.close()
