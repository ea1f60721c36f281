"""Shared helpers of the GPU parity tests: the same seeded workload evaluated
independently at the GPU library's node coordinates (for the CUDA path) and
at the oracle's node coordinates (for the oracle)."""

import numpy as np
import torch

import oracle.hps_oracle as O
from paper_2211_14969_b300 import hps

EPS = np.finfo(np.float64).eps


def gpu_inputs(w, plan, coef_fn=None, load_fn=None):
    """Coefficients and body loads evaluated at the nodes the library reports."""
    lay = plan.layout
    xy = plan.leaf_nodes().cpu().numpy()
    coef = np.empty(int(6 * lay.o_p2[-1]))
    f = np.empty(int(lay.o_p2[-1] * w.m)) if w.m > 0 else None
    for l in range(lay.n_leaves):
        p2 = int(lay.p2[l])
        o = int(lay.o_p2[l])
        x = xy[2 * o: 2 * o + p2]
        y = xy[2 * o + p2: 2 * o + 2 * p2]
        c = (coef_fn or w.coefficients)(x, y)
        coef[6 * o: 6 * o + 6 * p2] = np.asarray(c).ravel()
        if f is not None:
            f[o * w.m: (o + p2) * w.m] = np.asarray((load_fn or w.body_load)(x, y)).reshape(p2, w.m).ravel()
    t = lambda a: None if a is None else torch.from_numpy(a).cuda()
    return t(coef), t(f), xy


def oracle_leaf(w, l, coef_fn=None, load_fn=None):
    p = int(w.p[l])
    box = w.boxes()[l]
    x, y = O.leaf_nodes(p, box)
    coef = (coef_fn or w.coefficients)(x, y)
    f = (load_fn or w.body_load)(x, y).reshape(p * p, -1) if w.m > 0 else None
    return O.condense_leaf(p, box, coef, w.kappa, f)


def leaf_slices(lay, out, l, m):
    ni, nb = int(lay.ni[l]), int(lay.nb[l])
    res = {}
    if out.get("S") is not None:
        res["S"] = out["S"][int(lay.o_sb[l]): int(lay.o_sb[l + 1])].reshape(ni, nb)
    res["T"] = out["T"][int(lay.o_bb[l]): int(lay.o_bb[l + 1])].reshape(nb, nb)
    if m > 0:
        res["h"] = out["h"][int(lay.o_nb[l]) * m: int(lay.o_nb[l + 1]) * m].reshape(nb, m)
        if out.get("W") is not None:
            res["W"] = out["W"][int(lay.o_ni[l]) * m: int(lay.o_ni[l + 1]) * m].reshape(ni, m)
    return res


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def compare_leaves(w, plan, out, leaves, tol_fp64, cond_factor=10.0, coef_fn=None, load_fn=None):
    """Per-leaf relative Frobenius errors of every output against the oracle.

    The bar for a leaf is max(tol, cond_factor * cond(A_ii) * eps): two
    correct FP64 eliminations of the same system with different pivoting or
    summation order may differ by about cond * eps.  Returns the records."""
    recs = []
    cpu = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    for l in leaves:
        ref = oracle_leaf(w, l, coef_fn, load_fn)
        got = leaf_slices(plan.layout, cpu, l, w.m)
        cond = np.linalg.cond(ref["A_ii"])
        bar = max(tol_fp64, cond_factor * cond * EPS)
        rec = {"leaf": l, "cond": cond, "bar": bar}
        for k in ("S", "T", "W", "h"):
            if k in got and k in ref:
                rec[k] = relerr(got[k], ref[k])
        recs.append(rec)
    return recs


def assert_within(recs):
    bad = [r for r in recs if any(r[k] > r["bar"] for k in ("S", "T", "W", "h") if k in r)]
    assert not bad, bad[:3]
