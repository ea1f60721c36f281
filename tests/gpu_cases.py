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


# Interior blocks more ill-conditioned than this belong to leaves near an
# interior Dirichlet resonance.  Two correct FP64 eliminations of the same
# system (other pivot or summation order) may differ by about
# cond(A_ii) eps; above cond = 1e5 the bound 10 cond eps exceeds 2e-10, more
# than even the mixed path's bar.  Only such leaves get the cond term in
# their bar, and they are reported separately; every other leaf is held to
# the fixed bar (1e-12 on the FP64 path, 1e-10 on the mixed paths).  Of the
# full-size workloads, bumps_p20 has none (cond <= 5.2e3), bumps_p30 12 of
# 1024 (tests/golden/worst_cond_leaves.json).
COND_FLAG = 1e5


def leaf_bar(tol, cond, cond_factor=10.0):
    """(bar, flagged) of one leaf: the fixed bar, or for a near-resonant
    leaf (cond(A_ii) > COND_FLAG) max(tol, cond_factor cond eps)."""
    if cond > COND_FLAG:
        return max(tol, cond_factor * cond * EPS), True
    return tol, False


def _oracle_outputs(w, l, coef_fn=None, load_fn=None):
    ref = oracle_leaf(w, l, coef_fn, load_fn)
    cond = float(np.linalg.cond(ref["A_ii"]))
    return {k: ref[k] for k in ("S", "T", "W", "h") if k in ref}, cond


def _oracle_job(args):
    w, l = args
    return l, _oracle_outputs(w, l)


def _one_blas_thread():
    import os
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass


def oracle_pool(workers=None):
    """A pool of spawned processes (one BLAS thread each) for the oracle's
    per-leaf work; spawned, not forked, since the parent holds a CUDA
    context."""
    import multiprocessing as mp
    import os
    # read by the workers when they import numpy (set before they start)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(workers or max(1, min(32, os.cpu_count() or 1)),
                                        initializer=_one_blas_thread)


def compare_leaves(w, plan, out, leaves, tol, cond_factor=10.0, coef_fn=None, load_fn=None, pool=None):
    """Per-leaf relative Frobenius errors of every output against the oracle.

    The bar of a leaf is the fixed tol, or max(tol, cond_factor cond(A_ii)
    eps) when its interior block is near-resonant (leaf_bar).  With a pool
    (oracle_pool; only for workloads without custom coefficient or load
    functions) the oracle leaves are computed in parallel.  Returns the
    records."""
    recs = []
    cpu = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    leaves = [int(l) for l in leaves]
    if pool is not None and coef_fn is None and load_fn is None:
        refs = dict(pool.map(_oracle_job, [(w, l) for l in leaves]))
    else:
        refs = {l: _oracle_outputs(w, l, coef_fn, load_fn) for l in leaves}
    for l in leaves:
        ref, cond = refs[l]
        got = leaf_slices(plan.layout, cpu, l, w.m)
        bar, flagged = leaf_bar(tol, cond, cond_factor)
        rec = {"leaf": l, "cond": cond, "bar": bar, "flagged": flagged}
        for k in ("S", "T", "W", "h"):
            if k in got and k in ref:
                rec[k] = relerr(got[k], ref[k])
        recs.append(rec)
    return recs


def assert_within(recs):
    """Every output of every leaf within its bar; near-resonant leaves (the
    ones whose bar carries the cond term) are printed separately."""
    outs = ("S", "T", "W", "h")
    flagged = [r for r in recs if r.get("flagged")]
    plain = [r for r in recs if not r.get("flagged")]
    if plain:
        worst = {k: max(r[k] for r in plain if k in r) for k in outs if any(k in r for r in plain)}
        print(f"{len(plain)} leaves at the fixed bar {plain[0]['bar']:.0e}: max errors "
              + ", ".join(f"{k} {v:.1e}" for k, v in worst.items()))
    for r in flagged:
        print(f"near-resonant leaf {r['leaf']}: cond(A_ii) {r['cond']:.2e}, bar {r['bar']:.1e}, errors "
              + ", ".join(f"{k} {r[k]:.1e}" for k in outs if k in r))
    bad = [r for r in recs if any(r[k] > r["bar"] for k in outs if k in r)]
    assert not bad, bad[:3]
