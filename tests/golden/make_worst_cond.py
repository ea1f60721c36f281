"""Writes tests/golden/worst_cond_leaves.json: for each full-size workload,
the 2-norm condition number cond(A_ii) of every leaf's interior block,
summarised as the worst leaves (largest cond first) and the distribution.

A_ii comes from the oracle alone (oracle.hps_oracle.leaf_operator, the
collocation operator of Eq. (var_helm) in the form of Eq. (chain_rule) on
the Section 2 mesh), with the coefficients of the seeded workloads evaluated
at the oracle's own nodes.  The GPU parity tests use the list to pick the
leaves they compare (the worst-conditioned ones are where a wrong pivot or a
lost digit shows first) and to decide which leaves carry the cond(A_ii) eps
term in their bar.

Usage: python tests/golden/make_worst_cond.py [workload ...]
"""

import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "worst_cond_leaves.json")
NAMES = ("bumps_p20", "bumps_p30", "annulus_p24", "uneven", "psi_p20")
TOP = 32


def _init():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _conds(args):
    name, leaves = args
    import numpy as np

    import oracle.hps_oracle as O
    from paper_2211_14969_b300 import workloads as WL
    w = getattr(WL, name)()
    boxes = w.boxes()
    out = []
    for l in leaves:
        p = int(w.p[l])
        x, y = O.leaf_nodes(p, boxes[l])
        A, _, _, _ = O.leaf_operator(p, boxes[l], w.coefficients(x, y), w.kappa)
        I = O.leaf_index_sets(p)["I"]
        out.append((int(l), float(np.linalg.cond(A[np.ix_(I, I)]))))
    return out


def main(names):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    _init()
    import numpy as np

    from paper_2211_14969_b300 import workloads as WL
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count(), initializer=_init) as pool:
        for name in names:
            n = getattr(WL, name)().n_leaves
            chunks = [(name, list(range(s, min(n, s + 64)))) for s in range(0, n, 64)]
            res = [r for part in pool.map(_conds, chunks) for r in part]
            c = np.array([v for _, v in res])
            order = sorted(res, key=lambda t: -t[1])
            data[name] = {"n_leaves": n, "worst": [[l, v] for l, v in order[:TOP]],
                          "cond_max": float(c.max()), "cond_median": float(np.median(c)),
                          "cond_min": float(c.min()),
                          "count_above": {f"{t:g}": int((c > t).sum()) for t in (1e4, 1e5, 1e6, 1e7, 1e8)}}
            print(name, json.dumps({k: v for k, v in data[name].items() if k != "worst"}), flush=True)
            with open(OUT, "w") as fh:
                json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or NAMES)
