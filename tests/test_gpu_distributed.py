"""The merge tree split over ranks with the CUDA library as the numerical
backend (hps_merge_boxes with the subtree root maps, hps_solve_boxes for the
grid of rank boxes, hps_solve per box), every rank simulated in this process
on one GPU (distributed.run_in_process: each step completes before the
next, no kernel waits on another rank).  The solution must equal the
single-plan hps_merge / hps_solve on the whole grid and the oracle's
single-rank merge tree to 1e-12; the root map of hps_merge_boxes must equal
the oracle's root T and h."""

import numpy as np
import pytest
import torch

import oracle.hps_oracle as O
from gpu_cases import gpu_inputs
from paper_2211_14969_b300 import distributed as D
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu


class Box:
    """The leaves of one rank box, as a workload for gpu_inputs."""

    def __init__(self, w, leaves):
        self.m, self.kappa = w.m, w.kappa
        self.p = w.p[leaves]
        self.box = w.boxes()[leaves]
        self.coefficients, self.body_load = w.coefficients, w.body_load

    def boxes(self):
        return self.box


def workload(nx, ny, p):
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=15.0, seed=3, m=1)
    w.dirichlet = "planewave"
    return w


def outer_g(w):
    p = int(w.p[0])
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    return np.array([w.dirichlet_data(*O.key_coords(p, k, w.nx, w.ny)) for k in keys])


def single_plan(w):
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
    u = plan.solve(torch.from_numpy(outer_g(w)).cuda(), out["S"], out["W"], 1)
    torch.cuda.synchronize()
    return u.cpu().numpy().reshape(w.n_leaves, -1), plan, out


@pytest.mark.parametrize("world", [2, 4, 8])
def test_split_equals_single_plan(world):
    w = workload(8, 8, 10)
    p, q = 10, 8
    part = D.Partition(w.nx, w.ny, world)
    backends = []
    for r in range(world):
        lv = part.leaves(r)
        be = D.LibraryBackend(p, w.kappa, part, r, w.boxes()[lv])
        coef, f, _ = gpu_inputs(Box(w, lv), be.plan)
        be.condense(coef, f, 1)
        backends.append(be)
    sols = D.run_in_process(backends, part, q, outer_g(w)[:, None], 1)
    torch.cuda.synchronize()
    u_ref, plan, _ = single_plan(w)
    worst = 0.0
    for r, u in enumerate(sols):
        got = u.cpu().numpy().reshape(len(part.leaves(r)), -1)
        ref = u_ref[part.leaves(r)]
        worst = max(worst, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    assert worst < 1e-12, worst
    # and the oracle's single-rank tree on the same grid
    leaves = []
    for l in range(w.n_leaves):
        x, y = O.leaf_nodes(p, w.boxes()[l])
        leaves.append(O.condense_leaf(p, w.boxes()[l], w.coefficients(x, y), w.kappa, w.body_load(x, y)))
    levels = O.hps_upward(p, w.nx, w.ny, leaves)
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    sol = O.hps_downward(p, w.nx, w.ny, levels, leaves, dict(zip(keys, outer_g(w)[:, None])))
    ix = O.leaf_index_sets(p)
    for r, u in enumerate(sols):
        got = u.cpu().numpy().reshape(len(part.leaves(r)), p * p)
        for j, l in enumerate(part.leaves(r)):
            ref = np.zeros(p * p)
            ref[ix["B"]] = sol[l]["u_b"].ravel()
            ref[ix["I"]] = sol[l]["u_i"].ravel()
            assert np.linalg.norm(got[j] - ref) / np.linalg.norm(ref) < 1e-12, (world, l)
    for be in backends:
        be.close()
    plan.close()


def test_merge_boxes_root_map_matches_oracle():
    """hps_merge_boxes(..., root) on condensed leaves: the root's T and h
    against the oracle's root merge record (hps_merge stops before it)."""
    w = workload(4, 4, 8)
    p = 8
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    th = plan.merge_boxes(4, 4, 1, 1, out["T"], out["h"], 1, root=True)
    torch.cuda.synchronize()
    n = 2 * (4 + 4) * (p - 2)
    th = th.cpu().numpy().reshape(n, n + 1)
    leaves = []
    for l in range(w.n_leaves):
        x, y = O.leaf_nodes(p, w.boxes()[l])
        leaves.append(O.condense_leaf(p, w.boxes()[l], w.coefficients(x, y), w.kappa, w.body_load(x, y)))
    root = O.hps_upward(p, 4, 4, leaves)[-1][(0, 0)]
    assert np.linalg.norm(th[:, :n] - root["T"]) / np.linalg.norm(root["T"]) < 1e-12
    assert np.linalg.norm(th[:, n:] - root["h"]) / np.linalg.norm(root["h"]) < 1e-12
    with pytest.raises(hps.HpsError):   # a box grid needs one plan entry per box (nx*ny = n_leaves)
        plan.merge_boxes(2, 2, 2, 2, out["T"][: 4 * (2 * 4 * 6) ** 2], out["h"][: 4 * 2 * 4 * 6], 1)
    plan.close()
