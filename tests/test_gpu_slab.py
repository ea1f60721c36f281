"""GPU parity of SlabLU (hps_slab_factor / hps_slab_solve; Section 2, the
slab block form of Eq. (dell1)) against the oracle's SlabLU on the reduced
system of Eq. (hps_reduced) (oracle.slab_downward) and against the merge
tree on the GPU (hps_merge / hps_solve), element by element per leaf;
and, at the full 64 x 64, p = 20 size, the flux continuity of the solution
across every interior leaf edge (the reduced system's rows)."""

import numpy as np
import pytest
import torch

import oracle.hps_oracle as O
from gpu_cases import gpu_inputs
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu


def workload(nx, ny, p, kappa=15.0):
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=kappa, seed=3, m=1)
    w.dirichlet = "planewave"
    return w


def outer_g(w):
    p = int(w.p[0])
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    return keys, np.array([w.dirichlet_data(*O.key_coords(p, k, w.nx, w.ny)) for k in keys])


def gpu_both(w, s):
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    g = torch.from_numpy(outer_g(w)[1]).cuda()
    plan.slab_factor(w.nx, w.ny, s, out["T"], out["h"], 1)
    u_slab = plan.slab_solve(g, out["S"], out["W"], 1)
    u_slab2 = plan.slab_solve(g, out["S"], out["W"], 1)       # a second solve reuses the factors
    plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
    u_tree = plan.solve(g, out["S"], out["W"], 1)
    torch.cuda.synchronize()
    assert torch.equal(u_slab, u_slab2)
    return plan, out, u_slab.cpu().numpy(), u_tree.cpu().numpy()


@pytest.mark.parametrize("nx,ny,s", [(8, 8, 2), (8, 8, 4), (8, 8, 8), (16, 4, 4), (4, 16, 2)])
def test_slab_solve_matches_oracle_and_tree(nx, ny, s):
    p = 10
    w = workload(nx, ny, p)
    plan, out, u_slab, u_tree = gpu_both(w, s)
    n = w.n_leaves
    assert np.linalg.norm(u_slab - u_tree) / np.linalg.norm(u_tree) < 1e-12
    leaves = []
    for l in range(n):
        x, y = O.leaf_nodes(p, w.boxes()[l])
        leaves.append(O.condense_leaf(p, w.boxes()[l], w.coefficients(x, y), w.kappa, w.body_load(x, y)))
    keys, g = outer_g(w)
    sol = O.slab_downward(p, nx, ny, s, leaves, {k: np.atleast_1d(v) for k, v in zip(keys, g)})
    ix = O.leaf_index_sets(p)
    got = u_slab.reshape(n, p * p)
    for l in range(n):
        ref = np.zeros(p * p)
        ref[ix["B"]] = sol[l]["u_b"].ravel()
        ref[ix["I"]] = sol[l]["u_i"].ravel()
        assert np.linalg.norm(got[l] - ref) / np.linalg.norm(ref) < 1e-12, l
    plan.close()


def test_slab_arguments():
    w = workload(4, 4, 6)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    g = torch.zeros(2 * 8 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(hps.HpsError):
        plan.slab_solve(g, out["S"], out["W"], 1)            # before the factorization
    for s in (3, 1, 8):
        with pytest.raises(hps.HpsError):
            plan.slab_factor(4, 4, s, out["T"], out["h"], 1)
    plan.close()


def test_full_size_slab_against_tree():
    """64 x 64 leaves, p = 20, kappa = 200 (bumps_p20), slabs of 8 leaf
    columns (7 interfaces of 1152 nodes): SlabLU and the merge tree solve
    the same reduced system in two elimination orders; the solutions agree
    to the system's conditioning, and SlabLU's satisfies flux continuity on
    every interior edge to rounding."""
    import bench
    w = WL.bumps_p20()
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f = bench.make_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    q = 18
    g = torch.from_numpy(np.random.default_rng(7).standard_normal(2 * (64 + 64) * q)).cuda()
    plan.slab_factor(64, 64, 8, out["T"], out["h"], 1)
    u_slab = plan.slab_solve(g, out["S"], out["W"], 1)
    torch.cuda.synchronize()
    mismatch = bench.flux_mismatch(w, plan.layout, out, u_slab, 1)
    plan.merge(64, 64, out["T"], out["h"], 1)
    u_tree = plan.solve(g, out["S"], out["W"], 1)
    torch.cuda.synchronize()
    diff = float((u_slab - u_tree).norm() / u_tree.norm())
    print(f"slab vs tree {diff:.2e}, flux mismatch {mismatch:.2e}")
    assert mismatch < 1e-12 and diff < 1e-9
    plan.close()


def test_large_interface_narrow_panels():
    """4 x 128 leaves, p = 20, slabs of 2 leaf columns: one interface of
    2304 nodes, above what a 16-column panel of the split solve holds in
    shared memory, so it factors with 8-column panels.  Against the merge
    tree; the flux continuity of SlabLU's solution with the default tensor
    path (the slab merges on the tensor cores, the interface solve on the
    FP64 pipe) within a few times that of the all-FP64 factorization; with
    the interface solve's right-hand side on the tensor cores as well
    (mode 2) it is measurably larger here (the columns of [-U | I] span many
    orders of magnitude) but still far inside the solve's bar."""
    import bench
    w = workload(4, 128, 20)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    g = torch.from_numpy(outer_g(w)[1]).cuda()
    plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
    u_tree = plan.solve(g, out["S"], out["W"], 1).clone()
    mism, diff = {}, {}
    for mode in (0, 1, 2):
        plan.set_merge_tensor(mode)
        plan.slab_factor(w.nx, w.ny, 2, out["T"], out["h"], 1)
        u = plan.slab_solve(g, out["S"], out["W"], 1)
        torch.cuda.synchronize()
        mism[mode] = bench.flux_mismatch(w, plan.layout, out, u, 1)
        diff[mode] = float((u - u_tree).norm() / u_tree.norm())
    print(f"slab vs tree {diff}, flux mismatch {mism}")
    assert max(diff.values()) < 1e-10
    assert mism[0] < 1e-10 and mism[1] < max(4 * mism[0], 1e-12) and mism[2] < 1e-10
    plan.close()
