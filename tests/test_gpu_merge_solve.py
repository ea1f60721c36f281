"""GPU parity of the full HPS pipeline (condense + merge + solve) on uniform
leaf grids against the CPU oracle's merge tree, the brute-force dense global
collocation solve, closed-form solutions and manufactured polynomials."""

import numpy as np
import pytest
import torch

import oracle.hps_oracle as O
from gpu_cases import gpu_inputs
from manufactured import random_coef, random_poly
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu


def gpu_pipeline(w, prec="fp64", coef_fn=None, load_fn=None, g_fn=None, split=None, tensor=True):
    p = int(w.p[0])
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    if split is not None:
        plan.set_merge_split(split)
    plan.set_merge_tensor(tensor)
    coef, f, _ = gpu_inputs(w, plan, coef_fn, load_fn)
    out = plan.condense(coef, f, m=1, prec=prec, tol=1e-13, kmax=8)
    plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    # Dirichlet data at the outer edge nodes, [W, E, S, N] of the root box
    g = np.array([(g_fn or w.dirichlet_data)(*O.key_coords(p, k, w.nx, w.ny)) for k in keys], dtype=np.float64)
    u = plan.solve(torch.from_numpy(g).cuda(), out["S"], out["W"], 1)
    torch.cuda.synchronize()
    assert (out["info"].cpu().numpy() == 0).all()
    return u.cpu().numpy().reshape(w.n_leaves, p * p)


def oracle_pipeline(w, coef_fn=None, load_fn=None, g_fn=None):
    p = int(w.p[0])
    boxes = w.boxes()
    coefs, fs = [], []
    for box in boxes:
        x, y = O.leaf_nodes(p, box)
        coefs.append((coef_fn or w.coefficients)(x, y))
        fs.append((load_fn or w.body_load)(x, y).reshape(p * p, 1))
    leaves = [O.condense_leaf(p, boxes[l], coefs[l], w.kappa, fs[l]) for l in range(w.n_leaves)]
    levels = O.hps_upward(p, w.nx, w.ny, leaves)
    gk = {k: np.atleast_1d((g_fn or w.dirichlet_data)(*O.key_coords(p, k, w.nx, w.ny)))
          for k in O.outer_boundary_keys(p, w.nx, w.ny)}
    sol = O.hps_downward(p, w.nx, w.ny, levels, leaves, gk)
    return sol, coefs, fs


def grid_from_sol(sol, p):
    ix = O.leaf_index_sets(p)
    out = np.zeros((len(sol), p * p))
    for l, s in enumerate(sol):
        out[l, ix["B"]] = s["u_b"].ravel()
        out[l, ix["I"]] = s["u_i"].ravel()
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_planewave_pipeline_matches_oracle_dense_and_closed_form():
    """kappa = 20, b = 1, p = 10, 8 x 8 leaves, Dirichlet data of the plane
    wave sin(kappa (0.6 x + 0.8 y)): condense, merge, solve on the GPU."""
    w = WL.planewave()
    p = 10
    u_gpu = gpu_pipeline(w)
    sol, coefs, fs = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert rel(u_gpu[:, mask], u_ora[:, mask]) < 1e-12
    dense, res = O.global_dense_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    assert rel(u_gpu[:, mask], grid_from_sol(dense, p)[:, mask]) < 1e-11
    exact = np.stack([w.dirichlet_data(*O.leaf_nodes(p, b)) for b in w.boxes()])
    err = rel(u_gpu[:, mask], exact[:, mask])
    assert err < 1e-4, err
    assert np.all(u_gpu[:, ~mask] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_manufactured_polynomial_is_exact(prec):
    """A tensor polynomial of degree p-1 is the exact discrete solution for
    any coefficient samples: the GPU pipeline reproduces it to rounding."""
    p, nx, ny, kappa = 8, 4, 4, 7.0
    rng = np.random.default_rng(11)
    u = random_poly(rng, p - 1, p - 1, xc=0.5, yc=0.5, sx=0.5, sy=0.5)
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=kappa, seed=1, m=1)
    coef_cache = {}

    def coef_fn(x, y):
        key = (round(float(x.min()), 12), round(float(y.min()), 12))
        if key not in coef_cache:
            r = np.random.default_rng(abs(hash(key)) % (2 ** 32))
            coef_cache[key] = random_coef(r, x.size)
        return coef_cache[key]

    def load_fn(x, y):
        return u.apply_operator(x, y, coef_fn(x, y), kappa)[:, None]

    u_gpu = gpu_pipeline(w, prec, coef_fn, load_fn, lambda x, y: u(x, y))
    exact = np.stack([u(*O.leaf_nodes(p, b)) for b in w.boxes()])
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert rel(u_gpu[:, mask], exact[:, mask]) < 1e-10


def test_rectangular_grid_and_body_load():
    """2 x 8 leaves (x merge once, then y only), variable b and bumps."""
    w = WL.bumps(p=9, nx=2, ny=8, kappa=15.0, seed=4, m=1)
    w.dirichlet = "planewave"
    p = 9
    u_gpu = gpu_pipeline(w)
    sol, _, _ = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert rel(u_gpu[:, mask], u_ora[:, mask]) < 1e-12


def test_single_leaf_solve():
    w = WL.planewave(p=12, nx=1, ny=1, kappa=6.0)
    u_gpu = gpu_pipeline(w)
    sol, _, _ = oracle_pipeline(w)
    mask = np.ones(144, bool)
    mask[[0, 11, 132, 143]] = False
    assert rel(u_gpu[:, mask], grid_from_sol(sol, 12)[:, mask]) < 1e-12


def test_merge_argument_errors():
    w = WL.planewave(p=6, nx=2, ny=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    T = torch.zeros(int(plan.layout.o_bb[-1]), dtype=torch.float64, device="cuda")
    with pytest.raises(hps.HpsError):
        plan.merge(3, 2, T, None, 0)          # not powers of two / wrong count
    with pytest.raises(hps.HpsError):
        g = torch.zeros(16, dtype=torch.float64, device="cuda")
        S = torch.zeros(int(plan.layout.o_sb[-1]), dtype=torch.float64, device="cuda")
        plan.solve(g, S, None, 1)             # solve before merge


@pytest.mark.parametrize("nx,ny,p", [(32, 32, 8), (16, 32, 10)])
def test_larger_and_rectangular_grids_match_oracle(nx, ny, p):
    """10 and 9 merge levels (top interfaces of 192 and 256 nodes), square
    and 1:2 grids, variable b and bumps, against the oracle's merge tree."""
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=30.0, seed=6, m=1)
    w.dirichlet = "planewave"
    u_gpu = gpu_pipeline(w)
    sol, _, _ = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert rel(u_gpu[:, mask], u_ora[:, mask]) < 1e-11


@pytest.mark.parametrize("p", [11])
def test_tensor_core_merge_matches_oracle(p):
    """32 x 32 leaves, p = 11, a root interface of 288 nodes (elimination
    blocks of 128, 128 and 32 rows, the last one ragged): the root's split solve
    with the right-hand side in blocks and tensor-core updates, and the
    parents' maps of the levels below on the tensor cores, against the
    oracle's merge tree; the FP64-pipe merge beside it."""
    w = WL.bumps(p=p, nx=32, ny=32, kappa=30.0, seed=8, m=1)
    w.dirichlet = "planewave"
    sol, _, _ = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    errs = {}
    for tensor in (True, False):
        u_gpu = gpu_pipeline(w, tensor=tensor)
        errs[tensor] = rel(u_gpu[:, mask], u_ora[:, mask])
    print(f"p = {p}: tensor cores {errs[True]:.2e}, FP64 pipe {errs[False]:.2e}")
    assert errs[True] < 1e-11 and errs[False] < 1e-11


EVERY_LEVEL_SPLIT = 1 << 30


@pytest.mark.parametrize("nx,ny,p", [(8, 8, 9), (8, 8, 13), (4, 16, 12)])
def test_split_and_one_cta_merges_match_oracle(nx, ny, p):
    """The merge solve over many CTAs on every level, and one CTA per merge
    on every level, both against the oracle's merge tree.  Shared edges of
    56 (p = 9) and 88 (p = 13) nodes end in a ragged 8-row panel; 4 x 16
    merges x once, then y alone."""
    w = WL.bumps(p=p, nx=nx, ny=ny, kappa=25.0, seed=7, m=1)
    w.dirichlet = "planewave"
    sol, _, _ = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    for split in (0, EVERY_LEVEL_SPLIT):
        u_gpu = gpu_pipeline(w, split=split)
        assert rel(u_gpu[:, mask], u_ora[:, mask]) < 1e-12, split


def test_merge_split_argument_error():
    w = WL.planewave(p=6, nx=2, ny=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    with pytest.raises(hps.HpsError):
        plan.set_merge_split(-2)


def test_full_size_grid_reproduces_manufactured_polynomial():
    """The benchmark's grid: 64 x 64 leaves of p = 20 (12 merge levels, a
    root interface of 1152 nodes), kappa = 200 with the bumps_p20 field b.
    A tensor polynomial of degree 19 in x and y is the exact discrete
    solution on every leaf, so condense + merge + solve must reproduce it
    to rounding at every node; the default schedule (the levels near the
    root solved over many CTAs) and one CTA per merge must agree."""
    p, n = 20, 64
    w = WL.bumps_p20()
    rng = np.random.default_rng(2020)
    u = random_poly(rng, p - 1, p - 1, xc=0.5, yc=0.5, sx=0.5, sy=0.5)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    xy = plan.leaf_nodes().cpu().numpy().reshape(n * n, 2, p * p)
    x, y = xy[:, 0], xy[:, 1]
    coef = np.moveaxis(w.coefficients(x, y), 0, 1)                 # (leaves, 6, p^2)
    f = u.apply_operator(x, y, np.moveaxis(coef, 1, 0), w.kappa)   # (leaves, p^2)
    exact = u(x, y)
    out = plan.condense(torch.from_numpy(coef.ravel()).cuda(), torch.from_numpy(f.ravel()).cuda(),
                        m=1, prec="fp64")
    q = p - 2
    j = np.arange(1, p - 1)
    ix = np.arange(n)
    # outer edge nodes, root order [W, E, S, N], each side by increasing coordinate
    W = exact[ix][:, j].ravel()
    E = exact[(n - 1) * n + ix][:, (p - 1) * p + j].ravel()
    S = exact[ix * n][:, j * p].ravel()
    N = exact[ix * n + n - 1][:, j * p + p - 1].ravel()
    g = torch.from_numpy(np.concatenate([W, E, S, N])).cuda()
    assert g.numel() == 4 * n * q
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    sols = []
    for split in (-1, 0):
        plan.set_merge_split(split)
        plan.merge(n, n, out["T"], out["h"], 1)
        sols.append(plan.solve(g, out["S"], out["W"], 1).cpu().numpy().reshape(n * n, p * p))
    torch.cuda.synchronize()
    assert (out["info"].cpu().numpy() == 0).all()
    for us in sols:
        assert rel(us[:, mask], exact[:, mask]) < 1e-9
    assert rel(sols[0][:, mask], sols[1][:, mask]) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_psi_curved_domain_pipeline(prec):
    """Section 3's curved domain Psi (c12 != 0, corners by extrapolation):
    condense + merge + solve on 4 x 4 leaves of p = 14 against the oracle's
    merge tree, and against the exact physical plane wave."""
    p = 14
    w = WL.psi_curved(p=p, nx=4, ny=4, kappa=10.0, m=1)
    w.load = "zero"
    u_gpu = gpu_pipeline(w, prec)
    sol, _, _ = oracle_pipeline(w)
    u_ora = grid_from_sol(sol, p)
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert rel(u_gpu[:, mask], u_ora[:, mask]) < (1e-12 if prec == "fp64" else 1e-10)
    exact = np.stack([w.dirichlet_data(*O.leaf_nodes(p, b)) for b in w.boxes()])
    assert rel(u_gpu[:, mask], exact[:, mask]) < 1e-9


def test_parent_maps_on_tensor_cores_match_fp64_pipe():
    """hps_set_merge_tensor: the parents' [T | h] of the levels with shared
    edges of at least 128 nodes formed from integer slices on the BF16 tensor
    cores against the same maps on the FP64 pipe (16 x 16 leaves of p = 20:
    the two top levels, shared edges of 144 and 288 nodes), root map and
    solution; and the tensor-core merge's solution against the oracle."""
    w = WL.bumps(p=20, nx=16, ny=16, kappa=60.0, seed=4, m=1)
    w.dirichlet = "planewave"
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    keys = O.outer_boundary_keys(20, 16, 16)
    g = torch.from_numpy(np.array([w.dirichlet_data(*O.key_coords(20, k, 16, 16)) for k in keys])).cuda()
    res = {}
    for on in (False, True):
        plan.set_merge_tensor(on)
        th = plan.merge_boxes(16, 16, 1, 1, out["T"], out["h"], 1, root=True)
        plan.merge(16, 16, out["T"], out["h"], 1)
        u = plan.solve(g, out["S"], out["W"], 1)
        torch.cuda.synchronize()
        res[on] = (th.clone(), u.clone())
    (th0, u0), (th1, u1) = res[False], res[True]
    assert float((th1 - th0).norm() / th0.norm()) < 1e-13
    assert float((u1 - u0).norm() / u0.norm()) < 1e-12
    plan.close()


def test_nonfinite_leaf_map_reaches_the_root_on_both_paths():
    """A NaN in leaf 0's T at (its west node 0, its north node 0), p = 12,
    8 x 8 leaves: at the second level the north node is on the shared edge
    (20 nodes, a tensor-core product), so the NaN sits in the left factor's
    row of the outer-boundary node; that row of every parent map, and of
    the root map, must be NaN on both paths (the integer slices cannot
    carry a NaN: the row's scale marks it), Z stays finite, and the NaN
    patterns of the two paths agree."""
    w = WL.bumps(p=12, nx=8, ny=8, kappa=20.0, seed=5, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    T = out["T"].clone()
    T[30] = float("nan")   # leaf 0 (40 edge nodes [W, E, S, N]): row 0 (west), column 30 (north)
    pattern = {}
    for tensor in (True, False):
        plan.set_merge_tensor(tensor)
        th = plan.merge_boxes(8, 8, 1, 1, T, out["h"], 1, root=True)
        torch.cuda.synchronize()
        pattern[tensor] = torch.isnan(th)
        assert pattern[tensor].any(), tensor
    assert torch.equal(pattern[True], pattern[False])
    plan.close()


def test_check_info_codes():
    """hps_check_info on device info arrays: success, an exact zero pivot
    (reported before a non-converged entry), a non-converged entry alone."""
    w = WL.planewave(p=6, nx=2, ny=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    mk = lambda v: torch.tensor(v, dtype=torch.int32, device="cuda")
    assert plan.check_info(mk([0, 0, 0])) is None
    assert plan.check_info(mk([0, -3, 7, 0])) == ("HPS_ERR_SINGULAR", 2)
    assert plan.check_info(mk([0, 0, -8])) == ("HPS_ERR_NOCONV", 2)
    with pytest.raises(ValueError):
        plan.check_info(torch.zeros(3, dtype=torch.float64, device="cuda"))
    plan.close()


_CPASYNC_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2])
from gpu_cases import gpu_inputs
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL
w = WL.bumps(p=20, nx=16, ny=16, kappa=60.0, seed=4, m=1)
plan = hps.Plan(w.p, w.boxes(), w.kappa)
coef, f, _ = gpu_inputs(w, plan)
out = plan.condense(coef, f, m=1)
th = plan.merge_boxes(16, 16, 1, 1, out["T"], out["h"], 1, root=True)
np.save(sys.argv[1], th.cpu().numpy())
"""


def test_tensor_core_loads_by_cp_async_match_tma(tmp_path):
    """The tensor-core products load their operands as TMA boxes where the
    driver encodes tensor maps, else by cp.async of the same runs
    (HPS_OZAKI_TMA=0 forces the latter, read once per process): the root
    map of a 16 x 16, p = 20 merge from a child process on cp.async equals
    this process's, bit for bit."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    path = str(tmp_path / "th_cpasync.npy")
    env = dict(os.environ, HPS_OZAKI_TMA="0", PYTHONPATH=os.pathsep.join([root, here]))
    subprocess.run([sys.executable, "-c", _CPASYNC_CHILD, path, here], check=True, env=env, cwd=root, timeout=600)
    w = WL.bumps(p=20, nx=16, ny=16, kappa=60.0, seed=4, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    th = plan.merge_boxes(16, 16, 1, 1, out["T"], out["h"], 1, root=True).cpu().numpy()
    assert np.array_equal(np.load(path), th)
    plan.close()


@pytest.mark.parametrize("m", [0, 3])
def test_tensor_core_merge_load_columns(m):
    """No body loads (the parents' maps without h columns) and three load
    columns: the root [T | h] of a 16 x 16, p = 20 merge with the
    tensor-core products against the FP64 pipe."""
    w = WL.bumps(p=20, nx=16, ny=16, kappa=60.0, seed=9, m=max(m, 1))
    w.m = m
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f if m else None, m=m)
    th = {}
    for tensor in (True, False):
        plan.set_merge_tensor(tensor)
        th[tensor] = plan.merge_boxes(16, 16, 1, 1, out["T"], out["h"] if m else None, m, root=True).clone()
        torch.cuda.synchronize()
    assert float((th[True] - th[False]).norm() / th[False].norm()) < 1e-13
    plan.close()
