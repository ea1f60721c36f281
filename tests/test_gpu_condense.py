"""GPU parity of the batched leaf condensation (hps_condense) against the FP64
CPU oracle, element by element per leaf, through the C ABI.

Bars (relative Frobenius error per leaf and output S, T, W, h):
  FP64 path                   1e-12
  FP32/TF32/BF16 + refinement 1e-10
Only a near-resonant leaf (cond(A_ii) > 1e5, gpu_cases.COND_FLAG) gets
max(bar, 10 cond(A_ii) eps), the rounding-order spread of two correct FP64
eliminations of the same system; such leaves are printed separately.
"""

import numpy as np
import pytest
import torch

import oracle.hps_oracle as O
from gpu_cases import assert_within, compare_leaves, gpu_inputs, leaf_slices, relerr
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-10, "tf32": 1e-10, "bf16": 1e-10}


class Sub:
    """A subset of a workload's leaves, as its own plan."""

    def __init__(self, w, leaves):
        self.w = w
        self.leaves = np.asarray(leaves)
        self.m = w.m
        self.kappa = w.kappa
        self.p = w.p[self.leaves]
        self.box = w.boxes()[self.leaves]
        self.coefficients = w.coefficients
        self.body_load = w.body_load

    def boxes(self):
        return self.box


def run(sub, prec, tol=1e-12, kmax=8, coef_fn=None, load_fn=None, m=None, fallback=True):
    plan = hps.Plan(sub.p, sub.box, sub.kappa)
    plan.set_fp64_fallback(fallback)
    coef, f, _ = gpu_inputs(sub, plan, coef_fn, load_fn)
    out = plan.condense(coef, f, m=sub.m if m is None else m, prec=prec, tol=tol, kmax=kmax)
    torch.cuda.synchronize()
    return plan, out


def check(sub, prec, leaves=None, coef_fn=None, load_fn=None, kmax=8):
    plan, out = run(sub, prec, tol=1e-13, kmax=kmax, coef_fn=coef_fn, load_fn=load_fn)
    info = out["info"].cpu().numpy()
    assert (info == 0).all(), info
    idx = range(len(sub.leaves)) if leaves is None else leaves
    recs = compare_leaves(sub, plan, out, idx, TOL[prec], coef_fn=coef_fn, load_fn=load_fn)
    assert_within(recs)
    return recs


def test_leaf_nodes_match_oracle():
    w = WL.uneven(nx=4, ny=4, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    xy = plan.leaf_nodes().cpu().numpy()
    lay = plan.layout
    for l in range(w.n_leaves):
        p2, o = int(lay.p2[l]), int(lay.o_p2[l])
        x, y = O.leaf_nodes(int(w.p[l]), w.boxes()[l])
        assert np.abs(xy[2 * o: 2 * o + p2] - x).max() < 4e-16
        assert np.abs(xy[2 * o + p2: 2 * o + 2 * p2] - y).max() < 4e-16


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("p", [4, 5, 6, 12, 20, 24, 30, 32])
def test_orders_and_ragged_tiles(prec, p):
    """Every order of the workloads plus the smallest ones: n_i = (p-2)^2 is
    not a multiple of the panel width for most p (ragged last panel)."""
    nx = 32 if p >= 20 else 16
    w = WL.bumps(p=p, nx=nx, ny=nx, kappa=200.0 if p >= 20 else 60.0, seed=7, m=1)
    check(Sub(w, [0, 1, nx + 5, w.n_leaves - 1]), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_bumps_p20_block(prec):
    """A 4 x 4 block of the 64 x 64, p = 20, kappa = 200 workload."""
    w = WL.bumps_p20()
    leaves = [ix * 64 + iy for ix in range(30, 34) for iy in range(30, 34)]
    check(Sub(w, leaves), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m", [0, 3])
def test_body_load_columns(prec, m):
    w = WL.bumps(p=12, nx=16, ny=16, kappa=60.0, seed=9, m=max(m, 1))
    w.m = m
    check(Sub(w, [3, 40, 100]), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_uneven_orders_one_launch(prec):
    """Leaves of p in {12, 16, 20, 24, 32} in one plan (largest first)."""
    w = WL.uneven(m=2)
    leaves = list(range(0, 10240, 331))[:24]
    recs = check(Sub(w, leaves), prec)
    assert len({int(w.p[l]) for l in leaves}) >= 4
    assert len(recs) == len(leaves)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_annulus_variable_coefficients(prec):
    """Mapped annulus: c22 = 4/(pi^2 r^2), c1 = 1/r, b variable (c1 != 0)."""
    w = WL.annulus_p24()
    leaves = [0, 127, 64 * 128 - 1, 40 * 128 + 77]
    check(Sub(w, leaves), prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_derivative_term(prec):
    """c12 != 0 (the mixed-derivative term of Eq. (chain_rule)); the
    corners enter on both sides through the corner extrapolation."""
    def coef_fn(x, y):
        one = np.ones_like(x)
        return np.stack([1.0 + 0.2 * x, 0.15 * np.sin(3 * y), 1.0 + 0.1 * y, 0.3 * one, -0.2 * x,
                         1.0 - 0.3 * np.cos(2 * x)])
    w = WL.bumps(p=14, nx=16, ny=16, kappa=40.0, seed=3, m=1)
    check(Sub(w, [0, 77, 255]), prec, coef_fn=coef_fn)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_term_reproduces_degree_p_minus_3_polynomial(prec):
    """c12 != 0 with random coefficient samples on every leaf: a tensor
    polynomial of degree p-3 (exact under the corner extrapolation) gives
    S u_b + W = u_i and T u_b + h = its analytic outward normal derivative."""
    from manufactured import random_coef, random_poly
    p = 12
    w = WL.bumps(p=p, nx=4, ny=4, kappa=20.0, seed=5, m=1)
    sub = Sub(w, list(range(16)))
    rng = np.random.default_rng(123)
    u = random_poly(rng, p - 3, p - 3, xc=0.5, yc=0.5, sx=0.5, sy=0.5)
    cache = {}

    def coef_fn(x, y):
        key = (round(float(np.min(x)), 12), round(float(np.min(y)), 12))
        if key not in cache:
            cache[key] = random_coef(np.random.default_rng(abs(hash(key)) % (2 ** 32)), x.size, c12=True)
        return cache[key]

    def load_fn(x, y):
        return u.apply_operator(x, y, coef_fn(x, y), w.kappa)[:, None]

    plan, out = run(sub, prec, tol=1e-13, coef_fn=coef_fn, load_fn=load_fn)
    assert (out["info"].cpu().numpy() == 0).all()
    cpu = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    ix = O.leaf_index_sets(p)
    for l in range(16):
        x, y = O.leaf_nodes(p, sub.box[l])
        got = leaf_slices(plan.layout, cpu, l, 1)
        uv = u(x, y)[:, None]
        dudx, dudy = u(x, y, 1, 0), u(x, y, 0, 1)
        dn = np.concatenate([-dudx[ix["W"]], dudx[ix["E"]], -dudy[ix["S"]], dudy[ix["N"]]])[:, None]
        e_int = relerr(got["S"] @ uv[ix["B"]] + got["W"], uv[ix["I"]])
        e_flux = relerr(got["T"] @ uv[ix["B"]] + got["h"], dn)
        assert e_int < 1e-10 and e_flux < 1e-10, (l, e_int, e_flux)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_largest_order(prec):
    w = WL.bumps(p=42, nx=16, ny=16, kappa=200.0, seed=11, m=1)
    check(Sub(w, [17]), prec)


def test_singular_leaf_reports_info():
    """A leaf with all coefficients zero at kappa = 0 has A_ii = 0: the first
    pivot is exactly zero (info = 1); its neighbour (Laplacian) is fine."""
    w = WL.bumps(p=8, nx=2, ny=1, kappa=0.0, seed=1, m=1)

    def coef_fn(x, y):
        c = w.coefficients(x, y)
        if np.all(x <= 0.5 + 1e-12):
            return np.zeros_like(c)
        return c
    for prec in ("fp64", "fp32"):
        plan, out = run(Sub(w, [0, 1]), prec, coef_fn=coef_fn)
        assert list(out["info"].cpu().numpy()) == [1, 0]


def test_refinement_nonconvergence_reported():
    w = WL.bumps(p=12, nx=8, ny=8, kappa=60.0, seed=1, m=1)
    plan, out = run(Sub(w, [0, 9]), "fp32", tol=0.0, kmax=2, fallback=False)
    assert list(out["info"].cpu().numpy()) == [-2, -2]
    # with the FP64 fallback (default) the same leaves are condensed in FP64
    plan, out = run(Sub(w, [0, 9]), "fp32", tol=0.0, kmax=2)
    assert list(out["info"].cpu().numpy()) == [0, 0] and plan.fallback_count() == 2
    assert_within(compare_leaves(Sub(w, [0, 9]), plan, out, [0, 1], 1e-12))
    plan, out = run(Sub(w, [0, 9]), "fp32", tol=1e-13, kmax=8)
    assert list(out["info"].cpu().numpy()) == [0, 0]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_full_size_bumps_p20_sampled(prec):
    """All 4096 leaves of the p = 20 workload in one launch (the benchmark's
    configuration); sampled leaves against the oracle one by one."""
    w = WL.bumps_p20()
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1, prec=prec, tol=1e-13, kmax=8)
    torch.cuda.synchronize()
    assert (out["info"].cpu().numpy() == 0).all()
    if prec in ("tf32", "bf16"):
        print(f"{prec}: {plan.fallback_count()} of 4096 leaves re-condensed in FP64")
    rng = np.random.default_rng(0)
    leaves = sorted(set(rng.integers(0, w.n_leaves, 6).tolist()) | {0, w.n_leaves - 1})
    assert_within(compare_leaves(w, plan, out, leaves, TOL[prec]))
    for k in ("S", "T", "h", "W"):
        assert torch.isfinite(out[k]).all()


def test_store_S_optional():
    w = WL.bumps(p=10, nx=8, ny=8, kappa=40.0, seed=2, m=1)
    sub = Sub(w, [1, 2])
    plan = hps.Plan(sub.p, sub.box, sub.kappa)
    coef, f, _ = gpu_inputs(sub, plan)
    a = plan.condense(coef, f, m=1, store_S=True)
    b = plan.condense(coef, f, m=1, store_S=False)
    torch.cuda.synchronize()
    assert "S" not in b
    assert torch.equal(a["T"], b["T"]) and torch.equal(a["h"], b["h"])


def test_true_residual_stop_after_first_correction():
    """hps_set_refine_stop(plan, 1): after the first correction the residual
    ratio eta_1 |R_1| / |R_0| decides (its own kernel instantiation).  At
    tol = 1e-11 leaves stop after one correction and still hold the mixed
    bar against the oracle (a 4 x 4 block of bumps_p20 and uneven leaves);
    at tol = 0 it never stops and reports non-convergence."""
    for w, leaves in ((WL.bumps_p20(), [ix * 64 + iy for ix in range(30, 34) for iy in range(30, 34)]),
                      (WL.uneven(m=2), list(range(0, 10240, 977)))):
        sub = Sub(w, leaves)
        plan = hps.Plan(sub.p, sub.box, sub.kappa)
        plan.set_refine_stop(True)
        coef, f, _ = gpu_inputs(sub, plan)
        out = plan.condense(coef, f, m=sub.m, prec="fp32", tol=1e-11, kmax=6)
        torch.cuda.synchronize()
        assert (out["info"].cpu().numpy() == 0).all()
        assert_within(compare_leaves(sub, plan, out, range(len(leaves)), TOL["fp32"]))
        plan.set_fp64_fallback(False)
        out = plan.condense(coef, f, m=sub.m, prec="fp32", tol=0.0, kmax=2)
        torch.cuda.synchronize()
        assert (out["info"].cpu().numpy() == -2).all()
        plan.close()
