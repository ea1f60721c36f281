"""GPU parity of the leaf solve by re-forming and re-factoring
(hps_leaf_resolve, Section 2 Remark) against the oracle's plain dense solve
of A_ii u_i = f_I - A_ib u_b, element by element per leaf; against the
stored-operator solve u_i = S u_b + W (hps_leaf_recover) on the same edge
values; and inside the full condense + merge + solve pipeline."""

import numpy as np
import pytest
import torch

import oracle.hps_oracle as O
from gpu_cases import gpu_inputs, leaf_bar, relerr
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-10}


class Sub:
    """A subset of a workload's leaves, as its own plan, with m loads."""

    def __init__(self, w, leaves, m=None):
        self.leaves = np.asarray(leaves)
        self.m = w.m if m is None else m
        self.kappa = w.kappa
        self.p = w.p[self.leaves]
        self.box = w.boxes()[self.leaves]
        self.coefficients = w.coefficients
        self.body_load = w.body_load

    def boxes(self):
        return self.box


def edge_values(plan, m, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(int(plan.layout.o_nb[-1] * m))


def resolve(sub, prec, m, seed=0, coef_fn=None, with_f=True, fallback=True, tol=1e-13, kmax=8):
    plan = hps.Plan(sub.p, sub.box, sub.kappa)
    plan.set_fp64_fallback(fallback)
    coef, f, _ = gpu_inputs(sub, plan, coef_fn)
    ub = edge_values(plan, m, seed)
    out = plan.leaf_resolve(coef, torch.from_numpy(ub).cuda(), f if with_f else None, m=m, prec=prec,
                            tol=tol, kmax=kmax)
    torch.cuda.synchronize()
    return plan, coef, f, ub, out


def check_against_oracle(sub, plan, ub, out, m, prec, leaves=None, coef_fn=None, with_f=True):
    lay = plan.layout
    u = out["u"].cpu().numpy()
    worst = 0.0
    for l in (range(lay.n_leaves) if leaves is None else leaves):
        p, box = int(sub.p[l]), sub.box[l]
        x, y = O.leaf_nodes(p, box)
        c = (coef_fn or sub.coefficients)(x, y)
        fl = sub.body_load(x, y).reshape(p * p, -1) if with_f else None
        ubl = ub[int(lay.o_nb[l]) * m: int(lay.o_nb[l + 1]) * m].reshape(-1, m)
        ref = O.leaf_resolve(p, box, c, sub.kappa, ubl, fl)
        got = u[int(lay.o_p2[l]) * m: int(lay.o_p2[l + 1]) * m].reshape(p * p, m)
        A, _, _, _ = O.leaf_operator(p, box, c, sub.kappa)
        I = O.leaf_index_sets(p)["I"]
        bar, flagged = leaf_bar(TOL[prec], np.linalg.cond(A[np.ix_(I, I)]))
        e = relerr(got, ref)
        if flagged:
            print(f"near-resonant leaf {l} (p = {p}): error {e:.1e}, bar {bar:.1e}")
        assert e < bar, (l, p, e, bar)
        worst = max(worst, e)
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [5, 12, 20, 30])
def test_orders(prec, p):
    """Every order class, including ragged last panels; one load column."""
    nx = 32 if p >= 20 else 16
    w = WL.bumps(p=p, nx=nx, ny=nx, kappa=200.0 if p >= 20 else 60.0, seed=7, m=1)
    sub = Sub(w, [0, 1, nx + 5, w.n_leaves - 1])
    plan, _, _, ub, out = resolve(sub, prec, 1, seed=p)
    assert (out["info"].cpu().numpy() == 0).all()
    check_against_oracle(sub, plan, ub, out, 1, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,with_f", [(3, True), (2, False), (40, True)])
def test_load_columns(prec, m, with_f):
    w = WL.bumps(p=12, nx=16, ny=16, kappa=60.0, seed=9, m=m)
    sub = Sub(w, [3, 40, 100])
    plan, _, _, ub, out = resolve(sub, prec, m, seed=m, with_f=with_f)
    assert (out["info"].cpu().numpy() == 0).all()
    check_against_oracle(sub, plan, ub, out, m, prec, with_f=with_f)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_orders_one_launch(prec):
    w = WL.uneven(m=2)
    leaves = list(range(0, 10240, 431))[:20]
    sub = Sub(w, leaves)
    plan, _, _, ub, out = resolve(sub, prec, 2, seed=5)
    assert (out["info"].cpu().numpy() == 0).all()
    check_against_oracle(sub, plan, ub, out, 2, prec)
    assert len({int(p) for p in sub.p}) >= 4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_annulus_first_derivative_terms(prec):
    """c1 != 0 (the annulus map): the general residual on the mixed path."""
    w = WL.annulus_p24()
    sub = Sub(w, [0, 127, 64 * 128 - 1, 40 * 128 + 77])
    plan, _, _, ub, out = resolve(sub, prec, 1, seed=3)
    assert (out["info"].cpu().numpy() == 0).all()
    check_against_oracle(sub, plan, ub, out, 1, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_derivative_term(prec):
    """c12 != 0: every edge value enters every row's right-hand side."""
    def coef_fn(x, y):
        one = np.ones_like(x)
        return np.stack([1.0 + 0.2 * x, 0.15 * np.sin(3 * y), 1.0 + 0.1 * y, 0.3 * one, -0.2 * x,
                         1.0 - 0.3 * np.cos(2 * x)])
    w = WL.bumps(p=14, nx=16, ny=16, kappa=40.0, seed=3, m=1)
    sub = Sub(w, [0, 77, 255])
    plan, _, _, ub, out = resolve(sub, prec, 1, seed=11, coef_fn=coef_fn)
    assert (out["info"].cpu().numpy() == 0).all()
    check_against_oracle(sub, plan, ub, out, 1, prec, coef_fn=coef_fn)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matches_stored_operator_solve(prec):
    """The re-factored solve and u_i = S u_b + W from the stored S, W of an
    FP64 condensation agree on the same edge values (mixed orders, m = 2)."""
    w = WL.uneven(nx=16, ny=8, m=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    cond = plan.condense(coef, f, m=2, prec="fp64")
    ub = torch.from_numpy(edge_values(plan, 2, 21)).cuda()
    u_rec = plan.leaf_recover(cond["S"], cond["W"], ub, 2)
    out = plan.leaf_resolve(coef, ub, f, m=2, prec=prec, tol=1e-13, kmax=8)
    torch.cuda.synchronize()
    assert (out["info"].cpu().numpy() == 0).all()
    lay = plan.layout
    a, b = out["u"].cpu().numpy(), u_rec.cpu().numpy()
    for l in range(lay.n_leaves):
        s = slice(int(lay.o_p2[l]) * 2, int(lay.o_p2[l + 1]) * 2)
        assert relerr(a[s], b[s]) < (1e-10 if prec == "fp32" else 1e-11), l


def test_completes_the_merge_and_solve():
    """The paper's procedure: condense, merge, solve the reduced system, then
    re-form and re-factor every leaf for its interior values from the edge
    values the solve produced.  Same u as the stored-S leaf recovery of the
    downward pass, plane-wave workload."""
    w = WL.planewave()
    p = 10
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    out = plan.condense(coef, f, m=1)
    plan.merge(w.nx, w.ny, out["T"], out["h"], 1)
    keys = O.outer_boundary_keys(p, w.nx, w.ny)
    g = np.array([w.dirichlet_data(*O.key_coords(p, k, w.nx, w.ny)) for k in keys], dtype=np.float64)
    u_full = plan.solve(torch.from_numpy(g).cuda(), out["S"], out["W"], 1).cpu().numpy().reshape(w.n_leaves, p * p)
    B = O.leaf_index_sets(p)["B"]
    ub = torch.from_numpy(np.ascontiguousarray(u_full[:, B]).ravel()).cuda()
    for prec in ("fp64", "fp32"):
        res = plan.leaf_resolve(coef, ub, f, m=1, prec=prec, tol=1e-13, kmax=8)
        torch.cuda.synchronize()
        assert (res["info"].cpu().numpy() == 0).all()
        u = res["u"].cpu().numpy().reshape(w.n_leaves, p * p)
        assert relerr(u, u_full) < (1e-10 if prec == "fp32" else 1e-12), prec


def test_singular_leaf_reports_info():
    w = WL.bumps(p=8, nx=2, ny=1, kappa=0.0, seed=1, m=1)

    def coef_fn(x, y):
        c = w.coefficients(x, y)
        if np.all(x <= 0.5 + 1e-12):
            return np.zeros_like(c)
        return c
    sub = Sub(w, [0, 1])
    for prec in ("fp64", "fp32"):
        _, _, _, _, out = resolve(sub, prec, 1, coef_fn=coef_fn)
        assert list(out["info"].cpu().numpy()) == [1, 0]


def test_nonconvergence_falls_back_to_fp64():
    w = WL.bumps(p=12, nx=8, ny=8, kappa=60.0, seed=1, m=1)
    sub = Sub(w, [0, 9])
    _, _, _, _, out = resolve(sub, "fp32", 1, tol=0.0, kmax=2, fallback=False)
    assert list(out["info"].cpu().numpy()) == [-2, -2]
    plan, _, _, ub, out = resolve(sub, "fp32", 1, tol=0.0, kmax=2)
    assert list(out["info"].cpu().numpy()) == [0, 0] and plan.fallback_count() == 2
    check_against_oracle(sub, plan, ub, out, 1, "fp64")


def test_argument_errors():
    """Host-side checks of the C ABI: m < 1, missing edge values or S."""
    w = WL.planewave(p=6, nx=2, ny=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, _, _ = gpu_inputs(w, plan)
    ub = torch.zeros(int(plan.layout.o_nb[-1]), dtype=torch.float64, device="cuda")
    u = torch.zeros(int(plan.layout.o_p2[-1]), dtype=torch.float64, device="cuda")
    info = torch.zeros(plan.layout.n_leaves, dtype=torch.int32, device="cuda")
    lib, P = hps.load_library(), hps._ptr
    assert lib.hps_leaf_resolve(plan.handle, 0, P(coef), None, 0, P(ub), 0.0, 0, P(u), P(info), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_resolve(plan.handle, 0, P(coef), None, 1, None, 0.0, 0, P(u), P(info), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_resolve(plan.handle, 1, P(coef), None, 1, P(ub), -1.0, 2, P(u), P(info), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_recover(plan.handle, None, None, 1, P(ub), P(u), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_recover(plan.handle, P(u), None, 0, P(ub), P(u), None) == hps.HPS_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_bumps_p20_sampled(prec):
    """All 4096 leaves of the p = 20 workload in one launch; sampled leaves
    against the oracle one by one."""
    w = WL.bumps_p20()
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    ub = edge_values(plan, 1, 2)
    out = plan.leaf_resolve(coef, torch.from_numpy(ub).cuda(), f, m=1, prec=prec, tol=1e-12, kmax=6)
    torch.cuda.synchronize()
    assert (out["info"].cpu().numpy() == 0).all()
    assert torch.isfinite(out["u"]).all()
    rng = np.random.default_rng(1)
    leaves = sorted(set(rng.integers(0, w.n_leaves, 5).tolist()) | {0, w.n_leaves - 1})
    check_against_oracle(Sub(w, np.arange(w.n_leaves)), plan, ub, out, 1, prec, leaves=leaves)
