"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (not against the oracle itself).

* exact spectral differentiation of polynomials of degree <= p-1 (Section 2),
  closed-form Chebyshev matrix entries and the hand-derived p = 2, 3 matrices
  in tests/golden;
* manufactured tensor-polynomial solutions: the collocated operator, the leaf
  condensation (S, T, W, h) and the full merge + solve reproduce them to
  rounding, for any wavenumber and coefficient samples;
* the brute-force dense global collocation solve of Eq. (Au=f) agrees with
  the merge tree;
* plane-wave and J0 closed-form Helmholtz solutions (Section 3, Eq.
  (constant_coeff_helm)) converge spectrally in p, and T maps a plane wave's
  boundary trace to its normal derivative;
* planted mistakes (a transposed D, a flipped normal, a dropped term, a wrong
  merge key order) make at least one pin fail.
"""

import os

import numpy as np
import pytest
import scipy.special

import oracle.hps_oracle as O
from manufactured import TensorPoly, random_coef, random_poly
from paper_2211_14969_b300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- pin helpers

def deriv_error(p):
    """max relative error of D applied to Chebyshev polynomials T_k, k < p."""
    t = O.cheb_points(p)
    D = O.cheb_diff(p)
    worst = 0.0
    for k in range(p):
        c = np.zeros(k + 1)
        c[k] = 1.0
        u = np.polynomial.chebyshev.chebval(t, c)
        du = np.polynomial.chebyshev.chebval(t, np.polynomial.chebyshev.chebder(c)) if k else 0 * t
        scale = max(1.0, np.abs(du).max())
        worst = max(worst, np.abs(D @ u - du).max() / scale)
    return worst


def operator_error(p, box, coef, kappa, u):
    x, y = O.leaf_nodes(p, box)
    A, _, _, _ = O.leaf_operator(p, box, coef, kappa)
    uv = u(x, y)
    f = u.apply_operator(x, y, coef, kappa)
    scale = np.abs(A) @ np.abs(uv)
    return np.max(np.abs(A @ uv - f) / scale)


def condense_errors(p, box, coef, kappa, u):
    x, y = O.leaf_nodes(p, box)
    f = u.apply_operator(x, y, coef, kappa)[:, None]
    out = O.condense_leaf(p, box, coef, kappa, f)
    ix = O.leaf_index_sets(p)
    uv = u(x, y)
    ub = uv[ix["B"]][:, None]
    ui = uv[ix["I"]][:, None]
    # analytic outward normal derivative on [W, E, S, N]
    dudx = u(x, y, 1, 0)
    dudy = u(x, y, 0, 1)
    dn = np.concatenate([-dudx[ix["W"]], dudx[ix["E"]], -dudy[ix["S"]], dudy[ix["N"]]])[:, None]
    e_int = O.relerr(out["S"] @ ub + out["W"], ui)
    e_flux = O.relerr(out["T"] @ ub + out["h"], dn)
    cond = np.linalg.cond(out["A_ii"])
    return e_int, e_flux, cond


def hps_grid_solve(p, nx, ny, coefs, kappa, f, g_fn):
    boxes = O.grid_boxes(nx, ny)
    leaves = [O.condense_leaf(p, boxes[l], coefs[l], kappa, f[l]) for l in range(nx * ny)]
    levels = O.hps_upward(p, nx, ny, leaves)
    gk = {k: np.atleast_1d(g_fn(*O.key_coords(p, k, nx, ny))) for k in O.outer_boundary_keys(p, nx, ny)}
    return O.hps_downward(p, nx, ny, levels, leaves, gk), leaves


def nodal_values(p, nx, ny, fn):
    """Per leaf (u_b, u_i) of a function sampled at the leaf nodes."""
    ix = O.leaf_index_sets(p)
    out = []
    for box in O.grid_boxes(nx, ny):
        x, y = O.leaf_nodes(p, box)
        v = fn(x, y)
        out.append((v[ix["B"]], v[ix["I"]]))
    return out


def grid_error(sol, ref):
    num = den = 0.0
    for s, (rb, ri) in zip(sol, ref):
        num += np.sum((s["u_b"].ravel() - rb.ravel()) ** 2) + np.sum((s["u_i"].ravel() - ri.ravel()) ** 2)
        den += np.sum(rb ** 2) + np.sum(ri ** 2)
    return np.sqrt(num / den)


def manufactured_grid_error(p=8, nx=4, ny=4, kappa=7.0, seed=11):
    rng = np.random.default_rng(seed)
    u = random_poly(rng, p - 1, p - 1, xc=0.5, yc=0.5, sx=0.5, sy=0.5)
    coefs, fs = [], []
    for box in O.grid_boxes(nx, ny):
        x, y = O.leaf_nodes(p, box)
        c = random_coef(rng, p * p)
        coefs.append(c)
        fs.append(u.apply_operator(x, y, c, kappa)[:, None])
    sol, _ = hps_grid_solve(p, nx, ny, coefs, kappa, fs, lambda x, y: u(x, y))
    return grid_error(sol, nodal_values(p, nx, ny, u))


# ------------------------------------------------------------------ the pins

@pytest.mark.parametrize("p", [2, 3])
def test_cheb_diff_golden(p):
    ref = np.loadtxt(os.path.join(GOLDEN, f"cheb_D_p{p}.txt"))
    assert np.allclose(O.cheb_diff(p), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [4, 6, 10, 12, 16, 20, 24, 30, 32, 42])
def test_cheb_diff_exact_on_polynomials(p):
    assert deriv_error(p) < 1e-13 * p * p


@pytest.mark.parametrize("p", [5, 10, 20, 32])
def test_cheb_diff_corner_closed_form(p):
    n = p - 1
    D = O.cheb_diff(p)
    assert np.isclose(D[-1, -1], (2 * n * n + 1) / 6.0, rtol=1e-13)
    assert np.isclose(D[0, 0], -(2 * n * n + 1) / 6.0, rtol=1e-13)


def test_leaf_nodes_layout():
    p, box = 5, (0.25, 0.5, 0.5, 0.25)
    x, y = O.leaf_nodes(p, box)
    # node id i*p + j, i the x index; endpoints of the box are nodes
    assert x[0] == 0.25 and np.isclose(x[(p - 1) * p], 0.75)
    assert y[0] == 0.5 and np.isclose(y[p - 1], 0.75)
    assert np.all(np.diff(x[::p]) > 0) and np.all(np.diff(y[:p]) > 0)
    ix = O.leaf_index_sets(10)
    assert len(ix["I"]) == 64 and len(ix["B"]) == 32   # p = 10: 64 interior, 32 edge nodes
    corners = {0, 9, 90, 99}
    assert not corners & set(ix["B"]) and not corners & set(ix["I"])


@pytest.mark.parametrize("p,c12", [(6, False), (10, True), (16, True), (20, False)])
def test_operator_manufactured(p, c12):
    rng = np.random.default_rng(p)
    box = (0.3, -0.2, 0.125, 0.25)
    u = random_poly(rng, p - 1, p - 1, xc=0.3625, yc=-0.075, sx=0.0625, sy=0.125)
    coef = random_coef(rng, p * p, c12=c12)
    assert operator_error(p, box, coef, 13.0, u) < 1e-12


@pytest.mark.parametrize("p,kappa", [(6, 3.0), (10, 20.0), (14, 40.0), (20, 200.0 / 8)])
def test_condense_manufactured(p, kappa):
    rng = np.random.default_rng(100 + p)
    box = (0.5, 0.25, 0.125, 0.0625)
    u = random_poly(rng, p - 1, p - 1, xc=0.5625, yc=0.28125, sx=0.0625, sy=0.03125)
    coef = random_coef(rng, p * p)
    e_int, e_flux, cond = condense_errors(p, box, coef, kappa, u)
    tol = max(1e-12, 100 * cond * EPS)
    assert e_int < tol, (e_int, cond)
    assert e_flux < tol, (e_flux, cond)


@pytest.mark.parametrize("p", [4, 5, 10, 20, 42])
def test_corner_extrapolation_exact_to_degree_p_minus_3(p):
    """Each corner from its two edges: exact for tensor polynomials of degree
    <= p-3 in each variable (the interpolant through p-2 points), each row a
    pair of partitions of unity, and not exact at degree p-2."""
    rng = np.random.default_rng(40 + p)
    box = (0.25, 0.5, 0.125, 0.0625)
    x, y = O.leaf_nodes(p, box)
    ix = O.leaf_index_sets(p)
    E = O.corner_extrapolation(p)
    corners = [0, p - 1, (p - 1) * p, p * p - 1]
    assert np.allclose(E.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    u = random_poly(rng, p - 3, p - 3, xc=0.3125, yc=0.53125, sx=0.0625, sy=0.03125)
    got, ref = E @ u(x, y)[ix["B"]], u(x, y)[corners]
    assert O.relerr(got, ref) < 1e-11, O.relerr(got, ref)
    # eta^(p-2): along W and E the extrapolation misses by the node
    # polynomial omega(t) = prod (t - t_k) over the p-2 interior Chebyshev
    # points t_k = -cos(k pi / (p-1)); along S and N it is constant (exact)
    C = np.zeros((1, p - 1))
    C[0, p - 2] = 1.0
    v = TensorPoly(C, xc=0.3125, yc=0.53125, sx=0.0625, sy=0.03125)
    tk = -np.cos(np.arange(1, p - 1) * np.pi / (p - 1))
    om = {s: np.prod(s - tk) for s in (-1.0, 1.0)}
    miss = np.array([om[-1.0], om[1.0], om[-1.0], om[1.0]])   # corners at y = -1, +1, -1, +1
    got_v = E @ v(x, y)[ix["B"]]
    assert np.allclose(got_v - v(x, y)[corners], -0.5 * miss, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("p,kappa", [(6, 3.0), (10, 20.0), (16, 40.0), (24, 50.0)])
def test_condense_with_mixed_term_manufactured(p, kappa):
    """c12 != 0: the corners enter through the corner extrapolation, so a
    tensor polynomial of degree p-3 is reproduced exactly by S u_b + W and
    T u_b + h (its analytic normal derivative), for any coefficient
    samples; at degree p-1 it is not (the corner values are extrapolated)."""
    rng = np.random.default_rng(500 + p)
    box = (0.5, 0.25, 0.125, 0.0625)
    coef = random_coef(rng, p * p, c12=True)
    u = random_poly(rng, p - 3, p - 3, xc=0.5625, yc=0.28125, sx=0.0625, sy=0.03125)
    e_int, e_flux, cond = condense_errors(p, box, coef, kappa, u)
    tol = max(1e-12, 100 * cond * EPS)
    assert e_int < tol, (e_int, cond)
    assert e_flux < tol, (e_flux, cond)
    v = random_poly(rng, p - 1, p - 1, xc=0.5625, yc=0.28125, sx=0.0625, sy=0.03125)
    assert condense_errors(p, box, coef, kappa, v)[0] > 100 * tol


def test_leaf_resolve_with_mixed_term_manufactured():
    """The re-formed leaf solve with c12 != 0 folds the corners the same way:
    exact for a degree p-3 tensor polynomial."""
    rng = np.random.default_rng(77)
    p, kappa = 12, 15.0
    box = (0.25, 0.5, 0.0625, 0.125)
    coef = random_coef(rng, p * p, c12=True)
    u = random_poly(rng, p - 3, p - 3, xc=0.28125, yc=0.5625, sx=0.03125, sy=0.0625)
    x, y = O.leaf_nodes(p, box)
    ix = O.leaf_index_sets(p)
    uv = u(x, y)[:, None]
    f = u.apply_operator(x, y, coef, kappa)[:, None]
    got = O.leaf_resolve(p, box, coef, kappa, uv[ix["B"]], f)
    assert O.relerr(got[ix["I"]], uv[ix["I"]]) < 1e-11


def psi_planewave_error(p, n=4, kappa=10.0):
    """The paper's curved domain Psi (Eq. (parametrization), operator of
    Eq. (chain_rule), c12 != 0): merged grid solve of n x n leaves with the
    physical plane wave as Dirichlet data, max error at the interior nodes."""
    w = WL.psi_curved(p=p, nx=n, ny=n, kappa=kappa, m=1)
    boxes = O.grid_boxes(n, n)
    coefs, fs = [], []
    for b in boxes:
        x, y = O.leaf_nodes(p, b)
        coefs.append(w.coefficients(x, y))
        fs.append(np.zeros((p * p, 1)))
    sol, _ = hps_grid_solve(p, n, n, coefs, kappa, fs, w.dirichlet_data)
    ix = O.leaf_index_sets(p)
    err = 0.0
    for l, s in enumerate(sol):
        x, y = O.leaf_nodes(p, boxes[l])
        err = max(err, float(np.abs(s["u_i"].ravel() - w.dirichlet_data(x, y)[ix["I"]]).max()))
    return err


def test_psi_curved_domain_spectral_convergence():
    """Section 3's curved domain: with the corner extrapolation the HPS
    solution converges spectrally to the exact plane wave as p grows."""
    errs = [psi_planewave_error(p) for p in (6, 10, 14)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-10, errs


def test_psi_curved_domain_fails_without_corner_reading(monkeypatch):
    """Dropping the corners (their values taken as zero) leaves an O(1e-2)
    error that does not decrease with p on the same problem."""
    real = O.corner_extrapolation
    monkeypatch.setattr(O, "corner_extrapolation", lambda p: 0.0 * real(p))
    errs = [psi_planewave_error(p) for p in (10, 14)]
    assert min(errs) > 1e-3, errs


@pytest.mark.parametrize("p,kappa,m", [(6, 3.0, 1), (12, 30.0, 2), (20, 200.0 / 8, 3)])
def test_leaf_resolve_manufactured(p, kappa, m):
    """Section 2 Remark: re-forming the leaf system and solving with the
    edge values reproduces a degree p-1 tensor polynomial at every non-corner
    node, for any coefficient samples; corners are returned as 0."""
    rng = np.random.default_rng(300 + p)
    box = (0.25, 0.5, 0.0625, 0.125)
    polys = [random_poly(rng, p - 1, p - 1, xc=0.28125, yc=0.5625, sx=0.03125, sy=0.0625) for _ in range(m)]
    coef = random_coef(rng, p * p)
    x, y = O.leaf_nodes(p, box)
    ix = O.leaf_index_sets(p)
    uv = np.stack([u(x, y) for u in polys], axis=1)
    f = np.stack([u.apply_operator(x, y, coef, kappa) for u in polys], axis=1)
    got = O.leaf_resolve(p, box, coef, kappa, uv[ix["B"]], f)
    A, _, _, _ = O.leaf_operator(p, box, coef, kappa)
    cond = np.linalg.cond(A[np.ix_(ix["I"], ix["I"])])
    mask = np.ones(p * p, bool)
    mask[[0, p - 1, (p - 1) * p, p * p - 1]] = False
    assert O.relerr(got[mask], uv[mask]) < max(1e-12, 100 * cond * EPS)
    assert np.all(got[~mask] == 0.0)


def test_leaf_resolve_equals_stored_operators():
    """The two routes to the interior values agree: a dense solve with the
    combined right-hand side f_I - A_ib u_b, and the stored S, W of the
    condensation (u_i = S u_b + W)."""
    rng = np.random.default_rng(7)
    p, kappa, m = 14, 40.0, 3
    box = (0.0, 0.0, 0.125, 0.125)
    coef = random_coef(rng, p * p)
    f = rng.standard_normal((p * p, m))
    ix = O.leaf_index_sets(p)
    ub = rng.standard_normal((len(ix["B"]), m))
    out = O.condense_leaf(p, box, coef, kappa, f)
    ui = O.leaf_interior_solve(out["S"], out["W"], ub)
    got = O.leaf_resolve(p, box, coef, kappa, ub, f)
    cond = np.linalg.cond(out["A_ii"])
    assert O.relerr(got[ix["I"]], ui) < max(1e-12, 100 * cond * EPS)
    assert np.array_equal(got[ix["B"]], ub)


def test_hps_merge_solve_manufactured():
    assert manufactured_grid_error() < 1e-10


def test_hps_merge_solve_manufactured_rectangular_grid():
    assert manufactured_grid_error(p=7, nx=2, ny=8, kappa=3.0, seed=5) < 1e-10


def test_merge_schedule():
    assert O.merge_schedule(8, 8) == ["x", "y"] * 3
    assert O.merge_schedule(2, 8) == ["x", "y", "y", "y"]
    assert O.merge_schedule(64, 128) == ["x", "y"] * 6 + ["y"]
    with pytest.raises(ValueError):
        O.merge_schedule(6, 8)


def planewave_case(p, nx=8, ny=8):
    w = WL.planewave(p=p, nx=nx, ny=ny)
    coefs, fs = [], []
    for box in w.boxes():
        x, y = O.leaf_nodes(p, box)
        coefs.append(w.coefficients(x, y))
        fs.append(w.body_load(x, y))
    return w, coefs, fs


def test_hps_equals_global_dense_solve_planewave():
    """Config: kappa = 20, b = 1, p = 10, 8 x 8 leaves (4096 interior + 896
    interface unknowns); merge tree vs brute-force dense solve of the same
    discrete system."""
    p = 10
    w, coefs, fs = planewave_case(p)
    sol, _ = hps_grid_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    dense, res = O.global_dense_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    A, rhs, lay = O.global_system(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    assert A.shape == (4992, 4992)
    assert res < 1e-12
    ref = [(d["u_b"], d["u_i"]) for d in dense]
    assert grid_error(sol, ref) < 1e-10


def test_planewave_spectral_convergence():
    errs = []
    for p in (6, 8, 10, 12, 14):
        w, coefs, fs = planewave_case(p)
        sol, _ = hps_grid_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
        errs.append(grid_error(sol, nodal_values(p, 8, 8, w.dirichlet_data)))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 10.0, errs
    assert errs[-1] < 1e-8, errs


def test_j0_spectral_convergence():
    """The paper's closed-form test: u = J0(kappa |x - (-0.1, 0.5)|) solves the
    homogeneous Helmholtz equation on [0,1]^2 (Section 3)."""
    kappa = 20.0

    def u_true(x, y):
        return scipy.special.j0(kappa * np.hypot(x + 0.1, y - 0.5))

    errs = []
    for p in (8, 11, 14):
        w, coefs, fs = planewave_case(p)
        sol, _ = hps_grid_solve(p, 8, 8, coefs, kappa, fs, u_true)
        errs.append(grid_error(sol, nodal_values(p, 8, 8, u_true)))
    assert errs[1] < errs[0] / 30 and errs[2] < errs[1] / 30, errs
    assert errs[-1] < 1e-8, errs


def test_dtn_maps_planewave_trace_to_normal_derivative():
    kappa, d = 20.0, (0.6, 0.8)
    errs = []
    for p in (8, 12, 16, 20):
        box = (0.25, 0.5, 0.125, 0.125)
        x, y = O.leaf_nodes(p, box)
        coef = np.stack([np.ones(p * p), 0 * x, np.ones(p * p), 0 * x, 0 * x, np.ones(p * p)])
        out = O.condense_leaf(p, box, coef, kappa)
        ix = O.leaf_index_sets(p)
        u = np.sin(kappa * (d[0] * x + d[1] * y))
        ux = kappa * d[0] * np.cos(kappa * (d[0] * x + d[1] * y))
        uy = kappa * d[1] * np.cos(kappa * (d[0] * x + d[1] * y))
        dn = np.concatenate([-ux[ix["W"]], ux[ix["E"]], -uy[ix["S"]], uy[ix["N"]]])
        errs.append(O.relerr(out["T"] @ u[ix["B"]], dn))
        # S maps the trace to the interior values
        assert O.relerr(out["S"] @ u[ix["B"]], u[ix["I"]]) < max(10 * errs[-1], 1e-12)
    assert errs[-1] < 1e-9 and errs[1] < errs[0] / 100, errs


# ----------------------------------------------------- planted-mistake checks

def _leaf_pins():
    rng = np.random.default_rng(3)
    p, box, kappa = 8, (0.0, 0.0, 0.25, 0.125), 9.0
    u = random_poly(rng, p - 1, p - 1, xc=0.125, yc=0.0625, sx=0.125, sy=0.0625)
    coef = random_coef(rng, p * p)
    e_op = operator_error(p, box, coef, kappa, u)
    e_int, e_flux, _ = condense_errors(p, box, coef, kappa, u)
    return max(e_op, e_int, e_flux), manufactured_grid_error(p=6, nx=2, ny=2, seed=4)


def test_pins_pass_unmutated():
    leaf, grid = _leaf_pins()
    assert leaf < 1e-10 and grid < 1e-10


@pytest.mark.parametrize("mutation", ["transpose_D", "flip_west_normal", "drop_c1",
                                      "kappa_sign", "c12_factor", "swap_merge_order",
                                      "corner_ends_swapped", "corners_dropped"])
def test_planted_mistake_is_caught(monkeypatch, mutation):
    real_diff, real_op, real_keys = O.cheb_diff, O.leaf_operator, O.box_keys
    if mutation == "transpose_D":
        monkeypatch.setattr(O, "cheb_diff", lambda p: real_diff(p).T)
    elif mutation == "flip_west_normal":
        def op(p, box, coef, kappa):
            A, N, Dx, Dy = real_op(p, box, coef, kappa)
            N = N.copy()
            N[: p - 2] *= -1.0
            return A, N, Dx, Dy
        monkeypatch.setattr(O, "leaf_operator", op)
    elif mutation == "drop_c1":
        def op(p, box, coef, kappa):
            c = np.array(coef, dtype=float)
            A, N, Dx, Dy = real_op(p, box, c, kappa)
            return A + c[3][:, None] * Dx, N, Dx, Dy
        monkeypatch.setattr(O, "leaf_operator", op)
    elif mutation == "kappa_sign":
        def op(p, box, coef, kappa):
            A, N, Dx, Dy = real_op(p, box, coef, kappa)
            return A + 2 * kappa ** 2 * np.diag(np.asarray(coef[5], float)), N, Dx, Dy
        monkeypatch.setattr(O, "leaf_operator", op)
    elif mutation == "c12_factor":
        def op(p, box, coef, kappa):
            A, N, Dx, Dy = real_op(p, box, coef, kappa)
            return A + np.asarray(coef[1], float)[:, None] * (Dx @ Dy), N, Dx, Dy
        monkeypatch.setattr(O, "leaf_operator", op)
    if mutation in ("corner_ends_swapped", "corners_dropped"):
        real_E = O.corner_extrapolation
        if mutation == "corner_ends_swapped":
            monkeypatch.setattr(O, "corner_extrapolation", lambda p: real_E(p)[::-1])
        else:
            monkeypatch.setattr(O, "corner_extrapolation", lambda p: 0.0 * real_E(p))
        rng = np.random.default_rng(9)
        p, box = 9, (0.0, 0.0, 0.25, 0.125)
        u = random_poly(rng, p - 3, p - 3, xc=0.125, yc=0.0625, sx=0.125, sy=0.0625)
        e_int, e_flux, _ = condense_errors(p, box, random_coef(rng, p * p, c12=True), 5.0, u)
        assert max(e_int, e_flux) > 1e-6, (e_int, e_flux)
        return
    if mutation == "c12_factor":
        rng = np.random.default_rng(8)
        p, box = 8, (0.0, 0.0, 0.25, 0.125)
        u = random_poly(rng, p - 1, p - 1, xc=0.125, yc=0.0625, sx=0.125, sy=0.0625)
        err = operator_error(p, box, random_coef(rng, p * p, c12=True), 5.0, u)
        assert err > 1e-6
        return
    if mutation == "swap_merge_order":
        # leaf T is computed in [W, E, S, N] order; reversed leaf keys mislabel
        # its rows, so the solve goes wrong or the key bookkeeping rejects it
        def keys_bad(p, ix0, iy0, wx, wy):
            k = real_keys(p, ix0, iy0, wx, wy)
            return k[::-1] if (wx, wy) == (1, 1) else k
        monkeypatch.setattr(O, "box_keys", keys_bad)
        try:
            err = manufactured_grid_error(p=6, nx=2, ny=2, seed=4)
        except (AssertionError, KeyError):
            return
        assert err > 1e-6, err
        return
    leaf, grid = _leaf_pins()
    assert max(leaf, grid) > 1e-6, (leaf, grid)


# ------------------------------------------------------------------ SlabLU

def _grid_leaves(p, nx, ny, coefs, kappa, fs):
    boxes = O.grid_boxes(nx, ny)
    return [O.condense_leaf(p, boxes[l], coefs[l], kappa, fs[l]) for l in range(nx * ny)]


def _gkeys(p, nx, ny, g_fn):
    return {k: np.atleast_1d(g_fn(*O.key_coords(p, k, nx, ny))) for k in O.outer_boundary_keys(p, nx, ny)}


def test_reduced_system_holds_for_the_merge_tree_solution():
    """The merge tree's edge values satisfy every flux-continuity row of the
    reduced system of Eq. (hps_reduced) to rounding; its size is the number
    of interface nodes (896 for 8 x 8 leaves of p = 10)."""
    p = 10
    w, coefs, fs = planewave_case(p)
    sol, leaves = hps_grid_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    A, f, keys = O.reduced_system(p, 8, 8, leaves, _gkeys(p, 8, 8, w.dirichlet_data))
    assert A.shape == (896, 896)
    vals = {}
    for l, s in enumerate(sol):
        ix, iy = divmod(l, 8)
        for k, v in zip(O.box_keys(p, ix, iy, 1, 1), s["u_b"]):
            vals[k] = v
    u = np.array([vals[k] for k in keys])
    assert np.abs(A @ u - f).max() / (np.abs(A) @ np.abs(u) + np.abs(f)).max() < 1e-13


@pytest.mark.parametrize("s", [2, 4])
def test_slab_blocks_are_block_tridiagonal(s):
    """Eq. (dell1): slab interiors do not interact with each other, a slab
    touches only the interfaces on its two sides, an interface only the
    slabs beside it (slabs at least two leaves wide)."""
    p, nx, ny = 6, 8, 4
    rng = np.random.default_rng(2)
    coefs = [random_coef(rng, p * p) for _ in range(nx * ny)]
    fs = [rng.standard_normal((p * p, 1)) for _ in range(nx * ny)]
    leaves = _grid_leaves(p, nx, ny, coefs, 5.0, fs)
    A, _, keys = O.reduced_system(p, nx, ny, leaves, _gkeys(p, nx, ny, lambda x, y: 0.0 * x))
    I, G = O.slab_blocks(p, nx, s, keys)
    S = nx // s
    assert len(I) == S and len(G) == S - 1
    assert sorted(sum(I, []) + sum(G, [])) == list(range(len(keys)))
    for a in range(S):
        for b in range(S):
            blk = A[np.ix_(I[a], I[b])]
            assert (np.abs(blk).max() > 0) == (a == b), (a, b)
        for k in range(S - 1):
            touches = np.abs(A[np.ix_(I[a], G[k])]).max() > 0
            assert touches == (k in (a - 1, a)), (a, k)
    for k in range(S - 1):
        for k2 in range(S - 1):
            assert (np.abs(A[np.ix_(G[k], G[k2])]).max() > 0) == (k == k2)


@pytest.mark.parametrize("s", [2, 4, 8])
def test_slab_solve_equals_merge_tree_and_dense_solve(s):
    """SlabLU and the merge tree eliminate the same reduced system in
    different orders: same solution; and the brute-force dense solve of
    the global system (plane wave, kappa = 20, p = 10, 8 x 8 leaves)."""
    p = 10
    w, coefs, fs = planewave_case(p)
    sol, leaves = hps_grid_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    slab = O.slab_downward(p, 8, 8, s, leaves, _gkeys(p, 8, 8, w.dirichlet_data))
    ref = [(d["u_b"], d["u_i"]) for d in sol]
    assert grid_error(slab, ref) < 1e-12
    dense, _ = O.global_dense_solve(p, 8, 8, coefs, w.kappa, fs, w.dirichlet_data)
    assert grid_error(slab, [(d["u_b"], d["u_i"]) for d in dense]) < 1e-10


def test_slab_solve_manufactured():
    """A tensor polynomial of degree p-1 with random coefficient samples is
    reproduced exactly through condensation and SlabLU (4 slabs of 2)."""
    p, nx, ny, kappa = 8, 8, 4, 7.0
    rng = np.random.default_rng(17)
    u = random_poly(rng, p - 1, p - 1, xc=0.5, yc=0.5, sx=0.5, sy=0.5)
    coefs, fs = [], []
    for box in O.grid_boxes(nx, ny):
        x, y = O.leaf_nodes(p, box)
        c = random_coef(rng, p * p)
        coefs.append(c)
        fs.append(u.apply_operator(x, y, c, kappa)[:, None])
    leaves = _grid_leaves(p, nx, ny, coefs, kappa, fs)
    sol = O.slab_downward(p, nx, ny, 2, leaves, _gkeys(p, nx, ny, lambda x, y: u(x, y)))
    assert grid_error(sol, nodal_values(p, nx, ny, u)) < 1e-10


def test_slab_planted_mistakes_are_caught(monkeypatch):
    """A horizontal edge put in the neighbouring slab breaks the block form;
    a sign error in the reduced system's Dirichlet terms breaks the solve."""
    real = O.slab_blocks

    def shifted(p, nx, s, keys):
        I, G = real(p, nx, s, keys)
        moved = [i for i in I[0] if keys[i][0] == "h"][:1]
        return [[i for i in I[0] if i not in moved]] + [I[1] + moved] + I[2:], G
    monkeypatch.setattr(O, "slab_blocks", shifted)
    with pytest.raises(AssertionError):
        test_slab_blocks_are_block_tridiagonal(2)
    monkeypatch.setattr(O, "slab_blocks", real)
    real_rs = O.reduced_system

    def flipped(p, nx, ny, leaves, g_keys):
        return real_rs(p, nx, ny, leaves, {k: -v for k, v in g_keys.items()})
    monkeypatch.setattr(O, "reduced_system", flipped)
    with pytest.raises(AssertionError):
        test_slab_solve_equals_merge_tree_and_dense_solve(2)


# --------------------------------------------- impedance-to-impedance maps

def _analytic_flux(u, x, y, ix):
    dudx, dudy = u(x, y, 1, 0), u(x, y, 0, 1)
    return np.concatenate([-dudx[ix["W"]], dudx[ix["E"]], -dudy[ix["S"]], dudy[ix["N"]]])


@pytest.mark.parametrize("c12", [False, True])
def test_iti_leaf_manufactured(c12):
    """A tensor polynomial with random coefficient samples: from its
    incoming impedance data u_n + i eta u the leaf solve reproduces it at
    every node, and R f + h is its outgoing data u_n - i eta u (u_n the
    analytic outward normal derivative; degree p - 1, or p - 3 with the
    corner extrapolation of the mixed term)."""
    rng = np.random.default_rng(31)
    p, box, kappa, eta = 9, (0.25, 0.5, 0.25, 0.125), 6.0, 4.0
    deg = p - 3 if c12 else p - 1
    u = random_poly(rng, deg, deg, xc=0.375, yc=0.5625, sx=0.125, sy=0.0625)
    coef = random_coef(rng, p * p, c12=c12)
    x, y = O.leaf_nodes(p, box)
    f = u.apply_operator(x, y, coef, kappa)[:, None]
    ix = O.leaf_index_sets(p)
    out = O.iti_leaf(p, box, coef, kappa, eta, f)
    uv = u(x, y)
    dn = _analytic_flux(u, x, y, ix)
    f_in = (dn + 1j * eta * uv[ix["B"]])[:, None]
    sol = out["Y"] @ f_in + out["uf"]
    assert np.abs(sol[: len(ix["I"]), 0] - uv[ix["I"]]).max() / np.abs(uv).max() < 1e-10
    assert np.abs(sol[len(ix["I"]):, 0] - uv[ix["B"]]).max() / np.abs(uv).max() < 1e-10
    g = out["R"] @ f_in + out["h"]
    ref = dn - 1j * eta * uv[ix["B"]]
    assert np.abs(g[:, 0] - ref).max() / np.abs(ref).max() < 1e-10


def test_iti_is_the_cayley_transform_of_the_dtn_map():
    """Where the DtN map exists: u_b = (T + i eta)^{-1} (f - h_D) gives
    R = (T - i eta)(T + i eta)^{-1} and h = (I - R) h_D (an algebraic
    identity between two independent computations)."""
    rng = np.random.default_rng(5)
    p, box, kappa, eta = 10, (0.0, 0.0, 0.125, 0.125), 20.0, 20.0
    coef = random_coef(rng, p * p)
    f = rng.standard_normal((p * p, 2))
    d = O.condense_leaf(p, box, coef, kappa, f)
    it = O.iti_leaf(p, box, coef, kappa, eta, f)
    nb = d["T"].shape[0]
    Rc = np.linalg.solve((d["T"] + 1j * eta * np.eye(nb)).T, (d["T"] - 1j * eta * np.eye(nb)).T).T
    assert np.abs(it["R"] - Rc).max() / np.abs(Rc).max() < 1e-11
    hc = (np.eye(nb) - Rc) @ d["h"]
    assert np.abs(it["h"] - hc).max() / np.abs(hc).max() < 1e-11


def _resonant_leaf_grid(p=8, n=2):
    """An n x n grid of leaves with constant coefficients, b = 1 + 0.25 l on
    leaf l, and kappa^2 the smallest eigenvalue of leaf 0's discrete
    Dirichlet operator: leaf 0's A_ii is singular (a Dirichlet resonance),
    the other leaves and the global problem are not."""
    boxes = O.grid_boxes(n, n)
    one, zero = np.ones(p * p), np.zeros(p * p)
    coefs = [np.stack([one, zero, one, zero, zero, (1.0 + 0.25 * l) * one]) for l in range(n * n)]
    A0, _, _, _ = O.leaf_operator(p, boxes[0], coefs[0], 0.0)
    I = O.leaf_index_sets(p)["I"]
    lam = np.linalg.eigvals(A0[np.ix_(I, I)])
    return float(np.sqrt(np.min(lam.real))), coefs


def test_iti_solves_through_leaf_resonances():
    """A leaf at a Dirichlet resonance (cond(A_ii) ~ 1/eps, its DtN map does
    not exist): the ItI merge and solve still equals the brute-force dense
    solve of the global system."""
    p, n = 8, 2
    kappa, coefs = _resonant_leaf_grid(p, n)
    boxes = O.grid_boxes(n, n)
    I = O.leaf_index_sets(p)["I"]
    A_ii = O.leaf_operator(p, boxes[0], coefs[0], kappa)[0][np.ix_(I, I)]
    assert np.linalg.cond(A_ii) > 1e12
    g_fn = lambda x, y: np.sin(kappa * (0.6 * x + 0.8 * y))
    fs = [np.zeros((p * p, 1)) for _ in range(n * n)]
    leaves = [O.iti_leaf(p, b, coefs[l], kappa, kappa, fs[l]) for l, b in enumerate(boxes)]
    gk = {k: np.atleast_1d(g_fn(*O.key_coords(p, k, n, n))) for k in O.outer_boundary_keys(p, n, n)}
    sol = O.iti_solve(p, n, n, leaves, gk, kappa)
    dense, res = O.global_dense_solve(p, n, n, coefs, kappa, fs, g_fn)
    assert res < 1e-12
    ref = [(d["u_b"], d["u_i"]) for d in dense]
    assert grid_error(sol, ref) < 1e-9
    # the DtN merge tree on the same leaves loses its accuracy there
    dl = [O.condense_leaf(p, b, coefs[l], kappa, fs[l]) for l, b in enumerate(boxes)]
    dtn = O.hps_downward(p, n, n, O.hps_upward(p, n, n, dl), dl, gk)
    assert grid_error(dtn, ref) > 1e-4


def test_iti_solve_equals_merge_tree():
    p = 10
    w, coefs, fs = planewave_case(p, 4, 4)
    sol, _ = hps_grid_solve(p, 4, 4, coefs, w.kappa, fs, w.dirichlet_data)
    boxes = O.grid_boxes(4, 4)
    leaves = [O.iti_leaf(p, boxes[l], coefs[l], w.kappa, w.kappa, fs[l]) for l in range(16)]
    gk = {k: np.atleast_1d(w.dirichlet_data(*O.key_coords(p, k, 4, 4))) for k in O.outer_boundary_keys(p, 4, 4)}
    it = O.iti_solve(p, 4, 4, leaves, gk, w.kappa)
    assert grid_error(it, [(d["u_b"], d["u_i"]) for d in sol]) < 1e-12


def test_iti_planted_sign_is_caught(monkeypatch):
    """Incoming data on the shared edge taken as +g of the other box (the
    normals' opposition dropped) breaks the merged solve."""
    real = O.iti_merge_two

    def wrong(ka, Ra, ha, kb, Rb, hb, kpar):
        return real(ka, Ra, ha, kb, -Rb, -hb, kpar)
    monkeypatch.setattr(O, "iti_merge_two", wrong)
    with pytest.raises(AssertionError):
        test_iti_solve_equals_merge_tree()
