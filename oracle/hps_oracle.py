"""FP64 CPU oracle for the HPS leaf static condensation, merge and solve.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain, obviously correct
statement of what the GPU library computes.  Only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import or run it; the
product path (the CUDA library and its Python binding) never does, and this
module imports nothing from the product package.  Coefficients, body loads
and boundary data are passed in as arrays; the seeded workload generators
live elsewhere and hold none of the arithmetic below.

Everything is float64 numpy, with LAPACK (scipy.linalg.lu_factor/lu_solve)
and numpy.linalg.solve as the only library primitives.

Paper: Yesypenko & Martinsson, "GPU Optimizations for the Hierarchical
Poincare-Steklov Scheme" (arXiv 2211.14969).  Citations below are to its
sections and equations:

* Eq. (bvp), Eq. (var_helm): the BVP  A u = f in Omega, u = g on dOmega,
  with A u = -Lap u - kappa^2 b(x) u.
* Section 2: p x p tensor mesh of Chebyshev points per leaf, spectral
  collocation of the PDE at interior nodes, flux continuity on element
  boundaries, static condensation of the interior nodes leaving the reduced
  system of Eq. (hps_reduced) on the leaf edges.
* Section 2 Remark: leaf factorizations are re-formed after the reduced solve.
* Eq. (chain_rule): the general second-order form with mixed derivative,
  which fixes the "2 c12 d^2/dx1dx2" convention of the operator here.
* Eq. (accuracy_formula): relerr_res and relerr_true.

The paper defers the formulas of the leaf solution operator, the
Dirichlet-to-Neumann (DtN) map and the merge to its references
[babb2018accelerated, 2019_martinsson_book, hao2016direct]; the standard
forms are used:  S = -A_ii^{-1} A_ib,  T = N_b + N_i S,  and the merge of two
boxes as a Schur complement on their shared edge.

Readings where the paper is silent (each is also listed in the design notes):
* p is the number of Chebyshev points per direction (degree p-1).
* Leaf corners are not unknowns.  With c12 == 0 no interior or normal row
  touches a corner, so dropping them is exact.  With c12 != 0 the mixed
  derivative at an interior node reaches the four corners; each corner
  value is then taken as the average of the two polynomial extrapolations,
  of degree p-3, through the p-2 edge nodes of its two adjacent edges
  (corner_extrapolation), so the corner columns fold into the edge columns:
  A_ib <- A_ib + A_ic E.  Exact for tensor polynomials of degree <= p-3.
* Node id i*p + j, i the x index; interior nodes lexicographic (i major);
  boundary order [W, E, S, N], each edge by increasing coordinate.
* Normal rows use the outward normal: -d/dx on W, +d/dx on E, -d/dy on S,
  +d/dy on N, so flux continuity across an interface is "sum == 0".
* Merges alternate x then y (x first), siblings ordered west/east or
  south/north; the parent boundary is again [W, E, S, N] by increasing
  coordinate.
"""

import numpy as np
import scipy.linalg as sla

# ----------------------------------------------------------------------------
# Chebyshev grid and differentiation  (Section 2: "p x p tensor product mesh of
# Chebyshev points", "spectral differentiation")
# ----------------------------------------------------------------------------


def cheb_points(p):
    """The p Chebyshev-Gauss-Lobatto points on [-1, 1] in increasing order."""
    k = np.arange(p, dtype=np.float64)
    return -np.cos(np.pi * k / (p - 1))


def cheb_diff(p):
    """Chebyshev spectral differentiation matrix on cheb_points(p).

    Textbook definition (Trefethen, Spectral Methods in MATLAB, ch. 6):
    off-diagonal D[i, j] = (c_i / c_j) (-1)^(i+j) / (t_i - t_j) with
    c_0 = c_{p-1} = 2 and c_k = 1 otherwise; the diagonal is minus the row sum
    of the off-diagonal entries (D applied to a constant is zero).
    """
    t = cheb_points(p)
    c = np.ones(p)
    c[0] = 2.0
    c[-1] = 2.0
    D = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            if i != j:
                D[i, j] = (c[i] / c[j]) * (-1.0) ** (i + j) / (t[i] - t[j])
    for i in range(p):
        D[i, i] = -(D[i, :].sum() - D[i, i])
    return D


def leaf_nodes(p, box):
    """Node coordinates (x, y), each of length p*p, node id i*p + j.

    box = (x0, y0, hx, hy); x_i = x0 + (1 + t_i) hx / 2, likewise y_j.
    """
    x0, y0, hx, hy = box
    t = cheb_points(p)
    xs = x0 + (1.0 + t) * hx / 2.0
    ys = y0 + (1.0 + t) * hy / 2.0
    X = np.repeat(xs, p)   # x index i is the slow one
    Y = np.tile(ys, p)
    return X, Y


def leaf_index_sets(p):
    """Interior set I and boundary edges W, E, S, N (corners dropped)."""
    q = range(1, p - 1)
    I = [i * p + j for i in q for j in q]
    W = [0 * p + j for j in q]
    E = [(p - 1) * p + j for j in q]
    S = [i * p + 0 for i in q]
    N = [i * p + (p - 1) for i in q]
    return {"I": I, "W": W, "E": E, "S": S, "N": N, "B": W + E + S + N}


def corner_extrapolation(p):
    """E (4 x n_b): the corner values from the edge values.

    Corners in node order [(0, 0), (0, p-1), (p-1, 0), (p-1, p-1)] (node id
    i*p + j, i the x index); edge nodes in the boundary order [W, E, S, N].
    A corner's value is the mean of the extrapolations along its two
    adjacent edges, each the polynomial of degree p-3 through that edge's
    p-2 interior Chebyshev nodes evaluated at the edge's end (the reading
    for c12 != 0, where the mixed derivative reaches the corners).  Lagrange
    basis by its product formula.
    """
    q = p - 2
    t = cheb_points(p)[1:p - 1]          # interior nodes on [-1, 1], increasing

    def ends(at):
        out = np.ones(q)
        for k in range(q):
            for m in range(q):
                if m != k:
                    out[k] *= (at - t[m]) / (t[k] - t[m])
        return out

    lo, hi = ends(-1.0), ends(1.0)
    W, E, S, N = (slice(0, q), slice(q, 2 * q), slice(2 * q, 3 * q), slice(3 * q, 4 * q))
    Emat = np.zeros((4, 4 * q))
    # (x, y) = (-1, -1): along W to y = -1, along S to x = -1
    Emat[0, W] += 0.5 * lo
    Emat[0, S] += 0.5 * lo
    # (-1, +1): W to y = +1, N to x = -1
    Emat[1, W] += 0.5 * hi
    Emat[1, N] += 0.5 * lo
    # (+1, -1): E to y = -1, S to x = +1
    Emat[2, E] += 0.5 * lo
    Emat[2, S] += 0.5 * hi
    # (+1, +1): E to y = +1, N to x = +1
    Emat[3, E] += 0.5 * hi
    Emat[3, N] += 0.5 * hi
    return Emat


def corner_ids(p):
    return [0, p - 1, (p - 1) * p, p * p - 1]


def leaf_operator(p, box, coef, kappa):
    """Full p^2 x p^2 collocation matrix of the leaf and its normal rows.

    coef is a (6, p*p) array of (c11, c12, c22, c1, c2, b) at the leaf nodes.
    The operator is the variable-coefficient Helmholtz operator of
    Eq. (var_helm) in the general form of Eq. (chain_rule):
        A u = -(c11 u_xx + 2 c12 u_xy + c22 u_yy + c1 u_x + c2 u_y)
              - kappa^2 b u,
    with the derivatives replaced by Kronecker products of the 1D Chebyshev
    matrix scaled to the leaf (Section 2).  Returns (A, Nrow, Dx, Dy), where
    Nrow (n_b x p^2) holds the outward normal derivative at the boundary
    nodes in [W, E, S, N] order.
    """
    x0, y0, hx, hy = box
    D = cheb_diff(p)
    Ip = np.eye(p)
    Dx = np.kron((2.0 / hx) * D, Ip)   # acts on the x index i of id i*p+j
    Dy = np.kron(Ip, (2.0 / hy) * D)   # acts on the y index j
    c11, c12, c22, c1, c2, b = (np.asarray(c, dtype=np.float64) for c in coef)
    A = -(c11[:, None] * (Dx @ Dx)
          + 2.0 * c12[:, None] * (Dx @ Dy)
          + c22[:, None] * (Dy @ Dy)
          + c1[:, None] * Dx
          + c2[:, None] * Dy)
    A = A - kappa ** 2 * np.diag(b)
    ix = leaf_index_sets(p)
    Nrow = np.vstack([-Dx[ix["W"]], Dx[ix["E"]], -Dy[ix["S"]], Dy[ix["N"]]])
    return A, Nrow, Dx, Dy


# ----------------------------------------------------------------------------
# Leaf static condensation  (Section 2: eliminate the interior nodes of each
# leaf with dense LU and matrix-matrix products)
# ----------------------------------------------------------------------------


def condense_leaf(p, box, coef, kappa, f=None):
    """Condense one leaf.

    f is the body load at the p*p nodes, shape (p*p, m) (or None for m = 0).
    Returns a dict with
        S (n_i x n_b) = -A_ii^{-1} A_ib     solution operator,
        T (n_b x n_b) = N_b + N_i S         DtN map,
        W (n_i x m)   = A_ii^{-1} f_I       particular interior solution,
        h (n_b x m)   = N_i W               its outgoing flux,
    and the blocks used (A_ii, A_ib, N_b, N_i) for diagnostics.
    With u_i = S u_b + W on the leaf, the outgoing flux is T u_b + h.
    """
    A, Nrow, _, _ = leaf_operator(p, box, coef, kappa)
    ix = leaf_index_sets(p)
    I, B = ix["I"], ix["B"]
    A_ii = A[np.ix_(I, I)]
    A_ib = interior_edge_block(A, p)
    N_b = Nrow[:, B]
    N_i = Nrow[:, I]
    lu = sla.lu_factor(A_ii)
    S = -sla.lu_solve(lu, A_ib)
    T = N_b + N_i @ S
    out = {"S": S, "T": T, "A_ii": A_ii, "A_ib": A_ib, "N_b": N_b, "N_i": N_i}
    if f is not None:
        f = np.asarray(f, dtype=np.float64).reshape(p * p, -1)
        W = sla.lu_solve(lu, f[I])
        out["W"] = W
        out["h"] = N_i @ W
    return out


def interior_edge_block(A, p):
    """A_ib with the corner columns folded in through the corner
    extrapolation: A_ib + A_ic E (A_ic is zero when c12 == 0)."""
    ix = leaf_index_sets(p)
    I, B = ix["I"], ix["B"]
    A_ib = A[np.ix_(I, B)]
    A_ic = A[np.ix_(I, corner_ids(p))]
    if np.any(A_ic != 0.0):
        A_ib = A_ib + A_ic @ corner_extrapolation(p)
    return A_ib


def leaf_interior_solve(S, W, u_b):
    """Interior values from boundary values: u_i = S u_b + W (Section 2 Remark)."""
    u_b = np.asarray(u_b).reshape(S.shape[1], -1)
    return S @ u_b + (0.0 if W is None else W)


def leaf_resolve(p, box, coef, kappa, u_b, f=None):
    """Leaf solve by re-forming the leaf system (Section 2 Remark: the leaf
    factorizations are not kept but formed again after the reduced solve;
    Section 4: the leaf systems are re-factorized to obtain the solution on
    the full grid).  The interior values are the solution of
        A_ii u_i = f_I - A_ib u_b
    by a plain dense solve.  u_b: edge values (n_b x m, [W, E, S, N]); f: the
    body load at the p*p nodes (p*p x m) or None.  Returns u at all p*p nodes
    (p*p x m): interior from the solve, edges from u_b, corners 0 (they are
    not unknowns)."""
    A, _, _, _ = leaf_operator(p, box, coef, kappa)
    ix = leaf_index_sets(p)
    I, B = ix["I"], ix["B"]
    u_b = np.asarray(u_b, dtype=np.float64).reshape(len(B), -1)
    rhs = -interior_edge_block(A, p) @ u_b
    if f is not None:
        rhs = rhs + np.asarray(f, dtype=np.float64).reshape(p * p, -1)[I]
    u = np.zeros((p * p, u_b.shape[1]))
    u[I] = np.linalg.solve(A[np.ix_(I, I)], rhs)
    u[B] = u_b
    return u


# ----------------------------------------------------------------------------
# Uniform grids of leaves: edge-node keys, merges and the downward solve
# ----------------------------------------------------------------------------
#
# An edge node is named by a key (kind, line, seg, k):
#   kind 'v': the vertical grid line x = line * hx, seg = leaf row iy,
#   kind 'h': the horizontal grid line y = line * hy, seg = leaf column ix,
#   k = 0 .. p-3 along the edge by increasing coordinate.


def grid_boxes(nx, ny, x0=0.0, y0=0.0, lx=1.0, ly=1.0):
    """Leaf boxes of an nx x ny tiling, leaf index ix * ny + iy."""
    hx, hy = lx / nx, ly / ny
    return [(x0 + ix * hx, y0 + iy * hy, hx, hy) for ix in range(nx) for iy in range(ny)]


def box_keys(p, ix0, iy0, wx, wy):
    """Boundary keys of the box of leaves [ix0, ix0+wx) x [iy0, iy0+wy), [W, E, S, N]."""
    ks = range(p - 2)
    W = [("v", ix0, iy, k) for iy in range(iy0, iy0 + wy) for k in ks]
    E = [("v", ix0 + wx, iy, k) for iy in range(iy0, iy0 + wy) for k in ks]
    S = [("h", iy0, ix, k) for ix in range(ix0, ix0 + wx) for k in ks]
    N = [("h", iy0 + wy, ix, k) for ix in range(ix0, ix0 + wx) for k in ks]
    return W + E + S + N


def merge_schedule(nx, ny):
    """Merge directions bottom-up: 'x' first, then alternate; one direction
    continues alone once the other spans the grid.  nx, ny powers of two."""
    for n in (nx, ny):
        if n < 1 or (n & (n - 1)):
            raise ValueError("merge tree needs power-of-two leaf counts")
    wx, wy, out = 1, 1, []
    while wx < nx or wy < ny:
        if wx < nx and (wx <= wy or wy == ny):
            out.append("x")
            wx *= 2
        else:
            out.append("y")
            wy *= 2
    return out


def merge_two(ka, Ta, ha, kb, Tb, hb, kpar):
    """Merge sibling boxes alpha and beta along their shared edge (Schur
    complement; the merge the paper defers to its HPS references).

    ka, kb, kpar: boundary key lists; T*, h*: DtN maps and outgoing fluxes in
    those orders.  With 1 = alpha's exterior, 2 = beta's exterior, 3 = shared:
        Z  = Ta33 + Tb33
        S3 = -Z^{-1} [Ta31  Tb32],   w3 = -Z^{-1} (ha3 + hb3)
        T  = diag(Ta11, Tb22) + [Ta13; Tb23] S3
        h  = [ha1; hb2] + [Ta13; Tb23] w3
    T and h are returned in kpar order, S3 maps [u1; u2] (in the order
    `k12`) to the shared-edge values (in the order `k3`).
    """
    pa = {k: i for i, k in enumerate(ka)}
    pb = {k: i for i, k in enumerate(kb)}
    k3 = [k for k in ka if k in pb]
    k1 = [k for k in ka if k not in pb]
    k2 = [k for k in kb if k not in pa]
    a1 = [pa[k] for k in k1]
    a3 = [pa[k] for k in k3]
    b2 = [pb[k] for k in k2]
    b3 = [pb[k] for k in k3]
    Z = Ta[np.ix_(a3, a3)] + Tb[np.ix_(b3, b3)]
    rhs = np.hstack([Ta[np.ix_(a3, a1)], Tb[np.ix_(b3, b2)]])
    lu = sla.lu_factor(Z)
    S3 = -sla.lu_solve(lu, rhs)
    w3 = -sla.lu_solve(lu, ha[a3] + hb[b3])
    n1, n2 = len(k1), len(k2)
    T12 = np.zeros((n1 + n2, n1 + n2))
    T12[:n1, :n1] = Ta[np.ix_(a1, a1)]
    T12[n1:, n1:] = Tb[np.ix_(b2, b2)]
    C = np.vstack([Ta[np.ix_(a1, a3)], Tb[np.ix_(b2, b3)]])
    T12 = T12 + C @ S3
    h12 = np.vstack([ha[a1], hb[b2]]) + C @ w3
    k12 = k1 + k2
    pos = {k: i for i, k in enumerate(k12)}
    perm = [pos[k] for k in kpar]
    if sorted(perm) != list(range(n1 + n2)):
        raise AssertionError("parent keys are not the exterior of the children")
    T = T12[np.ix_(perm, perm)]
    h = h12[perm]
    return {"T": T, "h": h, "S3": S3, "w3": w3, "k12": k12, "k3": k3}


def hps_upward(p, nx, ny, leaves):
    """Bottom-up merges over an nx x ny grid of condensed leaves.

    leaves[ix * ny + iy] holds the leaf's T and h.  Returns the list of levels;
    each level is a dict mapping the box origin (ix0, iy0) to its record.
    """
    boxes = {}
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            boxes[(ix, iy)] = {"T": lf["T"], "h": lf["h"], "keys": box_keys(p, ix, iy, 1, 1)}
    wx, wy = 1, 1
    levels = []
    for d in merge_schedule(nx, ny):
        new = {}
        for (ix0, iy0) in sorted(boxes):
            if d == "x" and (ix0 // wx) % 2 == 0:
                a, b = boxes[(ix0, iy0)], boxes[(ix0 + wx, iy0)]
                kpar = box_keys(p, ix0, iy0, 2 * wx, wy)
            elif d == "y" and (iy0 // wy) % 2 == 0:
                a, b = boxes[(ix0, iy0)], boxes[(ix0, iy0 + wy)]
                kpar = box_keys(p, ix0, iy0, wx, 2 * wy)
            else:
                continue
            rec = merge_two(a["keys"], a["T"], a["h"], b["keys"], b["T"], b["h"], kpar)
            rec["keys"] = kpar
            rec["children"] = ((ix0, iy0), (ix0 + wx, iy0) if d == "x" else (ix0, iy0 + wy))
            new[(ix0, iy0)] = rec
        if d == "x":
            wx *= 2
        else:
            wy *= 2
        boxes = new
        levels.append(new)
    return levels


def hps_downward(p, nx, ny, levels, leaves, g_keys):
    """Top-down solve (Section 2 Remark: leaf values after the reduced solve).

    g_keys: dict key -> Dirichlet value(s) (shape (m,)) on the outer boundary.
    Returns per leaf the boundary values u_b (n_b x m) and interior values
    u_i (n_i x m) = S u_b + W.
    """
    vals = dict(g_keys)
    for lev in reversed(levels):
        for rec in lev.values():
            u12 = np.array([vals[k] for k in rec["k12"]])
            u3 = rec["S3"] @ u12 + rec["w3"]
            for k, v in zip(rec["k3"], u3):
                vals[k] = v
    out = []
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            ub = np.array([vals[k] for k in box_keys(p, ix, iy, 1, 1)])
            ui = lf["S"] @ ub + lf["W"]
            out.append({"u_b": ub, "u_i": ui})
    return out


def outer_boundary_keys(p, nx, ny):
    return box_keys(p, 0, 0, nx, ny)


def key_coords(p, key, nx, ny, lx=1.0, ly=1.0, x0=0.0, y0=0.0):
    """Physical coordinate of an edge node named by its key."""
    kind, line, seg, k = key
    t = cheb_points(p)[1:-1]
    hx, hy = lx / nx, ly / ny
    if kind == "v":
        return x0 + line * hx, y0 + seg * hy + (1.0 + t[k]) * hy / 2.0
    return x0 + seg * hx + (1.0 + t[k]) * hx / 2.0, y0 + line * hy


# ----------------------------------------------------------------------------
# Impedance-to-impedance (ItI) leaf maps and merges.  Not in the paper (its
# leaf maps are DtN maps, which do not exist when kappa^2 is an eigenvalue of
# the leaf's Dirichlet problem); the impedance formulation of Gillman,
# Barnett and Martinsson (BIT 2015), restated here from its definitions:
# incoming data f = u_n + i eta u, outgoing data g = u_n - i eta u on a box
# boundary (u_n the outward normal derivative, eta > 0), and the leaf
# problem with the impedance condition is solvable at every real kappa.
# ----------------------------------------------------------------------------


def iti_leaf(p, box, coef, kappa, eta, f=None):
    """ItI map of one leaf.  Unknowns: u at the interior and edge nodes
    (corners are not unknowns, as for the DtN maps); rows: the PDE at the
    interior nodes (corner columns folded in by interior_edge_block) and,
    at every edge node a, the impedance condition (N u)_a + i eta u_a =
    f_a.  With Y the solution for unit incoming data (one column per edge
    node) and uf the solution for the body load with zero incoming data:
        g = f - 2 i eta u_b   =>   R = I - 2 i eta Y_b,  h = -2 i eta uf_b.
    Returns R (n_b x n_b), h (n_b x m), Y and uf over [interior; edge]
    nodes (complex)."""
    A, Nrow, _, _ = leaf_operator(p, box, coef, kappa)
    ix = leaf_index_sets(p)
    I, B = ix["I"], ix["B"]
    ni, nb = len(I), len(B)
    M = np.zeros((ni + nb, ni + nb), dtype=complex)
    M[:ni, :ni] = A[np.ix_(I, I)]
    M[:ni, ni:] = interior_edge_block(A, p)
    M[ni:, :ni] = Nrow[:, I]
    M[ni:, ni:] = Nrow[:, B] + 1j * eta * np.eye(nb)
    m = 0 if f is None else np.asarray(f).reshape(p * p, -1).shape[1]
    rhs = np.zeros((ni + nb, nb + m), dtype=complex)
    rhs[ni:, :nb] = np.eye(nb)
    if m:
        rhs[:ni, nb:] = np.asarray(f, dtype=float).reshape(p * p, -1)[I]
    sol = np.linalg.solve(M, rhs)
    Y, uf = sol[:, :nb], sol[:, nb:]
    return {"R": np.eye(nb) - 2j * eta * Y[ni:], "h": -2j * eta * uf[ni:], "Y": Y, "uf": uf, "M": M}


def iti_merge_two(ka, Ra, ha, kb, Rb, hb, kpar):
    """Merge the ItI maps of sibling boxes alpha, beta along their shared
    edge 3.  On it the outward normals are opposite and u is continuous, so
    the incoming data of one box is minus the outgoing data of the other:
    f_a3 = -g_b3, f_b3 = -g_a3.  With t = g_a3:
        (I - Ra33 Rb33) t = Ra31 f1 - Ra33 Rb32 f2 + ha3 - Ra33 hb3,
        f_a3 = -Rb32 f2 + Rb33 t - hb3,   f_b3 = -t,
        g1 = Ra11 f1 + Ra13 f_a3 + ha1,   g2 = Rb22 f2 + Rb23 f_b3 + hb2.
    Returns the parent's R, h in kpar order and the maps from the parent's
    incoming data [f1; f2] (order k12) to the children's incoming data on
    edge 3 (Fa3, fa3, Fb3, fb3) for the downward pass."""
    pa = {k: i for i, k in enumerate(ka)}
    pb = {k: i for i, k in enumerate(kb)}
    k3 = [k for k in ka if k in pb]
    k1 = [k for k in ka if k not in pb]
    k2 = [k for k in kb if k not in pa]
    a1, a3 = [pa[k] for k in k1], [pa[k] for k in k3]
    b2, b3 = [pb[k] for k in k2], [pb[k] for k in k3]
    ix = np.ix_
    n1, n2, n3 = len(k1), len(k2), len(k3)
    Ra33, Rb33 = Ra[ix(a3, a3)], Rb[ix(b3, b3)]
    K = np.eye(n3) - Ra33 @ Rb33
    rhs = np.hstack([Ra[ix(a3, a1)], -Ra33 @ Rb[ix(b3, b2)], (ha[a3] - Ra33 @ hb[b3])])
    X = np.linalg.solve(K, rhs)
    T1, th = X[:, :n1 + n2], X[:, n1 + n2:]
    Fa3 = np.hstack([np.zeros((n3, n1)), -Rb[ix(b3, b2)]]) + Rb33 @ T1
    fa3 = Rb33 @ th - hb[b3]
    Fb3, fb3 = -T1, -th
    Rp = np.zeros((n1 + n2, n1 + n2), dtype=complex)
    Rp[:n1, :n1] = Ra[ix(a1, a1)]
    Rp[n1:, n1:] = Rb[ix(b2, b2)]
    Rp[:n1] += Ra[ix(a1, a3)] @ Fa3
    Rp[n1:] += Rb[ix(b2, b3)] @ Fb3
    hp = np.vstack([ha[a1] + Ra[ix(a1, a3)] @ fa3, hb[b2] + Rb[ix(b2, b3)] @ fb3])
    k12 = k1 + k2
    pos = {k: i for i, k in enumerate(k12)}
    perm = [pos[k] for k in kpar]
    return {"R": Rp[ix(perm, perm)], "h": hp[perm], "k12": k12, "k3": k3,
            "Fa3": Fa3, "fa3": fa3, "Fb3": Fb3, "fb3": fb3}


def iti_solve(p, nx, ny, leaves, g_keys, eta):
    """Merge the leaves' ItI maps over the grid (the schedule of hps_upward),
    impose the Dirichlet data at the root (f - g = 2 i eta u there, so
    (I - R) f = h + 2 i eta u_D), pass the incoming data down, and recover
    every leaf's values u = Y f + uf.  leaves[ix * ny + iy] holds an
    iti_leaf record.  Returns per leaf (u_b, u_i) as hps_downward does
    (complex; real for real data)."""
    boxes = {}
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            boxes[(ix, iy)] = {"R": lf["R"], "h": lf["h"], "keys": box_keys(p, ix, iy, 1, 1)}
    wx, wy = 1, 1
    levels = []
    for d in merge_schedule(nx, ny):
        new = {}
        for (ix0, iy0) in sorted(boxes):
            if d == "x" and (ix0 // wx) % 2 == 0:
                other = (ix0 + wx, iy0)
                kpar = box_keys(p, ix0, iy0, 2 * wx, wy)
            elif d == "y" and (iy0 // wy) % 2 == 0:
                other = (ix0, iy0 + wy)
                kpar = box_keys(p, ix0, iy0, wx, 2 * wy)
            else:
                continue
            a, b = boxes[(ix0, iy0)], boxes[other]
            rec = iti_merge_two(a["keys"], a["R"], a["h"], b["keys"], b["R"], b["h"], kpar)
            rec["keys"] = kpar
            rec["children"] = ((ix0, iy0), other)
            new[(ix0, iy0)] = rec
        wx, wy = (wx * 2, wy) if d == "x" else (wx, wy * 2)
        boxes = new
        levels.append(new)
    root = boxes[(0, 0)]
    keys = root["keys"]
    uD = np.array([np.atleast_1d(g_keys[k]) for k in keys], dtype=complex)
    f_root = np.linalg.solve(np.eye(len(keys)) - root["R"], root["h"] + 2j * eta * uD)
    # incoming data per box, key -> value, from the root down: a child keeps
    # the parent's data on its exterior edges and takes its own value on the
    # shared edge (the two children see different incoming data there)
    cur = {(0, 0): dict(zip(keys, f_root))}
    for lev in reversed(levels):
        nxt = {}
        for o, rec in lev.items():
            pf = cur[o]
            f12 = np.array([pf[k] for k in rec["k12"]])
            ca, cb = rec["children"]
            fa = {k: v for k, v in pf.items()}
            fb = dict(fa)
            fa.update(zip(rec["k3"], rec["Fa3"] @ f12 + rec["fa3"]))
            fb.update(zip(rec["k3"], rec["Fb3"] @ f12 + rec["fb3"]))
            nxt[ca], nxt[cb] = fa, fb
        cur = nxt
    ni = len(leaf_index_sets(p)["I"])
    out = []
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            fl = np.array([cur[(ix, iy)][k] for k in box_keys(p, ix, iy, 1, 1)])
            u = lf["Y"] @ fl + lf["uf"]
            out.append({"u_b": u[ni:], "u_i": u[:ni], "f_in": fl})
    return out


# ----------------------------------------------------------------------------
# SlabLU: the reduced system of Eq. (hps_reduced) in the slab block form of
# Eq. (dell1); slab interiors eliminated, the block-tridiagonal interface
# system factored densely (Section 2, the SlabLU paragraphs)
# ----------------------------------------------------------------------------


def reduced_system(p, nx, ny, leaves, g_keys):
    """The reduced system A~ u~ = f~ of Eq. (hps_reduced): the unknowns are
    the leaf edge nodes not on the outer boundary; each has one row, the
    flux continuity there (the outward fluxes T u_b + h of the two leaves
    sharing the node sum to zero).  Outer edge nodes carry the Dirichlet
    data g_keys and move to the right-hand side.  leaves[ix * ny + iy] holds
    the leaf's T and h.  Returns (A, f, keys): keys[i] names unknown i."""
    outer = set(outer_boundary_keys(p, nx, ny))
    keys, kid = [], {}
    for ix in range(nx):
        for iy in range(ny):
            for k in box_keys(p, ix, iy, 1, 1):
                if k not in outer and k not in kid:
                    kid[k] = len(keys)
                    keys.append(k)
    m = np.asarray(leaves[0]["h"]).reshape(4 * (p - 2), -1).shape[1]
    n = len(keys)
    A = np.zeros((n, n))
    f = np.zeros((n, m))
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            T = lf["T"]
            h = np.asarray(lf["h"]).reshape(T.shape[0], m)
            lk = box_keys(p, ix, iy, 1, 1)
            for r, k in enumerate(lk):
                if k in outer:
                    continue
                row = kid[k]
                f[row] -= h[r]
                for c, kc in enumerate(lk):
                    if kc in outer:
                        f[row] -= T[r, c] * np.atleast_1d(g_keys[kc])
                    else:
                        A[row, kid[kc]] += T[r, c]
    return A, f, keys


def slab_blocks(p, nx, s, keys):
    """Eq. (dell1)'s blocks for slabs of s leaf columns (vertical strips,
    x from 0): interface k = 1..S-1 is the vertical grid line x = k s hx,
    every other unknown is interior to the slab that contains it (a vertical
    line x = l hx inside slab l // s, or a horizontal edge of leaf column ix
    in slab ix // s).  Returns (interior index lists I[0..S-1], interface
    index lists G[1..S-1] as G[0..S-2])."""
    if nx % s or s < 2:
        raise ValueError("slab width must divide nx and be at least 2 leaves")
    S = nx // s
    I = [[] for _ in range(S)]
    G = [[] for _ in range(S - 1)]
    for i, (kind, line, seg, _) in enumerate(keys):
        if kind == "v" and line % s == 0:
            G[line // s - 1].append(i)
        elif kind == "v":
            I[line // s].append(i)
        else:
            I[seg // s].append(i)
    return I, G


def slab_solve(p, nx, ny, s, leaves, g_keys):
    """SlabLU on the reduced system (Section 2, Eq. (dell1)): order the
    unknowns as slab interiors and the interfaces between slabs; eliminate
    each slab's interior (dense solves with its diagonal block); the
    Schur complement on the interfaces is block tridiagonal, and is solved
    by block LU (forward elimination over the interfaces, then back
    substitution); the slab interiors follow from the interface values.
    Returns the values of all unknowns by key."""
    A, f, keys = reduced_system(p, nx, ny, leaves, g_keys)
    I, G = slab_blocks(p, nx, s, keys)
    S = len(I)
    ix = np.ix_
    # slab interiors: A_II^{-1} applied to [A_I,Gleft  A_I,Gright  f_I]
    elim = []
    for j in range(S):
        left = G[j - 1] if j > 0 else []
        right = G[j] if j < S - 1 else []
        Aii = A[ix(I[j], I[j])]
        X = np.linalg.solve(Aii, np.hstack([A[ix(I[j], left)], A[ix(I[j], right)], f[I[j]]]))
        elim.append((left, right, X))
    # block tridiagonal interface system: D_k u_k + L_k u_{k-1} + U_k u_{k+1} = r_k
    D, L, U, r = [], [], [], []
    for k in range(S - 1):
        g = G[k]
        Dk = A[ix(g, g)].copy()
        rk = f[g].copy()
        Lk = Uk = None
        for j in (k, k + 1):            # the slabs left and right of interface k
            left, right, X = elim[j]
            AgI = A[ix(g, I[j])]
            nl, nr = len(left), len(right)
            XL, XR, Xf = X[:, :nl], X[:, nl:nl + nr], X[:, nl + nr:]
            rk -= AgI @ Xf
            if j == k:                  # slab k: interface k is its right side
                Dk -= AgI @ XR
                if nl:
                    Lk = A[ix(g, left)] - AgI @ XL
            else:                       # slab k + 1: interface k is its left side
                Dk -= AgI @ XL
                if nr:
                    Uk = A[ix(g, right)] - AgI @ XR
        D.append(Dk)
        L.append(Lk)
        U.append(Uk)
        r.append(rk)
    # block LU: Delta_k = D_k - L_k Delta_{k-1}^{-1} U_{k-1}, then back substitution
    Delta, y = [], []
    for k in range(S - 1):
        if k == 0:
            Delta.append(D[0])
            y.append(r[0])
        else:
            Z = np.linalg.solve(Delta[k - 1], np.hstack([U[k - 1], y[k - 1]]))
            nu = U[k - 1].shape[1]
            Delta.append(D[k] - L[k] @ Z[:, :nu])
            y.append(r[k] - L[k] @ Z[:, nu:])
    u = [None] * (S - 1)
    for k in reversed(range(S - 1)):
        rhs = y[k] if k == S - 2 else y[k] - U[k] @ u[k + 1]
        u[k] = np.linalg.solve(Delta[k], rhs)
    vals = {}
    for k in range(S - 1):
        for i, v in zip(G[k], u[k]):
            vals[keys[i]] = v
    for j in range(S):
        left, right, X = elim[j]
        sides = ([u[j - 1]] if j > 0 else []) + ([u[j]] if j < S - 1 else [])
        ub = np.vstack([np.zeros((0, f.shape[1]))] + sides)
        nl, nr = len(left), len(right)
        ui = X[:, nl + nr:] - X[:, :nl + nr] @ ub
        for i, v in zip(I[j], ui):
            vals[keys[i]] = v
    return vals


def slab_downward(p, nx, ny, s, leaves, g_keys):
    """slab_solve, then every leaf's edge values from the reduced solution
    and the Dirichlet data, and its interior values u_i = S u_b + W: per
    leaf (u_b, u_i) in the form hps_downward returns."""
    vals = dict(g_keys)
    vals.update(slab_solve(p, nx, ny, s, leaves, g_keys))
    out = []
    for ix in range(nx):
        for iy in range(ny):
            lf = leaves[ix * ny + iy]
            ub = np.array([np.atleast_1d(vals[k]) for k in box_keys(p, ix, iy, 1, 1)])
            out.append({"u_b": ub, "u_i": lf["S"] @ ub + lf["W"]})
    return out


# ----------------------------------------------------------------------------
# Brute-force global collocation system (Eq. (Au=f)), independent of merges
# ----------------------------------------------------------------------------


def global_system(p, nx, ny, coefs, kappa, f, g_fn, lx=1.0, ly=1.0):
    """Assemble the global collocation system on an nx x ny leaf grid.

    Unknowns: every leaf-interior node, then every edge node not on the outer
    boundary.  Rows: the PDE at every leaf-interior node; flux continuity
    (sum of the two leaves' outward normal derivatives = 0) at every
    interface edge node.  Outer edge nodes carry Dirichlet data g and are
    moved to the right-hand side.  coefs[l] is (6, p*p), f[l] is (p*p, m).
    Returns (A, rhs, layout) with layout describing the unknown ordering.
    """
    boxes = grid_boxes(nx, ny, lx=lx, ly=ly)
    ix_sets = leaf_index_sets(p)
    I, B = ix_sets["I"], ix_sets["B"]
    n_i, n_b = len(I), len(B)
    nl = nx * ny
    m = np.asarray(f[0]).reshape(p * p, -1).shape[1]
    # edge keys
    outer = set(outer_boundary_keys(p, nx, ny))
    iface = []
    seen = set()
    for ix in range(nx):
        for iy in range(ny):
            for k in box_keys(p, ix, iy, 1, 1):
                if k not in outer and k not in seen:
                    seen.add(k)
                    iface.append(k)
    kid = {k: nl * n_i + i for i, k in enumerate(iface)}
    n = nl * n_i + len(iface)
    A = np.zeros((n, n))
    rhs = np.zeros((n, m))
    gvals = {}
    for k in outer:
        gvals[k] = np.atleast_1d(g_fn(*key_coords(p, k, nx, ny, lx, ly)))
    corners = [0, p - 1, (p - 1) * p, p * p - 1]
    for l, box in enumerate(boxes):
        ix, iy = divmod(l, ny)
        Al, Nrow, _, _ = leaf_operator(p, box, coefs[l], kappa)
        keys = box_keys(p, ix, iy, 1, 1)
        # local node -> ('u', col) or ('g', key)
        colmap = {}
        for q, node in enumerate(I):
            colmap[node] = ("u", l * n_i + q)
        for q, node in enumerate(B):
            k = keys[q]
            colmap[node] = ("g", k) if k in outer else ("u", kid[k])
        fl = np.asarray(f[l]).reshape(p * p, m)

        def put(row, coeffs, target_rhs_sign=1.0):
            for node in range(p * p):
                a = coeffs[node]
                if a == 0.0:
                    continue
                if node in corners:
                    raise NotImplementedError("operator row touches a leaf corner (c12 != 0)")
                kind, c = colmap[node]
                if kind == "u":
                    A[row, c] += a
                else:
                    rhs[row] -= a * gvals[c]

        for q, node in enumerate(I):
            row = l * n_i + q
            put(row, Al[node])
            rhs[row] += fl[node]
        for q in range(n_b):
            k = keys[q]
            if k in outer:
                continue
            put(kid[k], Nrow[q])
    layout = {"n_i": n_i, "iface": iface, "kid": kid, "gvals": gvals}
    return A, rhs, layout


def global_dense_solve(p, nx, ny, coefs, kappa, f, g_fn, lx=1.0, ly=1.0):
    """Solve the global system with numpy.linalg.solve; returns per-leaf
    (u_b, u_i) in the same form as hps_downward, plus relerr_res of
    Eq. (accuracy_formula) for the computed solution."""
    A, rhs, lay = global_system(p, nx, ny, coefs, kappa, f, g_fn, lx, ly)
    u = np.linalg.solve(A, rhs)
    res = np.linalg.norm(A @ u - rhs) / np.linalg.norm(rhs)
    n_i = lay["n_i"]
    out = []
    for ix in range(nx):
        for iy in range(ny):
            l = ix * ny + iy
            ub = []
            for k in box_keys(p, ix, iy, 1, 1):
                ub.append(lay["gvals"][k] if k in lay["gvals"] else u[lay["kid"][k]])
            out.append({"u_b": np.array(ub), "u_i": u[l * n_i:(l + 1) * n_i]})
    return out, res


# ----------------------------------------------------------------------------
# Error metrics (Eq. (accuracy_formula))
# ----------------------------------------------------------------------------


def relerr(calc, ref):
    """||calc - ref||_2 / ||ref||_2 (Frobenius for matrices)."""
    calc = np.asarray(calc, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(calc - ref) / np.linalg.norm(ref))
