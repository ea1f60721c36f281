"""Seeded synthetic workloads for the HPS leaf-condensation library.

This module defines problems, not the method: leaf tilings, wavenumbers,
coefficient fields, body loads and Dirichlet data as plain functions of the
reference coordinates (x, y), plus the seeded random draws (bump centres and
amplitudes, per-leaf orders).  It holds none of the discretization's
arithmetic: callers evaluate these functions at whatever node coordinates
their own discretization produces.  Both the GPU library's callers and the
CPU oracle's tests take their inputs from here, and it imports neither.

Workloads (synthetic stand-ins for the paper's experiments, Section 3):

* ``planewave``   unit square, kappa = 20, b = 1, p = 10, 8 x 8 leaves,
                  f = 0, Dirichlet data from u = sin(kappa (0.6 x + 0.8 y)).
* ``bumps_p20``   unit square, kappa = 200, b = 1 - 0.5 exp(-|x-c|^2/0.02),
                  c = (0.5, 0.5), p = 20, 64 x 64 leaves, m = 1 body load of
                  16 seeded Gaussian bumps (sigma = 0.05), seed 2.
* ``bumps_p30``   as bumps_p20 at p = 30 on 32 x 32 leaves, seed 3.
* ``annulus_p24`` the annular sector r in [1, 2], theta in [0, pi/2] mapped
                  to the unit square by r = 1 + x, theta = (pi/2) y; 64 leaves
                  in x (r) and 128 in y (theta); kappa = 400,
                  b = 1 - 0.3 sin(4 r) cos(6 theta), p = 24, m = 1, seed 4.
* ``psi_p20``     the paper's curved domain Psi = {(x1, x2 / psi(x1))},
                  psi(z) = 1 - sin(z)/4, over the unit square (mixed term
                  c12 != 0), b = 1, kappa = 200, p = 20, 64 x 64 leaves,
                  m = 1 body load of bumps (seed 6), Dirichlet data of the
                  physical plane wave sin(kappa (0.6 y1 + 0.8 y2)).
* ``uneven``      128 x 80 leaves of the unit square, p drawn per leaf from
                  {12, 16, 20, 24, 32} with weights {.3, .25, .2, .15, .1},
                  kappa = 300, b as bumps_p20, m = 64 body loads, seed 5.
"""

from dataclasses import dataclass, field
import math

import numpy as np

SIGMA = 0.05
N_BUMPS = 16


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    kappa: float
    p: np.ndarray            # per-leaf order, leaf index ix * ny + iy
    m: int                   # body-load right-hand sides
    seed: int
    geometry: str = "square"  # or "annulus"
    bcoef: str = "one"        # b field: "one", "gauss", "annulus"
    load: str = "bumps"       # "bumps" or "zero"
    dirichlet: str = "none"   # "planewave" or "none"
    centres: np.ndarray = field(default=None, repr=False)   # (m, 16, 2)
    amps: np.ndarray = field(default=None, repr=False)      # (m, 16)

    @property
    def n_leaves(self):
        return self.nx * self.ny

    def boxes(self):
        """(n_leaves, 4) array of x0, y0, hx, hy on the reference square."""
        hx, hy = 1.0 / self.nx, 1.0 / self.ny
        ix, iy = np.meshgrid(np.arange(self.nx), np.arange(self.ny), indexing="ij")
        out = np.empty((self.nx * self.ny, 4))
        out[:, 0] = ix.ravel() * hx
        out[:, 1] = iy.ravel() * hy
        out[:, 2] = hx
        out[:, 3] = hy
        return out

    # -- fields, as functions of reference coordinates -----------------------
    def coefficients(self, x, y, xp=np):
        """(6, ...) stack of c11, c12, c22, c1, c2, b at (x, y)."""
        one = xp.ones_like(x)
        zero = xp.zeros_like(x)
        if self.geometry == "psi":
            # the curved domain {(x1, x2 / psi(x1))}, psi(z) = 1 - sin(z)/4,
            # over the reference square (Eq. (parametrization), Eq. (chain_rule))
            ps = 1.0 - 0.25 * xp.sin(x)
            dps = -0.25 * xp.cos(x)
            ddps = 0.25 * xp.sin(x)
            g = y * dps / ps
            c11, c12, c22 = one, g, g * g + ps * ps
            c1, c2 = zero, y * ddps / ps
            b = one
        elif self.geometry == "annulus":
            r = 1.0 + x
            th = (math.pi / 2.0) * y
            c11, c12 = one, zero
            c22 = (4.0 / math.pi ** 2) / (r * r)
            c1, c2 = 1.0 / r, zero
            b = 1.0 - 0.3 * xp.sin(4.0 * r) * xp.cos(6.0 * th)
        else:
            c11, c12, c22, c1, c2 = one, zero, one, zero, zero
            if self.bcoef == "gauss":
                b = 1.0 - 0.5 * xp.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.02)
            else:
                b = one
        return xp.stack([c11, c12, c22, c1, c2, b])

    def body_load(self, x, y, xp=np):
        """(..., m) body loads at (x, y): sums of 16 Gaussian bumps
        a_k exp(-|x - c_k|^2 / (2 sigma^2)) per right-hand side."""
        if self.load == "zero" or self.m == 0:
            return xp.zeros(tuple(x.shape) + (max(self.m, 1),), dtype=x.dtype)
        cols = []
        for r in range(self.m):
            acc = xp.zeros_like(x)
            for k in range(N_BUMPS):
                cx, cy = float(self.centres[r, k, 0]), float(self.centres[r, k, 1])
                d2 = (x - cx) ** 2 + (y - cy) ** 2
                acc = acc + float(self.amps[r, k]) * xp.exp(-d2 / (2.0 * SIGMA ** 2))
            cols.append(acc)
        return xp.stack(cols, axis=-1)

    def dirichlet_data(self, x, y, xp=np):
        if self.dirichlet == "planewave":
            return xp.sin(self.kappa * (0.6 * x + 0.8 * y))
        if self.dirichlet == "psi_planewave":
            # the plane wave sin(kappa (0.6 y1 + 0.8 y2)) of the physical
            # domain at (y1, y2) = (x1, x2 / psi(x1))
            return xp.sin(self.kappa * (0.6 * x + 0.8 * y / (1.0 - 0.25 * xp.sin(x))))
        return xp.zeros_like(x)


def _bumps(seed, m):
    rng = np.random.default_rng(seed)
    centres = np.empty((m, N_BUMPS, 2))
    amps = np.empty((m, N_BUMPS))
    for r in range(m):
        centres[r] = rng.uniform(0.0, 1.0, size=(N_BUMPS, 2))
        amps[r] = rng.standard_normal(N_BUMPS)
    return centres, amps


def planewave(p=10, nx=8, ny=8, kappa=20.0):
    return Workload("planewave", nx, ny, kappa, np.full(nx * ny, p, dtype=np.int32), 1, 1,
                    bcoef="one", load="zero", dirichlet="planewave")


def bumps(p=20, nx=64, ny=64, kappa=200.0, seed=2, m=1, name=None):
    c, a = _bumps(seed, m)
    return Workload(name or f"bumps_p{p}", nx, ny, kappa, np.full(nx * ny, p, dtype=np.int32),
                    m, seed, bcoef="gauss", centres=c, amps=a)


def bumps_p20():
    return bumps(20, 64, 64, 200.0, seed=2, name="bumps_p20")


def bumps_p30():
    return bumps(30, 32, 32, 200.0, seed=3, name="bumps_p30")


def annulus(p=24, nx=64, ny=128, kappa=400.0, seed=4, m=1, name=None):
    c, a = _bumps(seed, m)
    return Workload(name or f"annulus_p{p}", nx, ny, kappa, np.full(nx * ny, p, dtype=np.int32),
                    m, seed, geometry="annulus", bcoef="annulus", centres=c, amps=a)


def annulus_p24():
    return annulus()


def psi_curved(p=20, nx=64, ny=64, kappa=200.0, seed=6, m=1, name=None):
    """The paper's curved domain Psi (b = 1) on the reference square: the
    mixed-derivative coefficient c12 is nonzero; bump loads and the physical
    plane wave as Dirichlet data."""
    c, a = _bumps(seed, m)
    return Workload(name or f"psi_p{p}", nx, ny, kappa, np.full(nx * ny, p, dtype=np.int32), m, seed,
                    geometry="psi", bcoef="one", dirichlet="psi_planewave", centres=c, amps=a)


def psi_p20():
    return psi_curved()


P_SET = (12, 16, 20, 24, 32)
P_WEIGHTS = (0.3, 0.25, 0.2, 0.15, 0.1)


def uneven(nx=128, ny=80, kappa=300.0, seed=5, m=64, name="uneven"):
    rng = np.random.default_rng(seed)
    p = rng.choice(np.array(P_SET), size=nx * ny, p=np.array(P_WEIGHTS)).astype(np.int32)
    c, a = _bumps(seed + 1000, m)
    return Workload(name, nx, ny, kappa, p, m, seed, bcoef="gauss", centres=c, amps=a)


def scaled(w, nx, ny):
    """The same problem on a smaller leaf grid (for tests), keeping p's draw."""
    out = Workload(w.name + f"_{nx}x{ny}", nx, ny, w.kappa, w.p[: nx * ny].copy(), w.m, w.seed,
                   w.geometry, w.bcoef, w.load, w.dirichlet, w.centres, w.amps)
    return out
