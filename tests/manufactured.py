"""Manufactured tensor-polynomial solutions for pinning the HPS discretization.

A polynomial of degree <= p-1 in each variable is reproduced exactly by the
p-point Chebyshev collocation of Section 2, so its nodal values solve the
discrete leaf and global systems up to rounding, for any wavenumber and any
coefficient samples.  Derivatives here are taken analytically with
numpy.polynomial, independently of any differentiation matrix.
"""

import numpy as np
from numpy.polynomial import polynomial as P


class TensorPoly:
    """u(x, y) = sum_ab C[a, b] xi^a eta^b, xi = (x - xc)/sx, eta = (y - yc)/sy."""

    def __init__(self, C, xc=0.0, yc=0.0, sx=1.0, sy=1.0):
        self.C = np.asarray(C, dtype=np.float64)
        self.xc, self.yc, self.sx, self.sy = xc, yc, sx, sy

    def _d(self, dx, dy):
        c = self.C
        if dx:
            c = P.polyder(c, m=dx, scl=1.0 / self.sx, axis=0)
        if dy:
            c = P.polyder(c, m=dy, scl=1.0 / self.sy, axis=1)
        return c

    def __call__(self, x, y, dx=0, dy=0):
        c = self._d(dx, dy)
        return P.polyval2d((x - self.xc) / self.sx, (y - self.yc) / self.sy, c)

    def apply_operator(self, x, y, coef, kappa):
        """-(c11 u_xx + 2 c12 u_xy + c22 u_yy + c1 u_x + c2 u_y) - kappa^2 b u."""
        c11, c12, c22, c1, c2, b = coef
        return -(c11 * self(x, y, 2, 0) + 2.0 * c12 * self(x, y, 1, 1) + c22 * self(x, y, 0, 2)
                 + c1 * self(x, y, 1, 0) + c2 * self(x, y, 0, 1)) - kappa ** 2 * b * self(x, y)


def random_poly(rng, deg_x, deg_y, **kw):
    return TensorPoly(rng.standard_normal((deg_x + 1, deg_y + 1)), **kw)


def random_coef(rng, n, c12=False):
    """Random coefficient samples at n nodes, each field distinct so that a
    swapped or dropped term is visible.  c11, c22 kept positive."""
    c11 = 1.0 + 0.5 * rng.random(n)
    c22 = 0.5 + 0.5 * rng.random(n)
    c12v = (0.3 * rng.standard_normal(n)) if c12 else np.zeros(n)
    c1 = 2.0 * rng.standard_normal(n)
    c2 = 2.0 * rng.standard_normal(n)
    b = 0.2 + rng.random(n)
    return np.stack([c11, c12v, c22, c1, c2, b])
