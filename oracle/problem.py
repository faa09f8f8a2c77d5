"""Data of the time-harmonic acoustics problem, Eq. helmholtz (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

With the wavespeed reading rho = 1, bulk modulus c^2 the strong form is

    i w c^-2 p + div u = f,   i w u + grad p = g   in Omega,
    Z^-1 p - u.n = u0                               on Gamma,  Z = c.

The paper's own equations are the case c = 1, f = g = 0.  Three loads are
provided:

* ``GaussianSource``  f(x) = A exp(-|x - x0|^2 / (2 sigma^2)), g = 0, u0 = 0
  (the point-like source of Sec. 5, width read as a standard deviation);
* ``PlaneWave``       p = exp(-i w d.x / c), u = d p / c: f = g = 0 and
  u0 = (1 - d.n) p / c (an exact solution for constant c);
* ``Manufactured``    given polynomials p_ex, u_ex of degree < m on the box,
  f, g and u0 are whatever makes (p_ex, u_ex) exact; with m <= p they lie
  in the discrete trial space, so DPG must reproduce them to rounding.

``WithImpedanceLoad(base, u0)`` adds a caller's impedance data u0(X, n, c)
on Gamma to the f, g and u0 of another load (the boundary condition of
Eq. helmholtz with general data).

Polynomials of ``Manufactured`` are tensor Legendre series in the box
coordinate X = (x - x0) / (x1 - x0): coefficient array C[comp, c, b, a]
(comp 0 = p, 1..3 = u_x, u_y, u_z; complex).
"""
import numpy as np

from .basis import leg


class GaussianSource:
    def __init__(self, center, width, amp=1.0):
        self.center = np.asarray(center, dtype=np.float64)
        self.width = float(width)
        self.amp = float(amp)
        self.g = None
        self.u0 = None

    def f(self, X, c):
        r2 = np.sum((X - self.center) ** 2, axis=1)
        return (self.amp * np.exp(-r2 / (2.0 * self.width ** 2))).astype(np.complex128)


class PlaneWave:
    def __init__(self, direction, omega, c=1.0):
        d = np.asarray(direction, dtype=np.float64)
        self.d = d / np.linalg.norm(d)
        self.omega = float(omega)
        self.c = float(c)
        self.f = None
        self.g = None

    def p(self, X):
        return np.exp(-1j * self.omega * (X @ self.d) / self.c)

    def u(self, X):
        return self.p(X)[:, None] * self.d[None, :] / self.c

    def u0(self, X, n, c):
        return (1.0 - self.d @ n) * self.p(X) / c


class Manufactured:
    def __init__(self, coeffs, omega, x0=(0, 0, 0), x1=(1, 1, 1)):
        self.C = np.asarray(coeffs, dtype=np.complex128)   # (4, m, m, m)
        self.m = self.C.shape[1]
        self.omega = float(omega)
        self.x0 = np.asarray(x0, dtype=np.float64)
        self.L = np.asarray(x1, dtype=np.float64) - self.x0

    def _eval(self, comp, X):
        """Value and gradient of component comp at physical points X."""
        Xh = (X - self.x0) / self.L
        vals, ders = [], []
        for d in range(3):
            V, D = leg(self.m - 1, Xh[:, d])
            vals.append(V)
            ders.append(D / self.L[d])
        C = self.C[comp]
        val = np.einsum("cba,an,bn,cn->n", C, vals[0], vals[1], vals[2])
        gx = np.einsum("cba,an,bn,cn->n", C, ders[0], vals[1], vals[2])
        gy = np.einsum("cba,an,bn,cn->n", C, vals[0], ders[1], vals[2])
        gz = np.einsum("cba,an,bn,cn->n", C, vals[0], vals[1], ders[2])
        return val, np.stack([gx, gy, gz], axis=1)

    def p(self, X):
        return self._eval(0, X)[0]

    def u(self, X):
        return np.stack([self._eval(1 + d, X)[0] for d in range(3)], axis=1)

    def f(self, X, c):
        pv, _ = self._eval(0, X)
        div = sum(self._eval(1 + d, X)[1][:, d] for d in range(3))
        return 1j * self.omega / c ** 2 * pv + div

    def g(self, X, c):
        _, gp = self._eval(0, X)
        u = self.u(X)
        return 1j * self.omega * u + gp

    def u0(self, X, n, c):
        return self.p(X) / c - self.u(X) @ n


class WithImpedanceLoad:
    """f and g of ``base``; u0 = base's u0 (if any) + extra(X, n, c)."""

    def __init__(self, base, extra):
        self.base = base
        self.extra = extra
        self.f = base.f
        self.g = base.g

    def u0(self, X, n, c):
        v = np.asarray(self.extra(X, n, c), dtype=np.complex128)
        if self.base.u0 is not None:
            v = v + self.base.u0(X, n, c)
        return v
