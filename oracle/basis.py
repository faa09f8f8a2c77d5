"""1D building blocks of the exact-sequence hexahedral spaces (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2 of the paper discretises the trial fields in L^2, the traces as
traces of H^1 / H(div) conforming elements and tests with the broken spaces
H^1(Omega_h) x H(div, Omega_h) enriched by one polynomial order (Sec. 2,
first paragraph).  On an axis-aligned hexahedron every one of these spaces is
a tensor product of two 1D families on the unit interval [0, 1]:

* ``leg(a, x)``  Legendre polynomial of degree a in xi = 2x - 1 (the L^2 /
  H(div)-normal-trace family),
* ``h1(k, x)``   hierarchical H^1 family of order p: the two vertex (hat)
  functions 1 - x and x, and for k >= 2 the integrated-Legendre bubbles
  (P_k(xi) - P_{k-2}(xi)) / sqrt(2 (2k - 1)).

Parity: pinned by ``tests/test_oracle_basis.py`` (Legendre orthogonality and
endpoint values, bubble endpoint zeros, derivative identity of the integrated
Legendre family, Gauss-rule exactness on monomials).
"""
import numpy as np


def gauss01(n):
    """Gauss-Legendre rule with n points mapped to [0, 1] (library primitive)."""
    xi, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (xi + 1.0), 0.5 * w


def legendre_xi(nmax, xi):
    """P_0..P_nmax at xi in [-1, 1] by the three-term (Bonnet) recurrence.

    Returns (P, dP/dxi), each of shape (nmax + 1, len(xi)).
    """
    xi = np.asarray(xi, dtype=np.float64)
    P = np.zeros((nmax + 1,) + xi.shape)
    dP = np.zeros_like(P)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = xi
        dP[1] = 1.0
    for k in range(1, nmax):
        # (k+1) P_{k+1} = (2k+1) xi P_k - k P_{k-1}
        P[k + 1] = ((2 * k + 1) * xi * P[k] - k * P[k - 1]) / (k + 1)
        # P'_{k+1} = P'_{k-1} + (2k+1) P_k
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k]
    return P, dP


def leg(nmax, x):
    """Legendre family on [0, 1]: L_a(x) = P_a(2x - 1), a = 0..nmax.

    Returns (values, d/dx) with shape (nmax + 1, len(x)).
    """
    x = np.asarray(x, dtype=np.float64)
    P, dP = legendre_xi(nmax, 2.0 * x - 1.0)
    return P, 2.0 * dP


def h1(p, x):
    """Hierarchical H^1 family of order p on [0, 1]: phi_0..phi_p.

    phi_0 = 1 - x, phi_1 = x, phi_k = (P_k(xi) - P_{k-2}(xi)) / sqrt(2(2k-1))
    for k >= 2 (xi = 2x - 1).  Returns (values, d/dx), shape (p + 1, len(x)).
    """
    x = np.asarray(x, dtype=np.float64)
    P, dP = legendre_xi(max(p, 1), 2.0 * x - 1.0)
    V = np.zeros((p + 1,) + x.shape)
    D = np.zeros_like(V)
    V[0] = 1.0 - x
    D[0] = -1.0
    if p >= 1:
        V[1] = x
        D[1] = 1.0
    for k in range(2, p + 1):
        s = np.sqrt(2.0 * (2 * k - 1))
        V[k] = (P[k] - P[k - 2]) / s
        D[k] = 2.0 * (dP[k] - dP[k - 2]) / s
    return V, D
