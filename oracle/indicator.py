"""DPG error indicator (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The DPG method minimises the residual of the ultraweak formulation in the
dual test norm; its element contributions are the method's built-in error
indicator (Sec. 1.2; the refinements of Sec. 3 and the "DPG residual" curves
of Sec. 4-5 are driven by it):

    eta_K^2 = (l_K - B_K u_K)^* G_K^{-1} (l_K - B_K u_K),

with the element Gram matrix G_K of the adjoint graph norm (Eq. Gnorm), the
enriched stiffness B_K = [B_field | B_trace] and load l_K of
``oracle.element.element_matrices``, and u_K the element's trial vector
(fields, then local traces; absent traces are zero).  The global DPG
residual is sum_K eta_K^2, which the discrete solution minimises over the
trial space.

Parity unpinned here; pinned by ``tests/test_oracle_indicator.py``
(polynomial solution reproduced => eta = 0; the exact quadratic identity
J(u + d) - J(u) = d^* K d around the discrete solution; plane-wave decay).
"""
import numpy as np

from .element import boundary_faces, element_matrices


def element_residual(fs, e, u):
    """eta_K^2 of element e for the element trial vector u = [fields, local traces]."""
    m = fs.mesh
    corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
    G, B, l = element_matrices(m.p, m.h, corner, fs.c[e], fs.omega, boundary_faces(m, e), fs.load)
    r = l - B @ u
    return float(np.real(np.conj(r) @ np.linalg.solve(G, r)))


def element_trial_vector(fs, e, x, fields):
    """[fields of e, its local traces from the global trace vector x (absent => 0)]."""
    g = fs.dofs[e]
    xt = np.where(g >= 0, x[np.maximum(g, 0)], 0.0)
    return np.concatenate([fields[e], xt])


def error_indicator(fs, x, fields=None):
    """eta_K^2 for every element, from the global trace solution x (fields recovered if not given)."""
    if fields is None:
        fields = fs.fields(x)
    return np.array([element_residual(fs, e, element_trial_vector(fs, e, x, fields))
                     for e in range(fs.mesh.n_elem)])
