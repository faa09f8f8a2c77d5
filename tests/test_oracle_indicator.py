"""Pins of the oracle's DPG error indicator (no GPU).

* a solution in the discrete trial space is reproduced, so every element
  residual vanishes (to rounding, relative to the element's load norm);
* minimum residual: around the discrete solution u the global residual
  J(v) = sum_K eta_K(v)^2 is exactly quadratic, J(u + d) - J(u) = d^* K d
  (K the block-diagonal element DPG matrices), for any admissible d;
* a plane wave: the global residual decays under h-refinement at about the
  rate p of the trial space.
"""
import numpy as np
import pytest

from oracle.assembly import build_fine
from oracle.element import boundary_faces, element_matrices
from oracle.indicator import element_residual, element_trial_vector, error_indicator
from oracle.problem import GaussianSource, Manufactured, PlaneWave


def _solve(fs):
    A, b = fs.assemble()
    x = np.linalg.solve(A.toarray(), b)
    return x, fs.fields(x)


def test_polynomial_solution_has_zero_residual():
    p = 2
    rng = np.random.default_rng(21)
    C = rng.standard_normal((4, p, p, p)) + 1j * rng.standard_normal((4, p, p, p))
    x0, x1 = (0.0, 0.0, 0.0), (1.0, 2.0, 1.0)
    ld = Manufactured(C, 4.0, x0, x1)
    fs = build_fine((2, 2, 2), p, 4.0, load=ld, x0=x0, x1=x1)
    x, f = _solve(fs)
    eta2 = error_indicator(fs, x, f)
    m = fs.mesh
    for e in range(m.n_elem):
        corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
        G, B, l = element_matrices(p, m.h, corner, 1.0, 4.0, boundary_faces(m, e), ld)
        ref = np.real(np.conj(l) @ np.linalg.solve(G, l))
        assert eta2[e] <= 1e-20 * ref, (e, eta2[e], ref)


def test_residual_is_exactly_quadratic_around_the_solution():
    p, n, om = 2, (2, 2, 2), 5.0
    fs = build_fine(n, p, om, load=GaussianSource((0.4, 0.5, 0.6), 0.2, 1.0))
    x, f = _solve(fs)
    J0 = error_indicator(fs, x, f).sum()
    rng = np.random.default_rng(3)
    dx = 1e-2 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
    df = 1e-2 * (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape))
    J1 = error_indicator(fs, x + dx, f + df).sum()
    quad = 0.0
    for e in range(fs.mesh.n_elem):
        d = element_trial_vector(fs, e, dx, df)
        quad += np.real(np.conj(d) @ fs.K[e] @ d)
    assert J1 > J0 >= 0.0
    assert abs((J1 - J0) - quad) < 1e-8 * quad
    # a perturbation of one element's fields alone costs exactly its own d^* K d
    e = 3
    df1 = np.zeros_like(f)
    df1[e] = df[e]
    J2 = error_indicator(fs, x, f + df1).sum()
    d = element_trial_vector(fs, e, np.zeros_like(x), df1)
    assert abs((J2 - J0) - np.real(np.conj(d) @ fs.K[e] @ d)) < 1e-8 * (J2 - J0)


@pytest.mark.parametrize("p,ns", [(2, (2, 4)), (3, (1, 2))])
def test_plane_wave_residual_decays_at_rate_p(p, ns):
    # measured rates at omega = 2: 1.89 (p = 2), 2.91 (p = 3)
    om = 2.0
    res = []
    for n in ns:
        ld = PlaneWave((1.0, 0.6, 0.3), om, 1.0)
        fs = build_fine((n, n, n), p, om, load=ld)
        x, f = _solve(fs)
        res.append(np.sqrt(error_indicator(fs, x, f).sum()))
    rate = np.log2(res[0] / res[1])
    assert abs(rate - p) < 0.3, (res, rate)
