"""Caller-supplied impedance data u0 (problem u0_samples, Sec. 2 impedance
condition Z^-1 p - u.n = u0) through the C ABI against the oracle.

The test picks a smooth non-polynomial u0, samples it at the points that
dpgmg_boundary_points lists and hands the samples to the library; the oracle
evaluates the same function at its own boundary quadrature points.  Loads,
PCG solution and error indicator must agree.
"""
import numpy as np
import pytest

from oracle.assembly import build_fine
from oracle.hierarchy import build_hierarchy
from oracle.indicator import error_indicator
from oracle.problem import GaussianSource, PlaneWave, WithImpedanceLoad
from oracle.solver import mg_pcg
from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import rel

TOL_FP64 = 1e-11

pytestmark = pytest.mark.gpu


def _u0_function(seed):
    rng = np.random.default_rng(seed)
    amp = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    k = rng.uniform(-6.0, 6.0, (3, 3))
    lin = rng.standard_normal(4) + 1j * rng.standard_normal(4)

    def u0(X, n=None, c=None):
        X = np.atleast_2d(X)
        v = np.exp(1j * (X @ k.T)) @ amp
        return v + lin[0] + X @ lin[1:]
    return u0


CASES = [
    # (problem, opts, base load of the oracle)
    (dict(n=(3, 2, 4), p=2, omega=5.0, x1=(1.5, 1.0, 2.0), src_center=(0.7, 0.5, 1.1), src_width=0.3,
          wavespeed=np.linspace(0.6, 1.4, 24)),
     dict(n_levels=2, p_min=1, precision="fp64", tol=1e-10), "gaussian"),
    (dict(n=(4, 4, 2), p=3, omega=6.0, src_center=(0.4, 0.5, 0.5), src_width=0.2, src_amp=0.0),
     dict(n_levels=3, p_min=2, precision="mixed", tol=1e-10), "gaussian"),
    (dict(n=(2, 3, 2), p=2, omega=4.0, source="plane_wave", wave_dir=(1.0, 0.3, -0.2)),
     dict(n_levels=2, p_min=1, precision="fp64", tol=1e-10), "plane_wave"),
]


@pytest.mark.parametrize("pk,ok,base", CASES)
def test_impedance_samples_match_oracle(pk, ok, base):
    fn = _u0_function(11)
    pb0, keep0 = D.make_problem(**pk)
    pts = D.dpgmg_boundary_points(pb0)
    pk = dict(pk, u0_samples=fn(pts))
    if base == "gaussian":
        bl = GaussianSource(pk["src_center"], pk["src_width"], pk.get("src_amp", 1.0))
    else:
        bl = PlaneWave(pk["wave_dir"], pk["omega"], 1.0)
    fs = build_fine(pk["n"], pk["p"], pk["omega"], wavespeed=pk.get("wavespeed"),
                    load=WithImpedanceLoad(bl, fn), x1=pk.get("x1", (1, 1, 1)))
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, ok["n_levels"], ok["p_min"])
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    with D.Solver(pk, **ok) as s:
        nt = A.shape[0]
        assert rel(D.dpgmg_rhs(s.h, s.s, nt), b) < TOL_FP64
        x, f, st, code = s.solve()
        assert code == D.DPGMG_OK
        assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref)
        assert rel(x, x_ref) < 1e-7
        nel = int(np.prod(pk["n"]))
        eta2 = D.dpgmg_error_indicator(s.h, s.s, x, nel)
    assert rel(eta2, error_indicator(fs, x)) < 1e-9
    # the samples matter: without them the load differs
    b_plain = build_fine(pk["n"], pk["p"], pk["omega"], wavespeed=pk.get("wavespeed"), load=bl,
                         x1=pk.get("x1", (1, 1, 1))).assemble()[1]
    assert rel(b_plain, b) > 1e-2
