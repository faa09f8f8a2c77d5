"""DPG error indicator on the GPU against the oracle (same trace vector on
both sides), and its defining property on a polynomial solution."""
import numpy as np
import pytest

from oracle.indicator import error_indicator
from paper_2304_01728_gb300 import dpgmg as D
from paper_2304_01728_gb300 import workloads
from tests.oracle_adapter import oracle_system, rel

pytestmark = pytest.mark.gpu

CASES = [
    (workloads.config1()["problem"], dict(n_levels=2, p_min=1, precision="fp64")),
    (dict(n=(3, 2, 4), p=3, omega=7.0, x1=(1.5, 1.0, 2.0), src_center=(0.7, 0.5, 1.1), src_width=0.3,
          wavespeed=np.linspace(0.6, 1.4, 24)), dict(n_levels=2, p_min=2, precision="mixed")),
    (dict(n=(3, 3, 3), p=2, omega=5.0, source="plane_wave", wave_dir=(1.0, 0.4, -0.3)),
     dict(n_levels=2, p_min=1, precision="fp64")),
]


@pytest.mark.parametrize("pk,ok", CASES)
def test_indicator_matches_oracle(pk, ok):
    with D.Solver(pk, **ok) as s:
        x, f, st, code = s.solve()
        assert code == D.DPGMG_OK
        nel = int(np.prod(pk["n"]))
        eta2 = D.dpgmg_error_indicator(s.h, s.s, x, nel)
        eta0 = D.dpgmg_error_indicator(s.h, s.s, np.zeros_like(x), nel)
    fs, _, _, _ = oracle_system(pk, ok, hierarchy=False)
    ref = error_indicator(fs, x)
    assert np.all(eta2 >= 0.0)
    assert rel(eta2, ref) < 1e-9, rel(eta2, ref)
    # the solution lowers the residual of the zero vector
    assert eta2.sum() < eta0.sum()


def test_polynomial_solution_has_zero_indicator():
    p = 2
    rng = np.random.default_rng(5)
    C = rng.standard_normal((4, p, p, p)) + 1j * rng.standard_normal((4, p, p, p))
    pk = dict(n=(2, 3, 2), p=p, omega=3.0, source="manufactured", mf_coeffs=C)
    with D.Solver(pk, n_levels=2, p_min=1, precision="fp64", tol=1e-13) as s:
        x, f, st, code = s.solve()
        assert code == D.DPGMG_OK
        eta2 = D.dpgmg_error_indicator(s.h, s.s, x, 12)
        eta0 = D.dpgmg_error_indicator(s.h, s.s, np.zeros_like(x), 12)
    assert eta2.sum() < 1e-18 * eta0.sum(), (eta2.sum(), eta0.sum())
