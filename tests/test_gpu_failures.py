"""Error statuses raised by failures made on the host, through the C ABI.

No GPU fault is involved: a NaN in a warm-start guess drives CG to a
non-finite (p, Ap) (DPGMG_ERR_BREAKDOWN); the host overwrites one entry of
the dense coarsest matrix with a negative pivot before its factorisation
(DPGMG_ERR_NOT_HPD); the tensor-core update issues no MMA so that its bounded
wait runs out with nothing in flight (DPGMG_ERR_TIMEOUT).  After each failure
the handle (and, for BREAKDOWN, the system) is used again and gives the
regular result.
"""
import numpy as np
import pytest

from paper_2304_01728_gb300 import dpgmg as D
from paper_2304_01728_gb300 import workloads
from tests.oracle_adapter import rel

pytestmark = pytest.mark.gpu


def _setup_solve(h, pk, ok):
    pb, keep = D.make_problem(**pk)
    op = D.make_opts(**ok)
    nt, nf, _ = D.dpgmg_query_sizes(pb, op)
    s = D.dpgmg_setup(h, pb, op)
    try:
        x = np.zeros(nt, complex)
        code, st = D.dpgmg_solve(h, s, x, None)
    finally:
        D.dpgmg_release(h, s)
    return code, st, x


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_breakdown_from_nan_guess_then_usable(precision):
    w = workloads.config1()
    ok = dict(w["opts"], precision=precision)
    h = D.dpgmg_create(0)
    try:
        code, st, x_ref = _setup_solve(h, w["problem"], ok)
        assert code == D.DPGMG_OK
        pb, keep = D.make_problem(**w["problem"])
        op = D.make_opts(**dict(ok, flags=D.FLAG_WARM_START))
        s = D.dpgmg_setup(h, pb, op)
        try:
            g = np.zeros_like(x_ref)
            g[len(g) // 3] = np.nan
            with pytest.raises(D.DpgmgError) as e:
                D.dpgmg_solve(h, s, g, None)
            assert e.value.code == D.DPGMG_ERR_BREAKDOWN
            # the same system, from a finite guess: the regular solution
            g = np.zeros_like(x_ref)
            code, st = D.dpgmg_solve(h, s, g, None)
            assert code == D.DPGMG_OK and rel(g, x_ref) < 1e-12
        finally:
            D.dpgmg_release(h, s)
    finally:
        D.dpgmg_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_not_hpd_from_host_fault_then_usable(precision):
    w = workloads.config1()
    ok = dict(w["opts"], precision=precision)
    h = D.dpgmg_create(0)
    try:
        pb, keep = D.make_problem(**w["problem"])
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, D.make_opts(**dict(ok, flags=D.FLAG_FAULT_NOT_HPD)))
        assert e.value.code == D.DPGMG_ERR_NOT_HPD
        code, st, x = _setup_solve(h, w["problem"], ok)
        assert code == D.DPGMG_OK and st.relres <= ok["tol"]
    finally:
        D.dpgmg_destroy(h)


def test_tensor_core_wait_timeout_then_usable():
    # 6^3 p2 -> 6^3 p1: level 0 has 883 DOFs, factored in 128-wide panels whose
    # products run on the tensor cores
    w = workloads.config1()
    w["problem"]["n"] = (6, 6, 6)
    ok = dict(w["opts"], precision="mixed")
    h = D.dpgmg_create(0)
    try:
        pb, keep = D.make_problem(**w["problem"])
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, D.make_opts(**dict(ok, flags=D.FLAG_FAULT_TC_WAIT)))
        assert e.value.code == D.DPGMG_ERR_TIMEOUT
        code, st, x = _setup_solve(h, w["problem"], ok)
        assert code == D.DPGMG_OK and st.relres <= ok["tol"]
        code, st, x64 = _setup_solve(h, w["problem"], dict(w["opts"], precision="fp64"))
        assert code == D.DPGMG_OK and rel(x, x64) < 1e-6
    finally:
        D.dpgmg_destroy(h)
