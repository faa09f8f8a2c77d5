"""The complex128 CG operator (DPGMG_FLAG_CG_C128) against the oracle.

Sec. 3 runs CG on the condensed FP64 trace system.  By default the library
applies that operator in double-float arithmetic (complex64 high and low
parts of each FP64 entry, error-free FP32 products and sums, ~48 bits); the
flag applies it in complex128 on the FP64 pipe and also runs the damping
estimate in FP64, so that with the FP64 V-cycle every step is complex128
(the 4^3, p = 2 workload's "complex128 throughout").  Both forms are checked
against the oracle: the operator at 1e-11 (1e-13 for complex128), theta at
1e-9 (1e-4 on the mixed path, whose patch factors are FP32), the solution at the parity bar of 1e-7 with the iteration count within
10%; the relative L2 error of each form against the oracle is printed.
"""
import numpy as np
import pytest

from oracle.solver import mg_pcg
from paper_2304_01728_gb300 import dpgmg as D
from paper_2304_01728_gb300 import workloads
from tests.oracle_adapter import MIXED_THETA_TOL, oracle_system, rand_vec, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1_oracle():
    w = workloads.config1()
    fs, A, b, levels = oracle_system(w["problem"], w["opts"])
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=w["opts"]["tol"])
    return w, fs, A, b, levels, x_ref, it_ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("flags", [0, D.FLAG_CG_C128])
def test_cg_operator_forms_against_oracle(c1_oracle, precision, flags):
    w, fs, A, b, levels, x_ref, it_ref = c1_oracle
    ok = dict(w["opts"], precision=precision, flags=flags)
    L = len(levels) - 1
    with D.Solver(w["problem"], **ok) as s:
        x = rand_vec(A.shape[0], 3)
        y = D.dpgmg_apply(s.h, s.s, D.OP_AFULL, L, x, A.shape[0])
        err_op = rel(y, A @ x)
        assert err_op < (1e-13 if flags else 1e-11), err_op
        th_tol = 1e-9 if precision == "fp64" else MIXED_THETA_TOL   # mixed: FP32 patch factors
        for l in range(1, L + 1):
            assert abs(s.level(l).theta - levels[l].theta) < th_tol * levels[l].theta
        xs, f, st, code = s.solve()
    err = rel(xs, x_ref)
    print("CG operator %s, %s V-cycle: operator error %.2e, solution error %.2e, iterations %d (oracle %d), "
          "PCG %.2f ms" % ("complex128" if flags else "double-float", precision, err_op, err, st.iters, it_ref,
                           st.t_pcg_ms))
    assert code == D.DPGMG_OK and st.true_relres <= 10 * ok["tol"]
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref)
    assert err < 1e-7
    f_ref = fs.fields(x_ref)
    assert rel(f.reshape(f_ref.shape), f_ref) < 1e-7


def test_cg_operator_forms_agree_on_an_h_hierarchy():
    """4^3 p2 -> 2^3 p2 with varying wavespeed: an h-transition below the
    finest level, so the CG operator is assembled apart from the smoothing
    (macro) operator; both forms give the same iterations and solutions within
    the parity bar of each other."""
    c = np.random.default_rng(11).uniform(0.6, 1.4, 64)
    pk = dict(n=(4, 4, 4), p=2, omega=5.0, wavespeed=c, src_center=(0.3, 0.6, 0.45), src_width=0.15)
    out = {}
    for flags in (0, D.FLAG_CG_C128):
        with D.Solver(pk, n_levels=2, p_min=2, precision="mixed", flags=flags) as s:
            x, f, st, code = s.solve()
        assert code == D.DPGMG_OK
        out[flags] = (x, st.iters)
    assert abs(out[0][1] - out[D.FLAG_CG_C128][1]) <= 1
    assert rel(out[0][0], out[D.FLAG_CG_C128][0]) < 1e-7
