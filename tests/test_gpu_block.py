"""Several loads at once (dpgmg_solve_block) through the C ABI.

Right-hand sides are the condensed loads of the same mesh and medium with
different Gaussian source positions (dpgmg_rhs of systems set up for each).
The block solve must give each column the single solve's result (the same
recurrence and preconditioner; 1e-10 on the FP64 path) and the oracle's
solution for that load at the parity bar.
"""
import numpy as np
import pytest

from oracle.solver import mg_pcg
from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import oracle_system, rel

pytestmark = pytest.mark.gpu

CENTERS = [(0.5, 0.5, 0.5), (0.3, 0.6, 0.45), (0.7, 0.35, 0.6), (0.45, 0.7, 0.3), (0.6, 0.55, 0.7)]


def _loads(pk, ok, centers):
    """Condensed loads and single-solve solutions (own system per source)."""
    bs, xs, its = [], [], []
    for c in centers:
        with D.Solver(dict(pk, src_center=c), **ok) as s:
            bs.append(D.dpgmg_rhs(s.h, s.s, s.n_trace))
            x, f, st, code = s.solve(fields=False)
            assert code == D.DPGMG_OK
            xs.append(x)
            its.append(st.iters)
    return np.array(bs), np.array(xs), its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 4, 5])
def test_block_solve_matches_single_solves(precision, k):
    pk = dict(n=(4, 4, 4), p=2, omega=4.0, src_width=0.15,
              wavespeed=np.random.default_rng(2).uniform(0.6, 1.2, 64))
    ok = dict(n_levels=3, p_min=1, precision=precision, tol=1e-8)
    B, Xs, its = _loads(pk, ok, CENTERS[:k])
    with D.Solver(dict(pk, src_center=CENTERS[0]), **ok) as s:
        code, X, stats = D.dpgmg_solve_block(s.h, s.s, B)
    assert code == D.DPGMG_OK
    for j in range(k):
        assert stats[j].relres <= 1e-8 and stats[j].true_relres <= 1e-8
        if precision == "fp64":
            assert stats[j].iters == its[j]
            assert rel(X[j], Xs[j]) < 1e-10, (j, rel(X[j], Xs[j]))
        else:
            # complex64 V-cycle: the block products sum in another order than
            # the single-vector kernels, so the iterates differ by FP32 rounding
            assert abs(stats[j].iters - its[j]) <= 1
            assert rel(X[j], Xs[j]) < 1e-6, (j, rel(X[j], Xs[j]))
    if k == 4:
        # against the oracle's PCG for each load (parity bar)
        for j in range(k):
            fs, A, b, levels = oracle_system(dict(pk, src_center=CENTERS[j]), ok)
            x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
            assert rel(B[j], b) < 1e-11
            assert abs(stats[j].iters - it_ref) <= max(1, 0.1 * it_ref)
            assert rel(X[j], x_ref) < 1e-7


def test_block_solve_zero_column_and_layered_hierarchy():
    # a zero right-hand side converges at once to x = 0 while the others iterate;
    # 8x8x4 p3 -> p2 -> 4x4x2 -> 2x2x1 (two stacked h-transitions), layered c
    c = np.repeat(np.random.default_rng(5).uniform(0.3, 1.0, 4), 64)
    pk = dict(n=(8, 8, 4), p=3, omega=8.0, src_width=0.1, x1=(2.0, 2.0, 1.0), wavespeed=c)
    ok = dict(n_levels=4, p_min=2, precision="mixed", tol=1e-8)
    centers = [(1.0, 1.0, 0.5), (0.6, 1.3, 0.4), (1.4, 0.7, 0.6)]
    B, Xs, its = _loads(pk, ok, centers)
    B = np.concatenate([B[:1], np.zeros_like(B[:1]), B[1:]])
    with D.Solver(dict(pk, src_center=centers[0]), **ok) as s:
        code, X, stats = D.dpgmg_solve_block(s.h, s.s, B)
    assert code == D.DPGMG_OK
    assert stats[1].iters == 0 and np.all(X[1] == 0)
    for j, jj in [(0, 0), (2, 1), (3, 2)]:
        assert abs(stats[j].iters - its[jj]) <= 1
        assert rel(X[j], Xs[jj]) < 1e-6
