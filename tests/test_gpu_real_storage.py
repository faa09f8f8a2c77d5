"""Real-packed storage of the mixed path (the default; the comparison is
DPGMG_FLAG_COMPLEX_STORAGE) through the C ABI.

Blocks touched only by elements without an impedance face and with a real
source are real once the unit phases of the real form are taken out (p-hat
DOFs carry i; Sec. 2, impedance condition and the test norm).  Such a vertex
patch keeps its FP32-factored inverse as a real matrix w with
A_j^-1[r][c] = w[r][c] i^(s_r - s_c); such a row entity of an operator keeps
its complex64 values (and the CG operator's high and low parts) as reals.
Every product applies the phases exactly.  Against complex64 storage of the
same values the products differ by FP32 rounding order only; against the
oracle they stay at the mixed path's parity bar.
"""
import numpy as np
import pytest

from oracle.hierarchy import smoother
from oracle.solver import mg_pcg, vcycle
from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import MIXED_THETA_TOL, MIXED_VCYCLE_TOL, oracle_system, rand_vec, rel

pytestmark = pytest.mark.gpu

CASES = [
    # 6^3 p = 2: interior vertex patches (indices 2..4 per axis) are real, the rest complex
    (dict(n=(6, 6, 6), p=2, omega=6.0, src_center=(0.4, 0.55, 0.5), src_width=0.2),
     dict(n_levels=3, p_min=1, precision="mixed", tol=1e-8)),
    # layered wavespeed, p3 -> p2 -> h -> h: every smoothed level of the headline's shape
    (dict(n=(8, 8, 4), p=3, omega=8.0, x1=(2.0, 2.0, 1.0), src_center=(1.0, 1.0, 0.5), src_width=0.1,
          wavespeed=np.repeat(np.random.default_rng(5).uniform(0.3, 1.0, 4), 64)),
     dict(n_levels=4, p_min=2, precision="mixed", tol=1e-8)),
    # p = 4 on a ragged mesh: patch sizes that are not multiples of 4 reals per row
    (dict(n=(5, 4, 4), p=4, omega=5.0, src_center=(0.5, 0.5, 0.5), src_width=0.2),
     dict(n_levels=2, p_min=3, precision="mixed", tol=1e-8)),
]


@pytest.mark.parametrize("pk,ok", CASES)
def test_packed_matches_complex_storage_and_oracle(pk, ok):
    okc = dict(ok, flags=D.FLAG_COMPLEX_STORAGE)
    fs, A, b, levels = oracle_system(pk, ok)
    L = len(levels) - 1
    with D.Solver(pk, **ok) as s0, D.Solver(pk, **okc) as s1:
        for l in range(1, L + 1):
            g0, g1 = s0.level(l), s1.level(l)
            assert g1.patch_real_sq == 0 and g0.sum_patch_sq == g1.sum_patch_sq
            assert 0 <= g0.patch_real_sq <= g0.sum_patch_sq
            if l == L:
                assert g0.patch_real_sq > 0   # the finest level has interior patches
            assert g1.op_real_nnz == 0 and 0 <= g0.op_real_nnz <= g0.op_nnz
            if l == L:
                assert g0.op_real_nnz > 0   # interior entities
            assert abs(g0.theta - g1.theta) < 1e-5 * g1.theta
            assert abs(g0.theta - levels[l].theta) < MIXED_THETA_TOL * levels[l].theta
            nl = levels[l].mesh.n_dof
            for G in (1, 16, 2, 4, 8, 64):   # row per warp (16: index prefetch), G rows of an entity, 64: half-warp
                D.dpgmg_spmv_group(s0.h, s0.s, l, G)
                x = rand_vec(nl, 50 + l)
                a0 = D.dpgmg_apply(s0.h, s0.s, D.OP_A, l, x, nl)
                assert rel(a0, D.dpgmg_apply(s1.h, s1.s, D.OP_A, l, x, nl)) < 1e-6
                assert rel(a0, levels[l].M @ x) < 1e-6
            for seed in (30 + l, 40 + l):
                x = rand_vec(nl, seed)
                y0 = D.dpgmg_apply(s0.h, s0.s, D.OP_SMOOTH, l, x, nl)
                y1 = D.dpgmg_apply(s1.h, s1.s, D.OP_SMOOTH, l, x, nl)
                assert rel(y0, y1) < 1e-5
                assert rel(y0, levels[l].theta * smoother(levels[l], x)) < MIXED_VCYCLE_TOL
        n = A.shape[0]
        v = rand_vec(n, 5)
        assert rel(D.dpgmg_apply(s0.h, s0.s, D.OP_VCYCLE, L, v, n), vcycle(levels, L, v)) < MIXED_VCYCLE_TOL
        for G in (1, 16, 2, 4, 8):   # the double-float CG operator on packed high and low parts
            D.dpgmg_spmv_group(s0.h, s0.s, -1, G)
            assert rel(D.dpgmg_apply(s0.h, s0.s, D.OP_AFULL, L, v, n), A @ v) < 1e-11
        x0, _, st0, c0 = s0.solve(fields=False)
        x1, _, st1, c1 = s1.solve(fields=False)
    assert c0 == c1 == D.DPGMG_OK
    assert abs(st0.iters - st1.iters) <= 1 and rel(x0, x1) < 1e-6
    assert st0.bytes_per_iter < st1.bytes_per_iter   # half the bytes of every real block
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    assert abs(st0.iters - it_ref) <= max(1, 0.1 * it_ref) and rel(x0, x_ref) < 1e-7


def test_packed_block_solve_and_c128_damping():
    """Several loads at once (block smoother, block SpMV and block CG operator
    on packed blocks) and the complex128 CG option, whose damping estimate
    streams the packed patch blocks in double-float arithmetic."""
    pk, ok = CASES[1]
    centers = [(1.0, 1.0, 0.5), (0.6, 1.3, 0.4), (1.4, 0.7, 0.6)]
    X1, B = [], []
    for c in centers:
        with D.Solver(dict(pk, src_center=c), **dict(ok, flags=D.FLAG_COMPLEX_STORAGE)) as s:
            B.append(D.dpgmg_rhs(s.h, s.s, s.n_trace))
            x, _, st, code = s.solve(fields=False)
            assert code == D.DPGMG_OK
            X1.append(x)
    with D.Solver(dict(pk, src_center=centers[0]), **ok) as s:
        code, X, stats = D.dpgmg_solve_block(s.h, s.s, np.array(B))
        assert code == D.DPGMG_OK
        for j in range(len(centers)):
            assert rel(X[j], X1[j]) < 1e-6 and stats[j].true_relres <= 1e-8
    okz = dict(ok, flags=D.FLAG_CG_C128)
    with D.Solver(pk, **okz) as s0, D.Solver(pk, **dict(okz, flags=D.FLAG_CG_C128 | D.FLAG_COMPLEX_STORAGE)) as s1:
        L = ok["n_levels"] - 1
        assert s0.level(L).patch_real_sq > 0 and s1.level(L).patch_real_sq == 0
        for l in range(1, L + 1):
            t0, t1 = s0.level(l).theta, s1.level(l).theta
            assert abs(t0 - t1) < 1e-5 * t1
        x0, _, st0, c0 = s0.solve(fields=False)
        x1, _, st1, c1 = s1.solve(fields=False)
    assert c0 == c1 == D.DPGMG_OK and abs(st0.iters - st1.iters) <= 1 and rel(x0, x1) < 1e-6
