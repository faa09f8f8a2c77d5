"""Memory-lean smoother (DPGMG_FLAG_RECOMPUTE_PATCHES, Sec. 5: patches
recomputed during the solve instead of stored) through the C ABI.

The recomputed patch inverses come from the same FP32 factorisation of the
same complex64 blocks as the stored ones, so the smoother, theta, iterations
and solution agree with the stored path (to FP32 rounding where the stored
path factors a level's patches by thread-block clusters) and with the oracle
at the parity bar; no patch inverse is stored.
"""
import numpy as np
import pytest

from oracle.hierarchy import smoother
from oracle.solver import mg_pcg, vcycle
from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import MIXED_THETA_TOL, MIXED_VCYCLE_TOL, oracle_system, rand_vec, rel

pytestmark = pytest.mark.gpu

CASES = [
    (dict(n=(4, 4, 4), p=2, omega=4.0, src_center=(0.4, 0.55, 0.5), src_width=0.2),
     dict(n_levels=3, p_min=1, precision="mixed", tol=1e-8)),
    (dict(n=(8, 8, 4), p=3, omega=8.0, x1=(2.0, 2.0, 1.0), src_center=(1.0, 1.0, 0.5), src_width=0.1,
          wavespeed=np.repeat(np.random.default_rng(5).uniform(0.3, 1.0, 4), 64)),
     dict(n_levels=4, p_min=2, precision="mixed", tol=1e-8)),
    (dict(n=(4, 4, 4), p=2, omega=4.0, src_center=(0.4, 0.55, 0.5), src_width=0.2),
     dict(n_levels=2, p_min=1, precision="mixed", tol=1e-8, coarsest="smooth")),
]


@pytest.mark.parametrize("pk,ok", CASES)
def test_recompute_matches_stored_and_oracle(pk, ok):
    okr = dict(ok, flags=D.FLAG_RECOMPUTE_PATCHES)
    fs, A, b, levels = oracle_system(pk, ok)
    L = len(levels) - 1
    with D.Solver(pk, **ok) as s0, D.Solver(pk, **okr) as s1:
        for l in range(L + 1):
            g0, g1 = s0.level(l), s1.level(l)
            if g0.n_patches == 0:
                continue
            assert g1.n_patches == g0.n_patches and g1.sum_patch_sq == g0.sum_patch_sq
            assert g1.patch_stored == 0 and g0.patch_stored > 0
            assert abs(g1.theta - g0.theta) < 1e-5 * g0.theta
            assert abs(g1.theta - levels[l].theta) < MIXED_THETA_TOL * levels[l].theta
            nl = levels[l].mesh.n_dof
            x = rand_vec(nl, 20 + l)
            y1 = D.dpgmg_apply(s1.h, s1.s, D.OP_SMOOTH, l, x, nl)
            y0 = D.dpgmg_apply(s0.h, s0.s, D.OP_SMOOTH, l, x, nl)
            assert rel(y1, y0) < 1e-5
            assert rel(y1, levels[l].theta * smoother(levels[l], x)) < MIXED_VCYCLE_TOL
        n = A.shape[0]
        v = rand_vec(n, 4)
        assert rel(D.dpgmg_apply(s1.h, s1.s, D.OP_VCYCLE, L, v, n), vcycle(levels, L, v)) < MIXED_VCYCLE_TOL
        x0, _, st0, c0 = s0.solve(fields=False)
        x1, _, st1, c1 = s1.solve(fields=False)
    assert c0 == c1 == D.DPGMG_OK
    assert abs(st1.iters - st0.iters) <= 1 and rel(x1, x0) < 1e-6
    assert s1.dev_bytes < s0.dev_bytes   # the memory estimate drops the stored inverses
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    assert abs(st1.iters - it_ref) <= max(1, 0.1 * it_ref) and rel(x1, x_ref) < 1e-7


def test_recompute_block_solve_and_options():
    pk, ok = CASES[1]
    okr = dict(ok, flags=D.FLAG_RECOMPUTE_PATCHES)
    centers = [(1.0, 1.0, 0.5), (0.6, 1.3, 0.4), (1.4, 0.7, 0.6), (0.8, 0.8, 0.3)]
    B, X1 = [], []
    for c in centers:
        with D.Solver(dict(pk, src_center=c), **okr) as s:
            B.append(D.dpgmg_rhs(s.h, s.s, s.n_trace))
            x, _, st, code = s.solve(fields=False)
            assert code == D.DPGMG_OK
            X1.append(x)
    with D.Solver(dict(pk, src_center=centers[0]), **okr) as s:
        code, X, stats = D.dpgmg_solve_block(s.h, s.s, np.array(B))
        assert code == D.DPGMG_OK
        for j in range(len(centers)):
            assert rel(X[j], X1[j]) < 1e-6 and stats[j].true_relres <= 1e-8
        # no stored inverses: the allocation-free smoother entry point refuses
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_smooth_noalloc(s.h, s.s, 1, 0, 0)
        assert e.value.code == D.DPGMG_ERR_ARG
    # recompute mode is the mixed path's FP32 factorisation only
    pb, keep = D.make_problem(**pk)
    for bad in [dict(ok, precision="fp64"), dict(ok, flags=D.FLAG_RECOMPUTE_PATCHES | D.FLAG_PATCH_FP64),
                dict(ok, flags=D.FLAG_RECOMPUTE_PATCHES | D.FLAG_CG_C128)]:
        bad.setdefault("flags", D.FLAG_RECOMPUTE_PATCHES)
        with pytest.raises(D.DpgmgError):
            D.dpgmg_query_sizes(pb, D.make_opts(**bad))
