"""Patch inversion by thread-block clusters (2 or 4 CTAs per patch) against
one CTA per patch.

Every output tile of the cluster version is computed by one CTA with the same
instructions in the same order as the single-CTA version, and setup is
bitwise reproducible (assembly in element-colour passes, no atomics), so the
patch inverses, theta, the smoother and the solution are bitwise equal.  The
cases
cover complex patches, patches on the real path (interior of a 6^3 mesh),
vertex patches of a p-level and macro patches of an h-level, with sizes below,
at and above the 32-row tile edge.  The oracle comparison of the default
choice is in test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import rand_vec, rel

pytestmark = pytest.mark.gpu

CASES = [
    (dict(n=(4, 4, 4), p=2, omega=5.0, wavespeed=np.random.default_rng(11).uniform(0.6, 1.4, 64),
          src_center=(0.3, 0.6, 0.45), src_width=0.15, x1=(1.0, 1.2, 0.9)),
     dict(n_levels=3, p_min=1, precision="fp64")),
    (dict(n=(6, 6, 6), p=2, omega=8.0, src_center=(0.5, 0.45, 0.55), src_width=0.2),
     dict(n_levels=2, p_min=2, precision="fp64")),
    (dict(n=(4, 4, 4), p=3, omega=9.0, src_center=(0.45, 0.5, 0.55), src_width=0.2),
     dict(n_levels=3, p_min=2, precision="fp64")),
    # complex64 blocks factored in FP32 (the mixed path), macro patches of two h-levels
    (dict(n=(8, 8, 8), p=2, omega=6.0, src_center=(0.4, 0.5, 0.6), src_width=0.15),
     dict(n_levels=3, p_min=2, precision="mixed")),
]


def _run(pk, ok, team, monkeypatch):
    monkeypatch.setenv("DPGMG_PATCH_TEAM", str(team))
    out = []
    with D.Solver(pk, **ok) as s:
        L = ok["n_levels"] - 1
        for l in range(1, L + 1):
            g = s.level(l)
            x = rand_vec(g.n_dof, 30 + l)
            y = D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, l, x, g.n_dof)
            out.append((g.theta, g.patch_max, y))
        x, f, st, code = s.solve()
        assert code == D.DPGMG_OK
        out.append((st.iters, x))
    return out


@pytest.mark.parametrize("pk,ok", CASES)
def test_cluster_patch_inversion_is_bitwise_single_cta(pk, ok, monkeypatch):
    ref = _run(pk, ok, 1, monkeypatch)
    assert max(r[1] for r in ref[:-1]) > 32   # some patch spans several tiles
    for team in (2, 4):
        got = _run(pk, ok, team, monkeypatch)
        for (th0, n0, y0), (th1, n1, y1) in zip(ref[:-1], got[:-1]):
            assert n1 == n0
            assert th1 == th0, (team, th0, th1)
            assert np.array_equal(y1, y0), (team, rel(y1, y0))
        assert got[-1][0] == ref[-1][0]
        assert np.array_equal(got[-1][1], ref[-1][1])
