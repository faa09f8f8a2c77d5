"""Edge and degenerate cases of the solve path, through the C ABI.

* zero load: b = 0 gives x = 0 and fields 0 after no CG step;
* one level: the V-cycle is the dense coarsest solve, so PCG converges at
  once and equals the oracle's dense solve;
* the smallest mesh (one element, p = 1) and a flat, ragged 1 x 2 x 5 mesh;
* a max_iter cap reports NOT_CONVERGED with the iterate written;
* invalid inputs are refused with DPGMG_ERR_ARG before any device work.
"""
import numpy as np
import pytest

from oracle.solver import mg_pcg
from paper_2304_01728_gb300 import dpgmg as D
from tests.oracle_adapter import oracle_system, rel

pytestmark = pytest.mark.gpu


def _solve(pk, ok):
    with D.Solver(pk, **ok) as s:
        x, f, st, code = s.solve()
    return x, f, st, code


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_load(precision):
    pk = dict(n=(3, 3, 3), p=2, omega=5.0, src_amp=0.0)
    x, f, st, code = _solve(pk, dict(n_levels=2, p_min=1, precision=precision))
    assert code == D.DPGMG_OK and st.iters == 0
    assert not np.any(x) and not np.any(f)


@pytest.mark.parametrize("n,p", [((1, 1, 1), 1), ((2, 1, 3), 2), ((3, 3, 3), 2)])
def test_single_level_is_a_direct_solve(n, p):
    pk = dict(n=n, p=p, omega=4.0, src_center=(0.4, 0.5, 0.6), src_width=0.3)
    ok = dict(n_levels=1, p_min=p, precision="fp64", tol=1e-10)
    fs, A, b, _ = oracle_system(pk, ok, hierarchy=False)
    x_ref = np.linalg.solve(A.toarray() if hasattr(A, "toarray") else A, b)
    x, f, st, code = _solve(pk, ok)
    assert code == D.DPGMG_OK and st.iters <= 2, st.iters
    assert rel(x, x_ref) < 1e-10
    f_ref = fs.fields(x_ref)
    assert rel(f.reshape(f_ref.shape), f_ref) < 1e-10


def test_flat_ragged_mesh_matches_oracle():
    pk = dict(n=(1, 2, 5), p=2, omega=6.0, x1=(0.4, 0.8, 2.0), src_center=(0.2, 0.4, 1.1), src_width=0.2)
    ok = dict(n_levels=2, p_min=1, precision="fp64", tol=1e-8)
    fs, A, b, levels = oracle_system(pk, ok)
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    x, f, st, code = _solve(pk, ok)
    assert code == D.DPGMG_OK
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(x, x_ref) < 1e-7


def test_iteration_cap_reports_not_converged():
    pk = dict(n=(4, 4, 4), p=2, omega=4.0)
    x, f, st, code = _solve(pk, dict(n_levels=2, p_min=1, precision="fp64", max_iter=2))
    assert code == D.DPGMG_ERR_NOT_CONVERGED
    assert st.iters == 2 and st.relres > 1e-8
    assert np.linalg.norm(x) > 0


@pytest.mark.parametrize("bad", [
    dict(problem=dict(n=(0, 4, 4))),
    dict(problem=dict(omega=0.0)),
    dict(problem=dict(omega=-1.0)),
    dict(problem=dict(p=6)),
    dict(problem=dict(src_width=0.0)),
    dict(problem=dict(x1=(1.0, 0.0, 1.0))),
    dict(problem=dict(wavespeed=np.r_[np.ones(63), -1.0])),
    dict(problem=dict(wavespeed=np.r_[np.ones(63), np.nan])),
    dict(opts=dict(tol=0.0)),
    dict(opts=dict(n_levels=0)),
    dict(opts=dict(max_iter=0)),
    dict(opts=dict(flags=1 << 20)),
    dict(problem=dict(wavespeed=np.r_[np.ones(63), 2.0]), opts=dict(flags=4)),   # stored needs constant c
])
def test_invalid_inputs_are_refused(bad):
    pk = dict(dict(n=(4, 4, 4), p=2, omega=4.0), **bad.get("problem", {}))
    ok = dict(dict(n_levels=2, p_min=1), **bad.get("opts", {}))
    pb, keep = D.make_problem(**pk)
    op = D.make_opts(**ok)
    with pytest.raises(D.DpgmgError) as e:
        D.dpgmg_query_sizes(pb, op)
    assert e.value.code == D.DPGMG_ERR_ARG
    h = D.dpgmg_create(0)
    try:
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, op)
        assert e.value.code == D.DPGMG_ERR_ARG
    finally:
        D.dpgmg_destroy(h)


def test_warm_start():
    pk = dict(n=(4, 4, 4), p=2, omega=6.0, src_center=(0.4, 0.5, 0.6))
    ok = dict(n_levels=2, p_min=1, precision="fp64", tol=1e-8)
    x, f, st, code = _solve(pk, ok)
    assert code == D.DPGMG_OK
    cold = st.iters
    with D.Solver(pk, **dict(ok, flags=D.FLAG_WARM_START)) as s:
        # from the converged solution: no iteration, the guess is returned
        g = x.copy()
        code, st = D.dpgmg_solve(s.h, s.s, g, None)
        assert code == D.DPGMG_OK and st.iters == 0 and st.relres <= ok["tol"]
        assert np.array_equal(g, x)
        # from a perturbed solution: converges in fewer iterations to the same solution
        rng = np.random.default_rng(2)
        g = x + 1e-4 * np.abs(x).max() * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
        code, st = D.dpgmg_solve(s.h, s.s, g, None)
        assert code == D.DPGMG_OK and 0 < st.iters < cold, (st.iters, cold)
        assert rel(g, x) < 1e-6
        # from zero: the cold iteration
        g = np.zeros_like(x)
        code, st = D.dpgmg_solve(s.h, s.s, g, None)
        assert code == D.DPGMG_OK and st.iters == cold
        assert rel(g, x) < 1e-12


def test_setup_phases_add_up():
    pk = dict(n=(6, 6, 6), p=2, omega=8.0, src_center=(0.5, 0.45, 0.55), src_width=0.2)
    with D.Solver(pk, n_levels=3, p_min=1, precision="mixed") as s:
        ph = D.dpgmg_setup_phases(s.h, s.s)
        el_ms, gflop, setup_ms = D.dpgmg_setup_profile(s.h, s.s)
    assert len(ph) == len(D.SETUP_PHASES) and min(ph) >= 0.0
    assert ph[0] == pytest.approx(el_ms)
    assert ph[0] + ph[1] + ph[2] + ph[4] + ph[5] == pytest.approx(setup_ms, rel=1e-3)
    assert ph[3] > 0.0   # the coarsest factorisation ran on the side stream


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_setup_and_solve_are_bitwise_reproducible(precision):
    # no atomics anywhere on the path (assembly in element-colour passes,
    # reductions in a fixed order): two systems of one problem agree bitwise
    pk = dict(n=(5, 4, 6), p=2, omega=7.0, src_center=(0.4, 0.6, 0.5), src_width=0.2,
              wavespeed=np.linspace(0.7, 1.3, 120))
    ok = dict(n_levels=3, p_min=1, precision=precision)
    runs = [_solve(pk, ok) for _ in range(2)]
    assert runs[0][3] == runs[1][3] == D.DPGMG_OK
    assert runs[0][2].iters == runs[1][2].iters
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("n,p,prec,layers", [((6, 6, 6), 2, "fp64", 0), ((8, 7, 6), 3, "mixed", 0),
                                              ((8, 7, 6), 3, "mixed", 3)])
def test_element_class_reuse_matches_full_pipeline(n, p, prec, layers, monkeypatch):
    # element classes = (impedance-face mask, wavespeed): 27 with a constant
    # wavespeed, up to 27 per distinct wavespeed with `layers` horizontal layers;
    # members of a class take the representative's factors and compute only
    # their load
    pk = dict(n=n, p=p, omega=9.0, src_center=(0.45, 0.55, 0.5), src_width=0.15)
    if layers:
        speeds = np.random.default_rng(7).uniform(0.3, 1.0, layers)
        kz = np.arange(n[2]) * layers // n[2]
        pk["wavespeed"] = np.repeat(speeds[kz], n[0] * n[1])
    ok = dict(n_levels=2, p_min=p - 1, precision=prec)
    nel = int(np.prod(n))
    picks = [0, n[0] // 2, (n[1] // 2) * n[0] + n[0] // 2, nel // 2 + n[0] // 2, nel - 1, nel // 3,
             nel - n[0] * n[1] // 2, n[0] * n[1] * (n[2] // 2) + 5]
    out = {}
    for reuse in ("0", "1"):
        monkeypatch.setenv("DPGMG_ELEMENT_REUSE", reuse)
        with D.Solver(pk, **ok) as s:
            ntr = (p + 1) ** 3 - (p - 1) ** 3 + 6 * p * p   # local traces: u-hat (H^1 trace) and p-hat
            mats = [D.dpgmg_element_matrix(s.h, s.s, ok["n_levels"] - 1, e, ntr, with_load=True) for e in picks]
            gflop = D.dpgmg_setup_profile(s.h, s.s)[1]
            x, f, st, code = s.solve()
            assert code == D.DPGMG_OK
            out[reuse] = (mats, x, f, st.iters, gflop)
    (m0, x0, f0, i0, g0), (m1, x1, f1, i1, g1) = out["0"], out["1"]
    assert g1 < 0.5 * g0, (g1, g0)   # the classes were used
    for a, b in zip(m0, m1):
        assert rel(b[0], a[0]) < 1e-13 and rel(b[1], a[1]) < 1e-11
    if prec == "fp64":
        assert i1 == i0
        assert rel(x1, x0) < 1e-9 and rel(f1, f0) < 1e-9
    else:
        # complex64 patch blocks rounded from operators that agree to ~1e-13 and
        # factored in FP32: the preconditioners may differ in a few entries
        assert abs(i1 - i0) <= 1
        assert rel(x1, x0) < 1e-7 and rel(f1, f0) < 1e-7

