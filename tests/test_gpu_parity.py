"""GPU parity of every step of the DPG-MG hot path against the FP64 oracle.

All calls go through the C ABI (libdpgmg.so via the ctypes binding).  The
FP64 path is compared at 1e-11 relative (roundoff of a different but
equivalent arithmetic order: the library uses the real form of the Gram
matrix and closed-form 1D integrals, the oracle complex quadrature); the
solution at the parity bar of 1e-7 relative L2 with the iteration count
within 10% (equal in practice on the FP64 path).
"""
import numpy as np
import pytest

from oracle.solver import mg_pcg, vcycle
from oracle.traces import field_dofs, trace_dofs
from paper_2304_01728_gb300 import dpgmg as D
from paper_2304_01728_gb300 import workloads
from tests.oracle_adapter import MIXED_VCYCLE_TOL, oracle_system, rand_vec, rel

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


class Case:
    def __init__(self, pk, ok):
        self.pk, self.ok = pk, ok
        self.solver = D.Solver(pk, **ok)
        self.fs, self.A, self.b, self.levels = oracle_system(pk, ok)
        self.L = len(self.levels) - 1

    def gpu_level(self, l):
        return self.solver.level(l)


@pytest.fixture(scope="module")
def c1():
    w = workloads.config1()
    c = Case(w["problem"], w["opts"])
    yield c
    c.solver.close()


@pytest.fixture(scope="module")
def ph():
    """4^3 p2 -> 4^3 p1 -> 2^3 p1: a p- and an h-transition, heterogeneous c."""
    c = np.random.default_rng(11).uniform(0.6, 1.4, 64)
    pk = dict(n=(4, 4, 4), p=2, omega=5.0, wavespeed=c, src_center=(0.3, 0.6, 0.45), src_width=0.15,
              x0=(0, 0, 0), x1=(1.0, 1.2, 0.9))
    ok = dict(n_levels=3, p_min=1, precision="fp64", tol=1e-10)
    case = Case(pk, ok)
    yield case
    case.solver.close()


@pytest.fixture(scope="module")
def hh():
    """4^3 p2 -> 2^3 p2: one h-transition at p = 2."""
    pk = dict(n=(4, 4, 4), p=2, omega=6.0, src_center=(0.55, 0.45, 0.5), src_width=0.2)
    ok = dict(n_levels=2, p_min=2, precision="fp64", tol=1e-10)
    case = Case(pk, ok)
    yield case
    case.solver.close()


CASES = ["c1", "ph", "hh"]


@pytest.mark.parametrize("name", CASES)
def test_element_matrices_every_level(name, request):
    c = request.getfixturevalue(name)
    s = c.solver
    for l in range(c.L + 1):
        lev = c.levels[c.L - l] if False else c.levels[l]
        nloc = lev.E.shape[1]
        for e in range(lev.E.shape[0]):
            M = D.dpgmg_element_matrix(s.h, s.s, l, e, nloc)
            assert rel(M, lev.E[e]) < TOL_FP64, (l, e, rel(M, lev.E[e]))
    # finest condensed loads
    nloc = c.fs.Kc.shape[1]
    for e in range(c.fs.mesh.n_elem):
        _, F = D.dpgmg_element_matrix(s.h, s.s, c.L, e, nloc, with_load=True)
        assert rel(F, c.fs.Fc[e]) < TOL_FP64


@pytest.mark.parametrize("name", CASES)
def test_rhs_and_cg_operator(name, request):
    c = request.getfixturevalue(name)
    s = c.solver
    b = D.dpgmg_rhs(s.h, s.s, c.A.shape[0])
    assert rel(b, c.b) < TOL_FP64
    x = rand_vec(c.A.shape[0], 1)
    y = D.dpgmg_apply(s.h, s.s, D.OP_AFULL, c.L, x, c.A.shape[0])
    assert rel(y, c.A @ x) < TOL_FP64


@pytest.mark.parametrize("name", CASES)
def test_level_structure_and_theta(name, request):
    c = request.getfixturevalue(name)
    for l in range(1, c.L + 1):
        g = c.gpu_level(l)
        o = c.levels[l]
        assert g.n_dof == o.mesh.n_dof
        assert g.kind == {"p": 1, "h": 2}[o.kind]
        sizes = np.array([len(x) for x in o.patches])
        assert g.n_patches == len(sizes) and g.patch_max == sizes.max()
        assert g.sum_patch_sq == int(np.sum(sizes ** 2))
        assert g.n_smooth == int(o.smask.sum())
        assert abs(g.theta - o.theta) < 1e-9 * o.theta, (g.theta, o.theta)


@pytest.mark.parametrize("name", CASES)
def test_smoothing_operator_and_smoother(name, request):
    c = request.getfixturevalue(name)
    s = c.solver
    for l in range(1, c.L + 1):
        o = c.levels[l]
        n = o.mesh.n_dof
        x = rand_vec(n, 10 + l)
        y = D.dpgmg_apply(s.h, s.s, D.OP_A, l, x, n)
        assert rel(y, o.M @ x) < TOL_FP64
        from oracle.hierarchy import smoother
        y = D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, l, x, n)
        assert rel(y, o.theta * smoother(o, x)) < TOL_FP64


@pytest.mark.parametrize("name", CASES)
def test_transfers(name, request):
    c = request.getfixturevalue(name)
    s = c.solver
    for l in range(1, c.L + 1):
        o, oc = c.levels[l], c.levels[l - 1]
        nf, nc = o.mesh.n_dof, oc.mesh.n_dof
        x = rand_vec(nf, 20 + l)
        xc = rand_vec(nc, 30 + l)
        r = D.dpgmg_apply(s.h, s.s, D.OP_RESTRICT, l, x, nc)
        p = D.dpgmg_apply(s.h, s.s, D.OP_PROLONG, l, xc, nf)
        if o.kind == "p":
            assert np.array_equal(r, x[o.inj])
            ref = np.zeros(nf, dtype=complex)
            ref[o.inj] = xc
            assert np.array_equal(p, ref)
        else:
            assert rel(r, o.P.conj().T @ x) < 1e-13
            assert rel(p, o.P @ xc) < 1e-13
            y = D.dpgmg_apply(s.h, s.s, D.OP_CONDENSE, l, x, nf)
            ref = np.where(o.smask, x, 0)
            for Sg, Ig, T in zip(o.S, o.I, o.T):
                ref[Sg] -= T @ x[Ig]
            assert rel(y, ref) < TOL_FP64


@pytest.mark.parametrize("name", CASES)
def test_coarse_solve_and_vcycle(name, request):
    c = request.getfixturevalue(name)
    s = c.solver
    import scipy.linalg as sla
    o0 = c.levels[0]
    x = rand_vec(o0.mesh.n_dof, 5)
    y = D.dpgmg_apply(s.h, s.s, D.OP_COARSE, 0, x, o0.mesh.n_dof)
    assert rel(y, sla.cho_solve(o0.chol, x)) < 1e-10
    for l in range(1, c.L + 1):
        n = c.levels[l].mesh.n_dof
        x = rand_vec(n, 40 + l)
        y = D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, l, x, n)
        ref = vcycle(c.levels, l, x)
        assert rel(y, ref) < 1e-10, rel(y, ref)


@pytest.mark.parametrize("name", CASES)
def test_pcg_solution_and_iterations(name, request):
    c = request.getfixturevalue(name)
    tol = c.ok["tol"]
    x_ref, it_ref, hist = mg_pcg(c.levels, c.A, c.b, tol=tol)
    x, f, st, code = c.solver.solve()
    assert code == D.DPGMG_OK
    assert st.relres <= tol and st.true_relres <= 10 * tol
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(x, x_ref) < 1e-7
    f_ref = c.fs.fields(x_ref)
    assert rel(f.reshape(f_ref.shape), f_ref) < 1e-7


def test_manufactured_solution_exact_through_gpu():
    p = 3
    C = np.random.default_rng(3).standard_normal((4, p, p, p)) + 1j * np.random.default_rng(4).standard_normal((4, p, p, p))
    x0, x1 = (0.0, 0.0, 0.0), (1.0, 2.0, 1.0)
    c = np.random.default_rng(5).uniform(0.5, 2.0, 4 * 2 * 2)
    pk = dict(n=(4, 2, 2), p=p, omega=7.0, x0=x0, x1=x1, wavespeed=c, source="manufactured", mf_coeffs=C)
    from oracle.mesh import Mesh
    from oracle.problem import Manufactured
    ld = Manufactured(C, 7.0, x0, x1)
    m = Mesh((4, 2, 2), p, x0, x1)
    with D.Solver(pk, n_levels=2, p_min=2, tol=1e-13, max_iter=500) as s:
        x, f, st, code = s.solve()
    assert rel(x, trace_dofs(m, ld.p, ld.u)) < 1e-9
    fe = field_dofs(m, ld.p, ld.u)
    assert rel(f.reshape(fe.shape), fe) < 1e-9


def test_plane_wave_load_matches_oracle():
    pk = dict(n=(3, 2, 2), p=2, omega=4.0, source="plane_wave", wave_dir=(1.0, 2.0, 2.0))
    fs, A, b, _ = oracle_system(pk, {}, hierarchy=False)
    with D.Solver(pk, n_levels=1) as s:
        g = D.dpgmg_rhs(s.h, s.s, A.shape[0])
        assert rel(g, b) < TOL_FP64
        x, f, st, code = s.solve()
        assert code == D.DPGMG_OK and st.iters <= 2
    import scipy.sparse.linalg as spla
    assert rel(x, spla.spsolve(A.tocsc(), b)) < 1e-10


def test_mixed_precision_c1(c1):
    w = workloads.config1()
    ok = dict(w["opts"], precision="mixed")
    x_ref, it_ref, _ = mg_pcg(c1.levels, c1.A, c1.b, tol=ok["tol"])
    with D.Solver(w["problem"], **ok) as s:
        n = c1.A.shape[0]
        v = rand_vec(n, 9)
        y = D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, c1.L, v, n)
        assert rel(y, vcycle(c1.levels, c1.L, v)) < MIXED_VCYCLE_TOL
        x, f, st, code = s.solve()
    assert code == D.DPGMG_OK and st.true_relres <= 1e-8 * 10
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref)
    assert rel(x, x_ref) < 1e-7


def test_coarsest_none_matches_oracle():
    w = workloads.config1()
    ok = dict(w["opts"], coarsest="none")
    fs, A, b, levels = oracle_system(w["problem"], ok)
    _, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    with D.Solver(w["problem"], **ok) as s:
        x, f, st, code = s.solve()
    assert code == D.DPGMG_OK and abs(st.iters - it_ref) <= max(1, 0.1 * it_ref)


@pytest.mark.parametrize("n,expect", [(10, "cholesky"), (11, "none")])
def test_coarsest_auto_rule(n, expect):
    """AUTO takes the dense coarsest solve when level 0 holds at most 20,000
    DOFs (10^3 elements of order 2: 19,061) and none above (11^3: 25,356):
    it allocates exactly what the explicit choice allocates and gives its
    result (assembly sums with FP64 atomics, so equal to rounding)."""
    pk = dict(n=(n, n, n), p=3, omega=10.0, src_center=(0.4, 0.5, 0.6), src_width=0.15)
    ok = dict(n_levels=2, p_min=2, precision="mixed", tol=1e-8)
    out = {}
    for c in ("auto", expect):
        with D.Solver(pk, **dict(ok, coarsest=c)) as s:
            x, f, st, code = s.solve()
            nd0 = D.dpgmg_level_info(s.h, s.s, 0).n_dof
        assert code == D.DPGMG_OK
        out[c] = (x, st.iters, st.dev_bytes_peak)
    assert (nd0 <= 20000) == (expect == "cholesky")
    assert out["auto"][1] == out[expect][1]
    assert out["auto"][2] == out[expect][2]
    assert rel(out["auto"][0], out[expect][0]) < 1e-6


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_graph_replay_matches_eager(precision, tol):
    """CG steps replayed from the captured graph give the eager result with
    the same iteration count and the same number of kernel launches."""
    w = workloads.config1()
    out = {}
    for flags in (0, D.FLAG_EAGER):
        ok = dict(w["opts"], precision=precision, flags=flags)
        with D.Solver(w["problem"], **ok) as s:
            l0 = D.dpgmg_launch_count()
            x, f, st, code = s.solve()
            out[flags] = (x, st.iters, D.dpgmg_launch_count() - l0)
        assert code == D.DPGMG_OK
    assert out[0][1] == out[D.FLAG_EAGER][1]
    assert out[0][2] == out[D.FLAG_EAGER][2]
    assert rel(out[0][0], out[D.FLAG_EAGER][0]) < tol


@pytest.mark.parametrize("n", [4, 6])
def test_coarse_factor_on_tensor_cores(n):
    """Mixed path: the complex64 coarsest factor built by panels whose solves
    and updates are tensor-core (3xTF32) products solves level 0 within a
    small factor of the accuracy of the CUDA-core FP32 factor.  Level 0 has
    269 (n = 4) and 883 (n = 6) DOFs: 128-wide panels (3 and 7 of them) with
    ragged last panels, 64-row and 128-column product tiles with ragged
    edges, lower-triangle tiles that cross the diagonal.  The 3xTF32 products
    keep ~22 of FP32's 24 bits and accumulate in the tensor cores' FP32, so the
    bar is an order of magnitude (16x) of the CUDA-core factor's error; the
    end-to-end parity of the mixed path is checked by the solution tests."""
    import scipy.linalg as sla
    w = workloads.config1()
    pk = dict(w["problem"], n=(n, n, n))
    ok = dict(w["opts"], precision="mixed")
    _, _, _, levels = oracle_system(pk, ok)
    o0 = levels[0]
    x = rand_vec(o0.mesh.n_dof, 7)
    y_ref = sla.cho_solve(o0.chol, x)
    y = {}
    for flags in (D.FLAG_CUDA_CORES, 0):
        with D.Solver(pk, **dict(ok, flags=flags)) as s:
            y[flags] = D.dpgmg_apply(s.h, s.s, D.OP_COARSE, 0, x, o0.mesh.n_dof)
    e_cc, e_tc = rel(y[D.FLAG_CUDA_CORES], y_ref), rel(y[0], y_ref)
    print("coarse solve error: CUDA cores %.2e, tensor cores %.2e" % (e_cc, e_tc))
    assert e_cc < 1e-3 and e_tc < 1e-3, (e_tc, e_cc)
    assert e_tc < 16 * e_cc + 1e-6, (e_tc, e_cc)


@pytest.mark.parametrize("name", CASES)
def test_spmv_group_sizes(name, request):
    """Every SpMV work decomposition (G rows of one entity per warp) applies
    the same operator: level operators against the oracle's, and the CG
    operator against the oracle's assembled matrix."""
    c = request.getfixturevalue(name)
    s = c.solver
    tuned = [D.dpgmg_spmv_group(s.h, s.s, l) for l in range(1, c.L + 1)] + [D.dpgmg_spmv_group(s.h, s.s, -1)]
    assert all(g in (1, 2, 4, 8, 16, 32, 64) for g in tuned)
    try:
        for G in (1, 2, 4, 8, 16, 32):
            for l in range(1, c.L + 1):
                D.dpgmg_spmv_group(s.h, s.s, l, G)
                n = c.levels[l].mesh.n_dof
                x = rand_vec(n, 60 + l)
                y = D.dpgmg_apply(s.h, s.s, D.OP_A, l, x, n)
                assert rel(y, c.levels[l].M @ x) < TOL_FP64, (G, l)
            D.dpgmg_spmv_group(s.h, s.s, -1, G)
            n = c.A.shape[0]
            x = rand_vec(n, 77)
            y = D.dpgmg_apply(s.h, s.s, D.OP_AFULL, c.L, x, n)
            assert rel(y, c.A @ x) < TOL_FP64, G
    finally:
        for l, g in zip(list(range(1, c.L + 1)) + [-1], tuned):
            D.dpgmg_spmv_group(s.h, s.s, l, g)
    # one row per warp with and without the index prefetch, and with the
    # cp.async ring: the same arithmetic, bitwise
    for l in list(range(1, c.L + 1)) + [-1]:
        n = c.A.shape[0] if l == -1 else c.levels[l].mesh.n_dof
        op, lv = (D.OP_AFULL, c.L) if l == -1 else (D.OP_A, l)
        x = rand_vec(n, 80 + l)
        ys = []
        for G in (1, 16, 32):
            D.dpgmg_spmv_group(s.h, s.s, l, G)
            ys.append(D.dpgmg_apply(s.h, s.s, op, lv, x, n))
        D.dpgmg_spmv_group(s.h, s.s, l, tuned[l - 1] if l > 0 else tuned[-1])
        assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2]), l
    with pytest.raises(D.DpgmgError):
        D.dpgmg_spmv_group(s.h, s.s, 1, 3)
    with pytest.raises(D.DpgmgError):   # no half-warp form of the CG operator
        D.dpgmg_spmv_group(s.h, s.s, -1, 64)


def test_spmv_group_sizes_mixed(c1):
    """The complex64 V-cycle operators under every work decomposition."""
    with D.Solver(c1.pk, **dict(c1.ok, precision="mixed")) as s:
        for G in (1, 2, 4, 8, 16, 32, 64):
            for l in range(1, c1.L + 1):
                D.dpgmg_spmv_group(s.h, s.s, l, G)
                n = c1.levels[l].mesh.n_dof
                x = rand_vec(n, 90 + l)
                y = D.dpgmg_apply(s.h, s.s, D.OP_A, l, x, n)
                assert rel(y, c1.levels[l].M @ x) < 1e-6, (G, l)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-11)])
def test_stored_coarse_operators(precision, tol):
    """Stored coarse operators (assembled on each coarser mesh, Sec. 3) against
    the oracle: every coarse element matrix, then PCG iterations and solution."""
    pk = dict(n=(4, 4, 4), p=2, omega=4.0, src_center=(0.45, 0.5, 0.55), src_width=0.15)
    ok = dict(n_levels=3, p_min=1, precision=precision, tol=1e-8, flags=D.FLAG_STORE_COARSE)
    fs, A, b, levels = oracle_system(pk, ok)
    L = len(levels) - 1
    with D.Solver(pk, **ok) as s:
        for l in range(L):
            E = levels[l].E
            for e in range(0, E.shape[0], max(1, E.shape[0] // 7)):
                M = D.dpgmg_element_matrix(s.h, s.s, l, e, E.shape[1])
                assert rel(M, E[e]) < tol, (l, e, rel(M, E[e]))
        x, f, st, code = s.solve()
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    assert code == D.DPGMG_OK
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(x, x_ref) < 1e-7


def test_error_statuses():
    w = workloads.config1()
    h = D.dpgmg_create(0)
    try:
        pb, keep = D.make_problem(**w["problem"])
        op = D.make_opts(**w["opts"])
        pb.p = 0
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, op)
        assert e.value.code == D.DPGMG_ERR_ARG
        pb.p = 2
        pb.dp = 2
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, op)
        assert e.value.code == D.DPGMG_ERR_ARG
    finally:
        D.dpgmg_destroy(h)
    # budget far below the footprint: refused before any allocation
    h = D.dpgmg_create(0, mem_budget_bytes=1 << 20)
    try:
        pb, keep = D.make_problem(**w["problem"])
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_setup(h, pb, D.make_opts(**w["opts"]))
        assert e.value.code == D.DPGMG_ERR_NOMEM
    finally:
        D.dpgmg_destroy(h)
    # iteration cap: NOT_CONVERGED with outputs and stats written
    with D.Solver(w["problem"], **dict(w["opts"], max_iter=2)) as s:
        x, f, st, code = s.solve()
        assert code == D.DPGMG_ERR_NOT_CONVERGED and st.iters == 2 and np.linalg.norm(x) > 0


@pytest.mark.parametrize("nl,precision", [(2, "fp64"), (3, "fp64"), (3, "mixed")])
def test_smoothing_coarsest_matches_oracle(nl, precision):
    """DPGMG_COARSEST_SMOOTH: one damped additive Schwarz step on level 0 with
    the vertex patches of its own mesh.  Level 0's patches and theta, its
    smoother and the whole V-cycle against the oracle; PCG iterations and
    solution at the parity bar."""
    from oracle.hierarchy import smoother
    from tests.oracle_adapter import MIXED_THETA_TOL, MIXED_VCYCLE_TOL
    pk = dict(n=(4, 4, 4), p=2, omega=4.0, src_center=(0.4, 0.55, 0.5), src_width=0.2)
    ok = dict(n_levels=nl, p_min=1, precision=precision, tol=1e-8, coarsest="smooth")
    fs, A, b, levels = oracle_system(pk, ok)
    o0 = levels[0]
    L = len(levels) - 1
    with D.Solver(pk, **ok) as s:
        g0 = s.level(0)
        sizes = np.array([len(x) for x in o0.patches])
        assert g0.n_patches == len(sizes) and g0.patch_max == sizes.max()
        assert g0.sum_patch_sq == int(np.sum(sizes ** 2))
        th_tol = 1e-9 if precision == "fp64" else MIXED_THETA_TOL
        assert abs(g0.theta - o0.theta) < th_tol * o0.theta, (g0.theta, o0.theta)
        n0 = o0.mesh.n_dof
        x = rand_vec(n0, 3)
        y = D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, 0, x, n0)
        vtol = 1e-10 if precision == "fp64" else MIXED_VCYCLE_TOL
        assert rel(y, o0.theta * smoother(o0, x)) < vtol
        n = A.shape[0]
        v = rand_vec(n, 4)
        assert rel(D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, L, v, n), vcycle(levels, L, v)) < vtol
        xs, f, st, code = s.solve()
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    assert code == D.DPGMG_OK
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(xs, x_ref) < 1e-7


@pytest.mark.parametrize("n,nl,pmin,coarsest,precision", [
    ((4, 4, 4), 3, 1, "cholesky", "fp64"),
    ((4, 4, 4), 3, 1, "cholesky", "mixed"),
    ((4, 4, 4), 2, 1, "smooth", "fp64"),
    ((8, 8, 4), 4, 1, "cholesky", "fp64"),
])
def test_patch_rule_r2_matches_oracle(n, nl, pmin, coarsest, precision):
    """DPGMG_FLAG_PATCH_R2: every smoothed level's patch statistics, the
    smoother of every level and the V-cycle against the oracle built with rule
    R2; PCG iterations and solution at the parity bar."""
    from oracle.hierarchy import smoother
    from tests.oracle_adapter import MIXED_VCYCLE_TOL
    pk = dict(n=n, p=2, omega=4.0, src_center=(0.4, 0.55, 0.5), src_width=0.2)
    if n[2] == 4 and n[0] == 8:
        pk["wavespeed"] = np.repeat(np.random.default_rng(3).uniform(0.5, 1.0, 4), 64)
    ok = dict(n_levels=nl, p_min=pmin, precision=precision, tol=1e-8, coarsest=coarsest,
              flags=D.FLAG_PATCH_R2)
    fs, A, b, levels = oracle_system(pk, ok)
    L = len(levels) - 1
    vtol = 1e-10 if precision == "fp64" else MIXED_VCYCLE_TOL
    with D.Solver(pk, **ok) as s:
        for l in range(L + 1):
            o = levels[l]
            if not hasattr(o, "patches") or o.patches is None:
                continue
            g = s.level(l)
            sizes = np.array([len(x) for x in o.patches])
            assert g.n_patches == len(sizes) and g.patch_max == sizes.max()
            assert g.sum_patch_sq == int(np.sum(sizes ** 2))
            nl_ = o.mesh.n_dof
            x = rand_vec(nl_, 5 + l)
            y = D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, l, x, nl_)
            assert rel(y, o.theta * smoother(o, x)) < vtol
        nt = A.shape[0]
        v = rand_vec(nt, 4)
        assert rel(D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, L, v, nt), vcycle(levels, L, v)) < vtol
        xs, f, st, code = s.solve()
    x_ref, it_ref, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    assert code == D.DPGMG_OK
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(xs, x_ref) < 1e-7
