"""Pins of the oracle's DPG-MG hierarchy, smoother, V-cycle and PCG (no GPU).

* P5: p-level coarse operators are principal submatrices; the natural
  inclusion reproduces the traces of polynomials of the coarse space on the
  fine skeleton; macro condensation + back-substitution solves the fine
  system exactly; the element-wise restriction equals P^* M P globally.
* R1 patch statistics equal the independently counted workload figures.
* R2 patches equal the DOFs of the entities whose closure holds the vertex,
  enumerated from the mesh's entity indices; they coincide with R1 away from
  the boundary and the V-cycle built on them is Hermitian positive.
* P6: the V-cycle is Hermitian and positive definite.
* P4: MG-PCG agrees with a brute-force dense solve.
"""
import numpy as np
import pytest

from oracle.assembly import build_fine
from oracle.hierarchy import _patch_rule_R1, _patch_rule_R2, assemble, build_hierarchy, level_specs, smoother
from oracle.mesh import tangential
from oracle.mesh import Mesh
from oracle.problem import GaussianSource, Manufactured
from oracle.solver import mg_pcg, vcycle
from oracle.traces import trace_dofs


@pytest.fixture(scope="module")
def small_h():
    """4^3 p2 -> 2^3 p2 (one h-transition) on a non-cubic box, heterogeneous c."""
    c = np.random.default_rng(5).uniform(0.5, 1.5, 64)
    fs = build_fine((4, 4, 4), 2, 6.0, wavespeed=c, load=GaussianSource((0.3, 0.6, 0.5), 0.2),
                    x0=(0, 0, 0), x1=(1.0, 1.5, 1.0))
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=2, p_min=2)
    return fs, A, b, levels


@pytest.fixture(scope="module")
def small_ph():
    """4^3 p2 -> 4^3 p1 -> 2^3 p1 (p- then h-transition)."""
    fs = build_fine((4, 4, 4), 2, 4.0, load=GaussianSource((0.5, 0.5, 0.5), 0.1))
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=3, p_min=1)
    return fs, A, b, levels


def test_level_specs_of_the_workloads():
    assert level_specs((4, 4, 4), 2, 2, p_min=1) == ([((4, 4, 4), 2), ((4, 4, 4), 1)], ["p"])
    assert level_specs((16, 16, 16), 3, 3)[0] == [((16,) * 3, 3), ((16,) * 3, 2), ((8,) * 3, 2)]
    assert level_specs((32, 32, 16), 3, 4)[0] == [((32, 32, 16), 3), ((32, 32, 16), 2),
                                                 ((16, 16, 8), 2), ((8, 8, 4), 2)]
    assert level_specs((9, 9, 9), 3, 4)[0] == [((9,) * 3, 3), ((9,) * 3, 2)]


def test_p_level_coarse_operator_is_principal_submatrix(small_ph):
    fs, A, b, levels = small_ph
    top, mid = levels[2], levels[1]
    Ac = assemble(mid.E, mid.dofs, mid.mesh.n_dof).toarray()
    assert np.allclose(Ac, A.toarray()[np.ix_(top.inj, top.inj)], rtol=0, atol=1e-15 * abs(Ac).max())


def test_inclusion_reproduces_coarse_traces(small_h):
    fs, A, b, levels = small_h
    fine, coarse = levels[1], levels[0]
    rng = np.random.default_rng(2)
    Cp = rng.standard_normal((3, 3, 3)) + 1j * rng.standard_normal((3, 3, 3))   # degree 2 = p
    Cu = rng.standard_normal((3, 2, 2, 2)) + 1j * rng.standard_normal((3, 2, 2, 2))  # degree 1 = p-1

    def pf(X):
        return np.einsum("cba,na,nb,nc->n", Cp, X[:, :1] ** np.arange(3), X[:, 1:2] ** np.arange(3),
                         X[:, 2:3] ** np.arange(3))

    def uf(X):
        return np.stack([np.einsum("cba,na,nb,nc->n", Cu[d], X[:, :1] ** np.arange(2),
                                   X[:, 1:2] ** np.arange(2), X[:, 2:3] ** np.arange(2))
                         for d in range(3)], axis=1)

    xc = trace_dofs(coarse.mesh, pf, uf)
    xf = trace_dofs(fine.mesh, pf, uf)
    Ix = fine.P @ xc
    sm = fine.smask
    assert np.linalg.norm(Ix[sm] - xf[sm]) / np.linalg.norm(xf[sm]) < 1e-12
    assert np.all(Ix[~sm] == 0)


def test_macro_condensation_is_exact_block_elimination(small_h):
    fs, A, b, levels = small_h
    lev = levels[1]
    Ad = A.toarray()
    x_ref = np.linalg.solve(Ad, b)
    # condense the load, solve the macro system, back-substitute
    bs = np.where(lev.smask, b, 0)
    for Sg, Ig, T in zip(lev.S, lev.I, lev.T):
        bs[Sg] -= T @ b[Ig]
    sm = np.nonzero(lev.smask)[0]
    x = np.zeros_like(b)
    x[sm] = np.linalg.solve(lev.M.toarray()[np.ix_(sm, sm)], bs[sm])
    for Sg, Ig, T, Ai in zip(lev.S, lev.I, lev.T, lev.Aii_inv):
        x[Ig] = Ai @ b[Ig] - T.conj().T @ x[Sg]
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-12


def test_restriction_equals_galerkin_product(small_h):
    fs, A, b, levels = small_h
    fine, coarse = levels[1], levels[0]
    Ac = assemble(coarse.E, coarse.dofs, coarse.mesh.n_dof).toarray()
    PMP = (fine.P.conj().T @ fine.M @ fine.P).toarray()
    assert np.linalg.norm(Ac - PMP) / np.linalg.norm(PMP) < 1e-13
    assert np.linalg.eigvalsh(Ac).min() > 0


def _patch_stats(n, p, kind):
    m = Mesh(n, p)
    tab = m.dof_table()
    if kind == "p":
        cm, smask = m, np.ones(m.n_dof, dtype=bool)
    else:
        cm = Mesh(tuple(v // 2 for v in n), p)
        # fine DOFs on the coarse skeleton: a flat coordinate on a coarse plane
        smask = np.array([any(c % 4 == 0 for c in ctr) for (_, ctr, _) in tab])
    pt = _patch_rule_R1(m, cm, tab, kind, smask)
    sizes = np.array([len(x) for x in pt])
    covered = np.zeros(m.n_dof, dtype=bool)
    for x in pt:
        covered[x] = True
    assert np.all(covered == smask)
    return len(pt), sizes.max(), round(sizes.mean(), 1), int(np.sum(sizes ** 2)), int(smask.sum())


def test_patch_statistics_small():
    assert _patch_stats((4, 4, 4), 2, "p")[:4] == (125, 104, 41.3, 312089)


@pytest.mark.slow
def test_patch_statistics_workloads():
    assert _patch_stats((16, 16, 16), 3, "p")[:4] == (4913, 260, 147.4, 118947107)
    assert _patch_stats((16, 16, 16), 2, "h") == (729, 488, 248.0, 54691605, 43617)


def test_interior_patch_sizes():
    # interior vertex patch: vertex + 6 edges + 12 faces (p level); the
    # macro version collects the fine DOFs on those coarse entities (h level)
    for p, expect_p, expect_h in [(2, 67, 319), (3, 169, 763)]:
        m = Mesh((4, 4, 4), p)
        tab = m.dof_table()
        pt = _patch_rule_R1(m, m, tab, "p", np.ones(m.n_dof, dtype=bool))
        assert len(pt[2 + 5 * (2 + 5 * 2)]) == expect_p
        m8 = Mesh((8, 8, 8), p)
        tab8 = m8.dof_table()
        sm = np.array([any(c % 4 == 0 for c in ctr) for (_, ctr, _) in tab8])
        pt8 = _patch_rule_R1(m8, Mesh((4, 4, 4), p), tab8, "h", sm)
        assert len(pt8[2 + 5 * (2 + 5 * 2)]) == expect_h


@pytest.mark.parametrize("fx", ["small_h", "small_ph"])
def test_vcycle_hermitian_positive(fx, request):
    fs, A, b, levels = request.getfixturevalue(fx)
    L = len(levels) - 1
    rng = np.random.default_rng(7)
    N = A.shape[0]
    for _ in range(3):
        u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        Bu, Bv = vcycle(levels, L, u), vcycle(levels, L, v)
        assert abs(np.vdot(v, Bu) - np.vdot(Bv, u)) / (np.linalg.norm(u) * np.linalg.norm(Bv)) < 1e-12
        val = np.vdot(u, Bu)
        assert val.real > 0 and abs(val.imag) < 1e-10 * val.real


def test_theta_from_power_iteration(small_ph):
    fs, A, b, levels = small_ph
    for lev in levels[1:]:
        sm = np.nonzero(lev.smask)[0]
        Md = lev.M.toarray()[np.ix_(sm, sm)]
        N = lev.M.shape[0]
        SM = np.zeros((len(sm), len(sm)), dtype=np.complex128)
        for k, j in enumerate(sm):
            e = np.zeros(N, dtype=np.complex128)
            e[j] = 1
            SM[:, k] = smoother(lev, lev.M @ e)[sm]
        lam = np.max(np.linalg.eigvals(SM).real)
        est = 1.0 / (1.05 * lev.theta)
        assert est <= lam * (1 + 1e-10) and est >= 0.95 * lam


@pytest.mark.parametrize("p,nl,pmin", [(2, 2, 1), (3, 3, 2), (2, 3, 1)])
def test_pcg_matches_dense_solve(p, nl, pmin):
    fs = build_fine((2, 2, 2), p, 3.0, load=GaussianSource((0.4, 0.45, 0.6), 0.15))
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=nl, p_min=pmin)
    x, it, hist = mg_pcg(levels, A, b, tol=1e-12)
    x_ref = np.linalg.solve(A.toarray(), b)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9


def test_pcg_reaches_manufactured_solution(small_ph):
    # MG-PCG to 1e-10 recovers the manufactured traces (end to end through the V-cycle)
    fs0, _, _, levels = small_ph
    ld = Manufactured(np.random.default_rng(4).standard_normal((4, 2, 2, 2)) + 0.5j, 4.0)
    fs = build_fine((4, 4, 4), 2, 4.0, load=ld)
    A, b = fs.assemble()
    lv = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=3, p_min=1)
    x, it, hist = mg_pcg(lv, A, b, tol=1e-10)
    xt = trace_dofs(fs.mesh, ld.p, ld.u)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) < 1e-8


@pytest.fixture(scope="module")
def stored_ph():
    """4^3 p2 -> 4^3 p1 -> 2^3 p1 with stored coarse operators (assembled on each coarser mesh)."""
    ld = GaussianSource((0.5, 0.5, 0.5), 0.1)
    fs = build_fine((4, 4, 4), 2, 4.0, load=ld)
    A, b = fs.assemble()

    def stored(cmesh):
        return build_fine(cmesh.n, cmesh.p, 4.0, load=ld, x0=cmesh.x0, x1=cmesh.x1).Kc
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=3, p_min=1, stored=stored)
    return fs, A, b, levels


def test_stored_coarse_operators_are_the_coarse_dpg_systems(stored_ph, small_ph):
    # each coarser level's operator is the DPG system of its own mesh and order,
    # which differs from the restriction of the finer operator
    fs, A, b, levels = stored_ph
    _, _, _, restricted = small_ph
    for l in range(len(levels) - 1):
        m = levels[l].mesh
        direct = build_fine(m.n, m.p, 4.0, load=GaussianSource((0.5, 0.5, 0.5), 0.1)).assemble()[0]
        Al = assemble(levels[l].E, levels[l].dofs, m.n_dof)
        assert abs(Al - direct).max() <= 1e-13 * abs(direct).max()
        Ar = assemble(restricted[l].E, restricted[l].dofs, m.n_dof)
        assert abs(Al - Ar).max() > 1e-3 * abs(Ar).max()


def test_stored_vcycle_hermitian_positive_and_same_solution(stored_ph, small_ph):
    fs, A, b, levels = stored_ph
    L = len(levels) - 1
    rng = np.random.default_rng(11)
    u = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    Bu, Bv = vcycle(levels, L, u), vcycle(levels, L, v)
    assert abs(np.vdot(v, Bu) - np.vdot(Bv, u)) / (np.linalg.norm(u) * np.linalg.norm(Bv)) < 1e-12
    assert np.vdot(u, Bu).real > 0
    # the preconditioner changes the iteration, not the discrete solution
    x_s, it_s, _ = mg_pcg(levels, A, b, tol=1e-12)
    x_r, it_r, _ = mg_pcg(small_ph[3], A, b, tol=1e-12)
    assert np.linalg.norm(x_s - x_r) <= 1e-9 * np.linalg.norm(x_r)


@pytest.mark.parametrize("nl,pmin", [(2, 1), (3, 1)])
def test_smoothing_coarsest_mode(nl, pmin):
    """Coarsest mode "smooth" (one damped additive Schwarz step on level 0 with
    the vertex patches of its own mesh): the V-cycle stays Hermitian positive,
    theta_0 is within 5% below the largest eigenvalue of S_0 A_0 (dense), and
    PCG reaches the dense solve."""
    fs = build_fine((4, 4, 4), 2, 4.0, load=GaussianSource((0.4, 0.55, 0.5), 0.2))
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=nl, p_min=pmin, coarsest="smooth")
    c0 = levels[0]
    assert c0.coarsest == "smooth" and len(c0.patches) == int(np.prod(np.asarray(c0.mesh.n) + 1))
    N0 = c0.A.shape[0]
    SA = np.zeros((N0, N0), dtype=np.complex128)
    for j in range(N0):
        e = np.zeros(N0, dtype=np.complex128)
        e[j] = 1
        SA[:, j] = smoother(c0, c0.A @ e)
    lam = np.max(np.linalg.eigvals(SA).real)
    est = 1.0 / (1.05 * c0.theta)
    assert est <= lam * (1 + 1e-10) and est >= 0.95 * lam
    L = len(levels) - 1
    rng = np.random.default_rng(8)
    u = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    Bu, Bv = vcycle(levels, L, u), vcycle(levels, L, v)
    assert abs(np.vdot(v, Bu) - np.vdot(Bv, u)) / (np.linalg.norm(u) * np.linalg.norm(Bv)) < 1e-12
    assert np.vdot(u, Bu).real > 0
    x, it, hist = mg_pcg(levels, A, b, tol=1e-12)
    x_ref = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9


def _closure_patch_by_entities(m, w):
    """DOFs of the entities of a p-level mesh whose closure contains vertex w,
    enumerated from the entity index functions (vertex, the edges ending at w,
    the faces with w as a corner)."""
    p, n = m.p, m.n
    out = [m.vertex(w)]
    for d in range(3):
        for off in (0, 1):
            c = list(w)
            c[d] -= off
            if 0 <= c[d] < n[d]:
                e = m.edge(d, c)
                out += [m.off_E + e * (p - 1) + k for k in range(p - 1)]
        t1, t2 = tangential(d)
        for a in (0, 1):
            for b in (0, 1):
                c = list(w)
                c[t1] -= a
                c[t2] -= b
                if 0 <= c[t1] < n[t1] and 0 <= c[t2] < n[t2]:
                    f = m.face(d, c)
                    out += [m.off_F + f * (p - 1) ** 2 + k for k in range((p - 1) ** 2)]
                    if not m.is_boundary_face(d, c):
                        u = m.iface(d, c)
                        out += [m.off_U + u * p * p + k for k in range(p * p)]
    return sorted(out)


@pytest.mark.parametrize("n,p", [((3, 2, 2), 2), ((2, 2, 3), 3)])
def test_patch_rule_R2_is_the_vertex_closure(n, p):
    m = Mesh(n, p)
    tab = m.dof_table()
    pt = _patch_rule_R2(m, m, tab, "p", np.ones(m.n_dof, dtype=bool))
    j = 0
    for k in range(n[2] + 1):
        for jj in range(n[1] + 1):
            for i in range(n[0] + 1):
                assert list(pt[j]) == _closure_patch_by_entities(m, (i, jj, k))
                j += 1
    # corner: the vertex, 3 edges and 3 boundary faces (no flux DOFs)
    assert len(pt[0]) == 1 + 3 * (p - 1) + 3 * (p - 1) ** 2


@pytest.mark.parametrize("kind", ["p", "h"])
def test_patch_rule_R2_against_R1(kind):
    # R2 <= R1 everywhere; what R1 adds are DOFs on boundary entities, which it
    # also gives to the vertices one layer inside (their one adjacent element
    # has those vertices as corners); R2 still covers the smoothed DOFs
    p = 2
    if kind == "p":
        m = Mesh((4, 4, 4), p)
        cm, sm = m, np.ones(m.n_dof, dtype=bool)
    else:
        m = Mesh((8, 8, 8), p)
        cm = Mesh((4, 4, 4), p)
        sm = np.array([any(c % 4 == 0 for c in ctr) for (_, ctr, _) in m.dof_table()])
    tab = m.dof_table()
    r1 = _patch_rule_R1(m, cm, tab, kind, sm)
    r2 = _patch_rule_R2(m, cm, tab, kind, sm)
    covered = np.zeros(m.n_dof, dtype=bool)
    j = 0
    for k in range(5):
        for jj in range(5):
            for i in range(5):
                a, b = set(r1[j].tolist()), set(r2[j].tolist())
                assert b <= a
                assert all(any(c in (0, 2 * m.n[d]) for d, c in enumerate(tab[g][1])) for g in a - b)
                assert (a == b) == all(v not in (1, 3) for v in (i, jj, k))
                covered[r2[j]] = True
                j += 1
    assert np.all(covered == sm)
    if kind == "p":
        # largest R2 patch is the interior one (67 at p2; R1 reaches 104 at the boundary)
        assert max(len(x) for x in r2) == 67 and max(len(x) for x in r1) == 104


def test_patch_rule_R2_vcycle_and_solution():
    fs = build_fine((4, 4, 4), 2, 4.0, load=GaussianSource((0.35, 0.5, 0.6), 0.15))
    A, b = fs.assemble()
    lv2 = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, n_levels=3, p_min=1, patch_rule="R2")
    L = len(lv2) - 1
    rng = np.random.default_rng(9)
    u = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    v = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    Bu, Bv = vcycle(lv2, L, u), vcycle(lv2, L, v)
    assert abs(np.vdot(v, Bu) - np.vdot(Bv, u)) / (np.linalg.norm(u) * np.linalg.norm(Bv)) < 1e-12
    assert np.vdot(u, Bu).real > 0
    x, it, hist = mg_pcg(lv2, A, b, tol=1e-12)
    x_ref = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
