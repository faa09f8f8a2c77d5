"""GPU parity at the orders and hierarchy shapes of the batched, served and
layered-medium workloads, against the FP64 oracle, through the C ABI.

* p = 4: 4x2x2 p4 -> p3 -> 2x1x1 p3 (a p-transition from order 4 and an
  h-transition at order 3, i.e. macro elements of order 3), wavespeed varying
  per element;
* p = 5: 3x2x2 p5 -> p4 -> p3 (element test spaces of 1,099 functions, vertex
  patches of order 5);
* the layered-medium shape: 8x8x4 p3 -> p2 -> 4x4x2 -> 2x2x1, one seeded
  wavespeed per element layer (contrast up to 10), two stacked
  h-transitions (Sec. 3 hierarchy; Sec. 5 layered medium).

FP64 path: every operator at 1e-11 relative (different but exact evaluations
of the same integrals), the solution at the parity bar of 1e-7 relative L2
with the iteration count within 10%.  Mixed path: the V-cycle and theta
within 1e-4 (complex64 storage and FP32 patch factorisations and macro
condensations, see tests/oracle_adapter.py), solution and iterations at the
same bar.
"""
import numpy as np
import pytest

from oracle.hierarchy import smoother
from oracle.solver import mg_pcg, vcycle
from paper_2304_01728_gb300 import dpgmg as D
from paper_2304_01728_gb300 import workloads
from tests.oracle_adapter import MIXED_THETA_TOL, MIXED_VCYCLE_TOL, oracle_system, rand_vec, rel

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def _cases():
    c4 = np.random.default_rng(12).uniform(0.7, 1.3, 16)
    w3 = workloads.config3_small("fp64")
    return {
        "p4": (dict(n=(4, 2, 2), p=4, omega=6.0, wavespeed=c4, src_center=(0.45, 0.5, 0.55), src_width=0.2,
                    x0=(0, 0, 0), x1=(2.0, 1.0, 1.0)),
               dict(n_levels=3, p_min=3, precision="fp64", tol=1e-10)),
        "p5": (dict(n=(3, 2, 2), p=5, omega=5.0, src_center=(0.5, 0.4, 0.6), src_width=0.25,
                    x0=(0, 0, 0), x1=(1.5, 1.0, 1.0)),
               dict(n_levels=3, p_min=3, precision="fp64", tol=1e-10)),
        "layered": (w3["problem"], dict(w3["opts"], tol=1e-10)),
    }


CASES = ["p4", "p5", "layered"]


class Case:
    def __init__(self, name):
        self.pk, self.ok = _cases()[name]
        self.fs, self.A, self.b, self.levels = oracle_system(self.pk, self.ok, parallel=True)
        self.L = len(self.levels) - 1
        self.solver = D.Solver(self.pk, **self.ok)


@pytest.fixture(scope="module")
def cases():
    made = {}
    yield lambda name: made[name] if name in made else made.setdefault(name, Case(name))
    for c in made.values():
        c.solver.close()


def _sample(n, k=12):
    return range(n) if n <= k else np.unique(np.linspace(0, n - 1, k).astype(int))


@pytest.mark.parametrize("name", CASES)
def test_structure(name, cases):
    c = cases(name)
    assert c.L == len(c.levels) - 1
    for l in range(0, c.L + 1):
        g, o = c.solver.level(l), c.levels[l]
        assert tuple(g.n) == tuple(o.mesh.n) and g.p == o.mesh.p and g.n_dof == o.mesh.n_dof
        if l == 0:
            continue
        assert g.kind == {"p": 1, "h": 2}[o.kind]
        sizes = np.array([len(x) for x in o.patches])
        assert g.n_patches == len(sizes) and g.patch_max == sizes.max()
        assert g.sum_patch_sq == int(np.sum(sizes ** 2))
        assert g.n_smooth == int(o.smask.sum())
        assert abs(g.theta - o.theta) < 1e-9 * o.theta, (l, g.theta, o.theta)
    if name == "layered":
        assert [lv.kind for lv in c.levels[1:]] == ["h", "h", "p"]


@pytest.mark.parametrize("name", CASES)
def test_element_matrices_and_loads(name, cases):
    c = cases(name)
    s = c.solver
    for l in range(c.L + 1):
        E = c.levels[l].E
        for e in _sample(E.shape[0]):
            M = D.dpgmg_element_matrix(s.h, s.s, l, int(e), E.shape[1])
            assert rel(M, E[e]) < TOL_FP64, (l, e, rel(M, E[e]))
    nloc = c.fs.Kc.shape[1]
    for e in _sample(c.fs.mesh.n_elem, 24):
        _, F = D.dpgmg_element_matrix(s.h, s.s, c.L, int(e), nloc, with_load=True)
        assert rel(F, c.fs.Fc[e]) < TOL_FP64, (e, rel(F, c.fs.Fc[e]))


@pytest.mark.parametrize("name", CASES)
def test_rhs_operators_transfers(name, cases):
    c = cases(name)
    s = c.solver
    b = D.dpgmg_rhs(s.h, s.s, c.A.shape[0])
    assert rel(b, c.b) < TOL_FP64
    x = rand_vec(c.A.shape[0], 1)
    assert rel(D.dpgmg_apply(s.h, s.s, D.OP_AFULL, c.L, x, c.A.shape[0]), c.A @ x) < TOL_FP64
    for l in range(1, c.L + 1):
        o, oc = c.levels[l], c.levels[l - 1]
        nf, nc = o.mesh.n_dof, oc.mesh.n_dof
        x = rand_vec(nf, 10 + l)
        assert rel(D.dpgmg_apply(s.h, s.s, D.OP_A, l, x, nf), o.M @ x) < TOL_FP64, l
        assert rel(D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, l, x, nf), o.theta * smoother(o, x)) < TOL_FP64, l
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
            assert rel(y, ref) < TOL_FP64, l


@pytest.mark.parametrize("name", CASES)
def test_coarse_solve_vcycle_and_pcg(name, cases):
    import scipy.linalg as sla
    c = cases(name)
    s = c.solver
    o0 = c.levels[0]
    x = rand_vec(o0.mesh.n_dof, 5)
    assert rel(D.dpgmg_apply(s.h, s.s, D.OP_COARSE, 0, x, o0.mesh.n_dof), sla.cho_solve(o0.chol, x)) < 1e-10
    for l in range(1, c.L + 1):
        n = c.levels[l].mesh.n_dof
        x = rand_vec(n, 40 + l)
        y = D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, l, x, n)
        assert rel(y, vcycle(c.levels, l, x)) < 1e-10, (l, rel(y, vcycle(c.levels, l, x)))
    tol = c.ok["tol"]
    x_ref, it_ref, _ = mg_pcg(c.levels, c.A, c.b, tol=tol)
    x, f, st, code = s.solve()
    print("%s fp64: iterations %d (oracle %d), solution error %.2e" % (name, st.iters, it_ref, rel(x, x_ref)))
    assert code == D.DPGMG_OK
    assert st.relres <= tol and st.true_relres <= 10 * tol
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(x, x_ref) < 1e-7
    f_ref = c.fs.fields(x_ref)
    assert rel(f.reshape(f_ref.shape), f_ref) < 1e-7


@pytest.mark.parametrize("name", CASES)
def test_mixed_path(name, cases):
    c = cases(name)
    ok = dict(c.ok, precision="mixed", tol=1e-8)
    x_ref, it_ref, _ = mg_pcg(c.levels, c.A, c.b, tol=ok["tol"])
    with D.Solver(c.pk, **ok) as s:
        ev, et = [], []
        for l in range(1, c.L + 1):
            n = c.levels[l].mesh.n_dof
            v = rand_vec(n, 50 + l)
            y = D.dpgmg_apply(s.h, s.s, D.OP_VCYCLE, l, v, n)
            ev.append(rel(y, vcycle(c.levels, l, v)))
            et.append(abs(s.level(l).theta - c.levels[l].theta) / c.levels[l].theta)
        x, f, st, code = s.solve()
    print("%s mixed: V-cycle error per level %s, theta error %s, iterations %d (oracle %d), solution error %.2e"
          % (name, ["%.1e" % v for v in ev], ["%.1e" % v for v in et], st.iters, it_ref, rel(x, x_ref)))
    assert max(ev) < MIXED_VCYCLE_TOL and max(et) < MIXED_THETA_TOL
    assert code == D.DPGMG_OK and st.true_relres <= 10 * ok["tol"]
    assert abs(st.iters - it_ref) <= max(1, 0.1 * it_ref), (st.iters, it_ref)
    assert rel(x, x_ref) < 1e-7
