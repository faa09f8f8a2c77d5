"""Pins of the oracle's element DPG work and fine system (no GPU).

* P1: a manufactured solution in the discrete trial space is reproduced to
  rounding (forms, signs, traces, impedance BC, load, condensation, recovery).
* P2: plane-wave field errors decay at the rate p under h-refinement and
  quickly under p-refinement.
* P3: condensed element matrices and the assembled system are Hermitian
  positive definite.
"""
import numpy as np
import pytest

from oracle.assembly import build_fine
from oracle.element import (boundary_faces, condense, dpg_element, element_matrices,
                            present_columns)
from oracle.mesh import Mesh
from oracle.problem import GaussianSource, Manufactured, PlaneWave, WithImpedanceLoad
from oracle.traces import field_dofs, trace_dofs


def _rand_coeffs(p, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, p, p, p)) + 1j * rng.standard_normal((4, p, p, p))


@pytest.mark.parametrize("p,n,omega", [(1, (2, 2, 3), 5.0), (2, (2, 3, 2), 2.0), (3, (2, 1, 2), 7.0)])
def test_manufactured_solution_is_exact(p, n, omega):
    x0, x1 = (0.0, -1.0, 0.5), (2.0, 1.0, 2.0)
    ld = Manufactured(_rand_coeffs(p, 10 + p), omega, x0, x1)
    c = np.random.default_rng(p).uniform(0.3, 2.0, int(np.prod(n)))
    fs = build_fine(n, p, omega, wavespeed=c, load=ld, x0=x0, x1=x1)
    A, b = fs.assemble()
    x = np.linalg.solve(A.toarray(), b)
    xt = trace_dofs(fs.mesh, ld.p, ld.u)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) < 1e-10
    F = fs.fields(x)
    Fe = field_dofs(fs.mesh, ld.p, ld.u)
    assert np.linalg.norm(F - Fe) / np.linalg.norm(Fe) < 1e-10


class _VolumeOnly:
    """f and g of a load, without its impedance data."""

    def __init__(self, ld):
        self.f, self.g, self.u0 = ld.f, ld.g, None


@pytest.mark.parametrize("p,n", [(2, (2, 3, 2)), (3, (2, 1, 2))])
def test_impedance_data_given_separately(p, n):
    # the manufactured solution with its u0 handed over as separate impedance
    # data (WithImpedanceLoad) is still reproduced exactly; with that data
    # left out it is not
    x0, x1 = (0.0, -1.0, 0.5), (2.0, 1.0, 2.0)
    omega = 4.0
    ld = Manufactured(_rand_coeffs(p, 20 + p), omega, x0, x1)
    c = np.random.default_rng(3 + p).uniform(0.3, 2.0, int(np.prod(n)))
    xt = None
    errs = []
    for load in (WithImpedanceLoad(_VolumeOnly(ld), ld.u0), _VolumeOnly(ld)):
        fs = build_fine(n, p, omega, wavespeed=c, load=load, x0=x0, x1=x1)
        A, b = fs.assemble()
        x = np.linalg.solve(A.toarray(), b)
        xt = trace_dofs(fs.mesh, ld.p, ld.u)
        errs.append(np.linalg.norm(x - xt) / np.linalg.norm(xt))
    assert errs[0] < 1e-10 and errs[1] > 1e-3


def test_manufactured_detects_wrong_order_data():
    # a solution one order too rich is NOT reproduced: the pin has teeth
    p = 2
    ld = Manufactured(np.random.default_rng(1).standard_normal((4, 3, 3, 3)) + 0j, 3.0)
    fs = build_fine((2, 2, 2), p, 3.0, load=ld)
    A, b = fs.assemble()
    x = np.linalg.solve(A.toarray(), b)
    F = fs.fields(x)
    Fe = field_dofs(fs.mesh, ld.p, ld.u)
    assert np.linalg.norm(F - Fe) / np.linalg.norm(Fe) > 1e-4


def _plane_wave_error(n, p, omega):
    """L2 error of the DPG fields (p, u) against the exact plane wave.

    ||U - U_h||^2 = ||U - PU||^2 + ||PU - U_h||^2 (P the element-wise L2
    projection onto the trial space; U_h - PU is orthogonal to U - PU), and
    ||U - PU||^2 = ||U||^2 - ||PU||^2.
    """
    from oracle.basis import gauss01
    import scipy.sparse.linalg as spla
    pw = PlaneWave((1.0, 2.0, 2.0), omega)
    fs = build_fine((n, n, n), p, omega, load=pw)
    A, b = fs.assemble()
    x = spla.spsolve(A.tocsc(), b)
    F = fs.fields(x)
    mesh = fs.mesh
    Fe = field_dofs(mesh, pw.p, pw.u)
    wts = []
    for comp in range(4):
        for c in range(p):
            for bb in range(p):
                for a in range(p):
                    wts.append(1.0 / ((2 * a + 1) * (2 * bb + 1) * (2 * c + 1)))
    wts = np.array(wts) * np.prod(mesh.h)
    disc2 = np.sum(np.abs(F - Fe) ** 2 * wts)
    proj2 = np.sum(np.abs(Fe) ** 2 * wts)
    xq, wq = gauss01(12)
    X = np.array([(xq[i], xq[j], xq[k]) for k in range(12) for j in range(12) for i in range(12)])
    W = np.array([wq[i] * wq[j] * wq[k] for k in range(12) for j in range(12) for i in range(12)])
    full2 = 0.0
    for e in range(mesh.n_elem):
        Xp = mesh.x0 + np.asarray(mesh.elem_coord(e)) * mesh.h + X * mesh.h
        full2 += np.prod(mesh.h) * np.sum(W * (np.abs(pw.p(Xp)) ** 2 + np.sum(np.abs(pw.u(Xp)) ** 2, axis=1)))
    return np.sqrt(full2 - proj2 + disc2)


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_plane_wave_h_convergence_rate(p):
    errs = [_plane_wave_error(n, p, 4.0) for n in (2, 4, 8)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # ultraweak DPG is quasi-optimal for the L2 fields: rate p
    assert abs(rates[-1] - p) < 0.3, rates


def test_plane_wave_p_convergence():
    errs = [_plane_wave_error(2, p, 4.0) for p in (1, 2, 3)]
    assert errs[1] < 0.3 * errs[0] and errs[2] < 0.3 * errs[1], errs


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("bf", [[False] * 6, [True, False, False, True, True, False]])
def test_condensed_element_is_hpd(p, bf):
    h = np.array([0.1, 0.07, 0.12])
    K, F = dpg_element(p, h, np.zeros(3), 0.7, 9.0, bf, GaussianSource((0.05, 0.03, 0.06), 0.05))
    keep = present_columns(p, bf)
    Kk = K[np.ix_(keep, keep)]
    assert np.linalg.norm(Kk - Kk.conj().T) / np.linalg.norm(Kk) < 1e-13
    assert np.linalg.eigvalsh(0.5 * (Kk + Kk.conj().T)).min() > 0
    Kc, Fc = condense(p, K, F, bf)
    nz = np.nonzero(np.abs(np.diag(Kc)) > 0)[0]
    Kcc = Kc[np.ix_(nz, nz)]
    assert np.linalg.norm(Kcc - Kcc.conj().T) / np.linalg.norm(Kcc) < 1e-13
    assert np.linalg.eigvalsh(0.5 * (Kcc + Kcc.conj().T)).min() > 0
    # absent unknowns (u-hat on Gamma) have empty rows and columns
    assert len(nz) == Kc.shape[0] - sum(bf) * p * p


def test_gram_closed_form_entries():
    # G for q = L0 L0 L0 (constant): ||i w c^-2 q||^2 + ||q||^2 = (w^2/c^4 + 1) |K|
    p, h, c, w = 2, np.array([0.3, 0.2, 0.5]), 0.8, 6.0
    G, B, l = element_matrices(p, h, np.zeros(3), c, w, [False] * 6)
    vol = np.prod(h)
    assert abs(G[0, 0] - (w ** 2 / c ** 4 + 1) * vol) < 1e-13 * abs(G[0, 0])
    assert np.linalg.norm(G - G.conj().T) < 1e-13 * np.linalg.norm(G)
    assert np.linalg.eigvalsh(G).min() > 0
    # b(p = const, q = const) = i w c^-2 |K| (the only volume term that survives)
    assert abs(B[0, 0] - 1j * w / c ** 2 * vol) < 1e-13


def test_global_system_hpd_and_test_basis_invariance():
    fs = build_fine((2, 2, 2), 2, 5.0, load=GaussianSource((0.4, 0.5, 0.6), 0.2))
    A, b = fs.assemble()
    Ad = A.toarray()
    assert np.linalg.norm(Ad - Ad.conj().T) / np.linalg.norm(Ad) < 1e-13
    assert np.linalg.eigvalsh(Ad).min() > 0
    # K = B^* G^{-1} B does not depend on the test basis: transform it
    bf = boundary_faces(fs.mesh, 0)
    G, B, l = element_matrices(2, fs.mesh.h, np.zeros(3), 1.0, 5.0, bf)
    T = np.random.default_rng(0).standard_normal(G.shape) + np.eye(G.shape[0]) * 10
    keep = present_columns(2, bf)
    K1 = B[:, keep].conj().T @ np.linalg.solve(G, B[:, keep])
    G2, B2 = T.conj().T @ G @ T, T.conj().T @ B
    K2 = B2[:, keep].conj().T @ np.linalg.solve(G2, B2[:, keep])
    assert np.linalg.norm(K1 - K2) / np.linalg.norm(K1) < 1e-10


def test_condensed_matrix_depends_only_on_impedance_faces_and_wavespeed():
    # the premise of computing each element class once (Sec. 2: on a uniform
    # mesh G, B and K depend on h, omega, c and the impedance faces only; the
    # load depends on the position): two interior elements and two elements
    # with the same boundary face set give equal condensed matrices and
    # different condensed loads; another face set or wavespeed gives another matrix
    p, om = 2, 6.0
    m = Mesh((5, 5, 5), p)
    ld = GaussianSource((0.35, 0.5, 0.6), 0.2)

    def cond(e, c=1.0):
        bf = boundary_faces(m, e)
        corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
        K, F = dpg_element(p, m.h, corner, c, om, bf, ld)
        return condense(p, K, F, bf)

    idx = lambda i, j, k: i + 5 * (j + 5 * k)
    pairs = [(idx(1, 1, 1), idx(3, 2, 3)),       # interior
             (idx(0, 2, 2), idx(0, 3, 1)),       # x- face
             (idx(4, 0, 2), idx(4, 0, 3)),       # x+ y- edge
             (idx(0, 0, 0), idx(0, 0, 0))]       # corner with itself (load equal too)
    for a, b in pairs:
        (Ka, Fa), (Kb, Fb) = cond(a), cond(b)
        assert np.linalg.norm(Ka - Kb) <= 1e-13 * np.linalg.norm(Ka)
        if a != b:
            assert np.linalg.norm(Fa - Fb) > 1e-3 * np.linalg.norm(Fa)
    K1, _ = cond(idx(1, 1, 1))
    K2, _ = cond(idx(0, 2, 2))
    K3, _ = cond(idx(1, 1, 1), c=1.3)
    assert np.linalg.norm(K1 - K2) > 1e-3 * np.linalg.norm(K1)
    assert np.linalg.norm(K1 - K3) > 1e-3 * np.linalg.norm(K1)


def test_interior_condensed_matrix_is_real_after_unit_phases():
    # premise of storing such blocks as reals on the mixed path: in the real
    # form the p-hat traces carry the unit phase i (Sec. 2, the first-order
    # system's i w terms), so an element without an impedance face and with a
    # real wavespeed has Kc[r][c] = a[r][c] i^(s_r - s_c) with a real (s = 1
    # on p-hat traces); the impedance term makes a boundary element's complex
    from oracle.mesh import local_trace_functions
    p, om = 2, 6.0
    m = Mesh((4, 4, 4), p)
    ld = GaussianSource((0.35, 0.5, 0.6), 0.2)
    s = np.array([1 if fn[0] == "p" else 0 for fn in local_trace_functions(p)])
    unphase = (1j) ** (s[None, :] - s[:, None])   # i^(s_c - s_r)

    def cond(e, c=1.0):
        bf = boundary_faces(m, e)
        corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
        K, F = dpg_element(p, m.h, corner, c, om, bf, ld)
        return condense(p, K, F, bf)[0]

    idx = lambda i, j, k: i + 4 * (j + 4 * k)
    for e, c in [(idx(1, 1, 1), 1.0), (idx(2, 1, 2), 0.7)]:
        a = cond(e, c) * unphase
        assert np.linalg.norm(a.imag) <= 1e-12 * np.linalg.norm(a.real)
        assert np.linalg.norm(a - a.T) <= 1e-12 * np.linalg.norm(a)   # real symmetric
    for e in (idx(0, 1, 1), idx(3, 3, 0)):
        a = cond(e) * unphase
        assert np.linalg.norm(a.imag) > 1e-3 * np.linalg.norm(a.real)


def test_assembled_rows_of_interior_entities_are_real_after_unit_phases():
    # the same on the assembled trace operator: every row whose DOF only
    # interior elements touch is real after the phases, and rows touched by an
    # impedance element are not all real
    p, om = 2, 5.0
    fs = build_fine((4, 4, 4), p, om)
    A, _ = fs.assemble()
    mesh = fs.mesh
    s = (np.arange(mesh.n_dof) < mesh.off_U).astype(int)
    touched = np.zeros(mesh.n_dof, dtype=bool)
    for e in range(mesh.n_elem):
        if any(fs.bflags[e]):
            g = fs.dofs[e]
            touched[g[g >= 0]] = True
    A = A.tocoo()
    a = A.data * (1j) ** (s[A.col] - s[A.row])
    inner = ~touched[A.row]
    assert inner.sum() > 0 and (~inner).sum() > 0
    assert np.abs(a[inner].imag).max() <= 1e-12 * np.abs(a[inner]).max()
    assert np.abs(a[~inner].imag).max() > 1e-3 * np.abs(a[~inner]).max()
