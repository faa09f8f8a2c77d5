"""Element-local DPG work on one hexahedron (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here is a plain transcription of Sec. 2 of the paper:

* trial fields (p, u) in L^2, discretised by tensor Legendre Q^{p-1} (the L^2
  member of the order-p exact sequence);
* trial traces (u-hat_n, p-hat) on the element boundary (``oracle.mesh``);
* broken test space (q, v) in H^1 x H(div), enriched by one order (Sec. 2,
  first paragraph): q in Q^{pt}, v_d in Q^{pt} along d and Q^{pt-1} across,
  pt = p + 1, spanned by tensor Legendre polynomials;
* forms of Eq. variational-formulation, with the wavespeed reading
  i omega c^{-2} p + div u = f, i omega u + grad p = g, impedance Z = c:
      b((p,u),(q,v)) = (i w c^-2 p, q) - (u, grad q) + (i w u, v) - (p, div v)
      bhat = s <uhat, q>_F + <phat, v.n_K>_F          on interior faces
      bhat = <phat, Z^-1 q + v.n_K>_F                  on boundary faces
      l(q,v) = (f, q) + (g, v) + <u0, q>_Gamma
  ((a, b) = int a conj(b); s = +1 on the element's high face, -1 on its low
  face, since u-hat is the flux along the +axis normal);
* test inner product of Eq. Gnorm with alpha = 1, with the adjoint
  A^* v = -(i w c^-2 q + div v, grad q + i w v);
* optimal test functions by inverting the Gram matrix (Sec. 2): the element
  DPG matrix K = B^* G^{-1} B and load F = B^* G^{-1} l;
* static condensation of the field DOFs onto the trace DOFs (Sec. 1.2).

All integrals use tensor Gauss rules: pt + 1 points per axis for every
polynomial integrand (exact), pt + 4 points per axis for the load.

Parity: pinned by ``tests/test_oracle_element.py`` (Hermitian positive
definiteness, test-basis invariance, the manufactured polynomial solution
reproduced exactly, plane-wave convergence rates).
"""
import numpy as np

from .basis import gauss01, h1, leg
from .mesh import local_trace_functions


def test_functions(p):
    """Enriched broken test basis: list of ("q", (a,b,c)) and ("v", d, (a,b,c))."""
    pt = p + 1
    out = []
    for c in range(pt + 1):
        for b in range(pt + 1):
            for a in range(pt + 1):
                out.append(("q", (a, b, c)))
    for d in range(3):
        ext = [pt if e == d else pt - 1 for e in range(3)]
        for c in range(ext[2] + 1):
            for b in range(ext[1] + 1):
                for a in range(ext[0] + 1):
                    out.append(("v", d, (a, b, c)))
    return out


def field_functions(p):
    """Trial field basis [p, u_x, u_y, u_z], each L_a L_b L_c, index a + p(b + p c)."""
    out = []
    for comp in range(4):
        for c in range(p):
            for b in range(p):
                for a in range(p):
                    out.append((comp, (a, b, c)))
    return out


def _tensor_points(nq):
    x, w = gauss01(nq)
    X = np.array([(x[i], x[j], x[k]) for k in range(nq) for j in range(nq) for i in range(nq)])
    W = np.array([w[i] * w[j] * w[k] for k in range(nq) for j in range(nq) for i in range(nq)])
    return X, W


def _leg_tables(nmax, Xr, h):
    """1D Legendre values and physical derivatives along each axis at the points."""
    tabs = []
    for d in range(3):
        V, D = leg(nmax, Xr[:, d])
        tabs.append((V, D / h[d]))
    return tabs


def _leg3(idx, tabs):
    """Value and physical gradient of L_a(x) L_b(y) L_c(z) from 1D tables."""
    (Vx, Dx), (Vy, Dy), (Vz, Dz) = tabs
    a, b, c = idx
    v = Vx[a] * Vy[b] * Vz[c]
    g = np.stack([Dx[a] * Vy[b] * Vz[c], Vx[a] * Dy[b] * Vz[c], Vx[a] * Vy[b] * Dz[c]])
    return v, g


def _h1_3(idx, Xr, p):
    vals = []
    for d in range(3):
        V, _ = h1(p, Xr[:, d])
        vals.append(V[idx[d]])
    return vals[0] * vals[1] * vals[2]


def eval_test(p, Xr, h):
    """Test functions at reference points: q, grad q, v, div v (physical)."""
    tf = test_functions(p)
    tabs = _leg_tables(p + 1, Xr, h)
    n = len(tf)
    N = Xr.shape[0]
    q = np.zeros((n, N))
    gq = np.zeros((n, 3, N))
    v = np.zeros((n, 3, N))
    dv = np.zeros((n, N))
    for i, f in enumerate(tf):
        if f[0] == "q":
            val, g = _leg3(f[1], tabs)
            q[i] = val
            gq[i] = g
        else:
            d = f[1]
            val, g = _leg3(f[2], tabs)
            v[i, d] = val
            dv[i] = g[d]
    return q, gq, v, dv


def eval_field(p, Xr, h):
    ff = field_functions(p)
    tabs = _leg_tables(max(p - 1, 0), Xr, h)
    out = np.zeros((len(ff), 4, Xr.shape[0]))
    for j, (comp, idx) in enumerate(ff):
        val, _ = _leg3(idx, tabs)
        out[j, comp] = val
    return out


def boundary_faces(mesh, e):
    """6 flags (x-, x+, y-, y+, z-, z+): face lies on the domain boundary."""
    ec = mesh.elem_coord(e)
    return [ec[d] + s in (0, mesh.n[d]) for d in range(3) for s in range(2)]


def element_matrices(p, h, corner, c, omega, bflags, load=None):
    """Gram G, enriched stiffness B = [B_field | B_trace] and load l of one element.

    Returns (G, B, l) with B columns ordered [field (4p^3), local traces]; the
    columns of u-hat on boundary faces (absent unknowns) are left zero.
    """
    h = np.asarray(h, dtype=np.float64)
    corner = np.asarray(corner, dtype=np.float64)
    pt = p + 1
    beta = omega / c ** 2
    Z = c
    J = h[0] * h[1] * h[2]

    # ---- volume terms ----------------------------------------------------
    Xr, Wr = _tensor_points(pt + 1)
    q, gq, v, dv = eval_test(p, Xr, h)
    w = Wr * J
    # Gram of the adjoint graph norm (Eq. Gnorm, alpha = 1)
    a0 = 1j * beta * q + dv                                  # i w c^-2 q + div v
    a1 = gq + 1j * omega * v                                 # grad q + i w v
    comps = [a0, a1[:, 0], a1[:, 1], a1[:, 2], q, v[:, 0], v[:, 1], v[:, 2]]
    G = np.zeros((q.shape[0], q.shape[0]), dtype=np.complex128)
    for A in comps:
        # G[i, j] = int A_j conj(A_i)
        G += (A.conj() * w) @ A.T

    fld = eval_field(p, Xr, h)                               # (nf, 4, N)
    nf = fld.shape[0]
    loc = local_trace_functions(p)
    ntr = len(loc)
    B = np.zeros((q.shape[0], nf + ntr), dtype=np.complex128)
    P_ = fld[:, 0]
    U_ = fld[:, 1:]
    # (i w c^-2 p, q) - (p, div v)
    B[:, :nf] += (q * w) @ (1j * beta * P_).T
    B[:, :nf] -= (dv * w) @ P_.T
    for d in range(3):
        # -(u, grad q) + (i w u, v)
        B[:, :nf] -= (gq[:, d] * w) @ U_[:, d].T
        B[:, :nf] += (v[:, d] * w) @ (1j * omega * U_[:, d]).T

    # ---- face terms ------------------------------------------------------
    xf, wf = gauss01(pt + 1)
    for d in range(3):
        t1, t2 = [e for e in range(3) if e != d]
        for s in range(2):
            fidx = 2 * d + s
            sgn = 2.0 * s - 1.0
            Xf = np.zeros((len(xf) ** 2, 3))
            Wf = np.zeros(len(xf) ** 2)
            k = 0
            for jb in range(len(xf)):
                for ia in range(len(xf)):
                    Xf[k, d] = s
                    Xf[k, t1] = xf[ia]
                    Xf[k, t2] = xf[jb]
                    Wf[k] = wf[ia] * wf[jb] * h[t1] * h[t2]
                    k += 1
            qf, _, vf, _ = eval_test(p, Xf, h)
            vn = sgn * vf[:, d]                                # v . n_K
            # p-hat columns: <phat, v.n_K> (+ <phat, Z^-1 q> on Gamma)
            pcols = [lj for lj, fn in enumerate(loc) if fn[0] == "p"]
            Ph = np.array([_h1_3(loc[lj][1], Xf, p) for lj in pcols])
            B[:, nf + np.array(pcols)] += (vn * Wf) @ Ph.T
            if bflags[fidx]:
                B[:, nf + np.array(pcols)] += (qf * Wf) @ Ph.T / Z
                continue
            # u-hat columns of this face: s <uhat, q>
            ucols = [lj for lj, fn in enumerate(loc) if fn[0] == "u" and fn[1] == d and fn[2] == s]
            Uh = []
            for lj in ucols:
                _, _, _, a, b = loc[lj]
                La, _ = leg(a, Xf[:, t1])
                Lb, _ = leg(b, Xf[:, t2])
                Uh.append(La[a] * Lb[b])
            B[:, nf + np.array(ucols)] += sgn * ((qf * Wf) @ np.array(Uh).T)

    # ---- load ------------------------------------------------------------
    l = np.zeros(q.shape[0], dtype=np.complex128)
    if load is not None:
        XL, WL = _tensor_points(pt + 4)
        qL, _, vL, _ = eval_test(p, XL, h)
        Xp = corner + XL * h
        wL = WL * J
        if load.f is not None:
            l += (qL * wL) @ load.f(Xp, c)
        if load.g is not None:
            gv = load.g(Xp, c)                                  # (N, 3)
            for d in range(3):
                l += (vL[:, d] * wL) @ gv[:, d]
        if load.u0 is not None:
            xl, wl = gauss01(pt + 4)
            for d in range(3):
                t1, t2 = [e for e in range(3) if e != d]
                for s in range(2):
                    if not bflags[2 * d + s]:
                        continue
                    Xf = np.zeros((len(xl) ** 2, 3))
                    Wf = np.zeros(len(xl) ** 2)
                    k = 0
                    for jb in range(len(xl)):
                        for ia in range(len(xl)):
                            Xf[k, d] = s
                            Xf[k, t1] = xl[ia]
                            Xf[k, t2] = xl[jb]
                            Wf[k] = wl[ia] * wl[jb] * h[t1] * h[t2]
                            k += 1
                    qf, _, _, _ = eval_test(p, Xf, h)
                    nrm = np.zeros(3)
                    nrm[d] = 2.0 * s - 1.0
                    l += (qf * Wf) @ load.u0(corner + Xf * h, nrm, c)
    return G, B, l


def present_columns(p, bflags):
    """Trial columns [field, local traces] that exist (u-hat on Gamma is eliminated)."""
    loc = local_trace_functions(p)
    nf = 4 * p ** 3
    keep = list(range(nf))
    for lj, fn in enumerate(loc):
        if fn[0] == "u" and bflags[2 * fn[1] + fn[2]]:
            continue
        keep.append(nf + lj)
    return np.array(keep)


def dpg_element(p, h, corner, c, omega, bflags, load=None):
    """DPG element matrix K = B^* G^{-1} B and load F = B^* G^{-1} l.

    Rows/columns of absent unknowns are zero.  Returns (K, F).
    """
    G, B, l = element_matrices(p, h, corner, c, omega, bflags, load)
    keep = present_columns(p, bflags)
    Bk = B[:, keep]
    X = np.linalg.solve(G, np.concatenate([Bk, l[:, None]], axis=1))
    m = B.shape[1]
    K = np.zeros((m, m), dtype=np.complex128)
    F = np.zeros(m, dtype=np.complex128)
    K[np.ix_(keep, keep)] = Bk.conj().T @ X[:, :-1]
    F[keep] = Bk.conj().T @ X[:, -1]
    return K, F


def condense(p, K, F, bflags):
    """Static condensation of the 4p^3 field DOFs onto the traces.

    Kc = K_tt - K_tf K_ff^{-1} K_ft,  Fc = F_t - K_tf K_ff^{-1} F_f.
    Returns (Kc, Fc) over the local trace ordering (absent rows/cols zero).
    """
    nf = 4 * p ** 3
    keep = present_columns(p, bflags)
    tk = keep[keep >= nf]
    Kff = K[:nf, :nf]
    Kft = K[:nf][:, tk]
    Ktf = K[tk][:, :nf]
    Y = np.linalg.solve(Kff, np.concatenate([Kft, F[:nf, None]], axis=1))
    ntr = K.shape[0] - nf
    Kc = np.zeros((ntr, ntr), dtype=np.complex128)
    Fc = np.zeros(ntr, dtype=np.complex128)
    Kc[np.ix_(tk - nf, tk - nf)] = K[np.ix_(tk, tk)] - Ktf @ Y[:, :-1]
    Fc[tk - nf] = F[tk] - Ktf @ Y[:, -1]
    return Kc, Fc


def recover_fields(p, K, F, xt):
    """Field DOFs u_f = K_ff^{-1} (F_f - K_ft x_t) from the element's trace values."""
    nf = 4 * p ** 3
    return np.linalg.solve(K[:nf, :nf], F[:nf] - K[:nf, nf:] @ xt)
