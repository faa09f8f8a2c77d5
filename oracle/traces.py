"""Global trace DOFs of a given pressure / velocity pair (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Used by the pins: the trace unknowns of Sec. 2 are p-hat = trace of p and
u-hat_n = u . n.  For a function whose traces lie in the discrete trace spaces
the face-wise L^2 projection below reproduces them exactly, independently of
how the solver or the natural inclusion computes them.
"""
import numpy as np

from .basis import gauss01, h1, leg
from .mesh import local_trace_functions


def trace_dofs(mesh, pfun, ufun):
    """x with x[p-hat DOFs] = face-wise L^2 projection of pfun, x[u-hat] of ufun . e_d."""
    p = mesh.p
    x = np.zeros(mesh.n_dof, dtype=np.complex128)
    loc = local_trace_functions(p)
    xq, wq = gauss01(p + 3)
    for e in range(mesh.n_elem):
        ec = np.asarray(mesh.elem_coord(e))
        corner = mesh.x0 + ec * mesh.h
        g = mesh.elem_dofs(e)
        for d in range(3):
            t1, t2 = [t for t in range(3) if t != d]
            for s in range(2):
                Xr = np.zeros((len(xq) ** 2, 3))
                W = np.zeros(len(xq) ** 2)
                k = 0
                for j in range(len(xq)):
                    for i in range(len(xq)):
                        Xr[k, d] = s
                        Xr[k, t1] = xq[i]
                        Xr[k, t2] = xq[j]
                        W[k] = wq[i] * wq[j]
                        k += 1
                Xp = corner + Xr * mesh.h
                # p-hat: the (p+1)^2 element functions that live on this face
                idx = [i for i, f in enumerate(loc) if f[0] == "p" and f[1][d] == s]
                Phi = []
                for i in idx:
                    a = loc[i][1]
                    v = np.ones(len(W))
                    for dd in range(3):
                        V, _ = h1(p, Xr[:, dd])
                        v = v * V[a[dd]]
                    Phi.append(v)
                Phi = np.array(Phi)
                Mm = (Phi * W) @ Phi.T
                c = np.linalg.solve(Mm, (Phi * W) @ pfun(Xp))
                x[g[idx]] = c
                # u-hat: Legendre coefficients of u . e_d on interior faces
                uidx = [i for i, f in enumerate(loc) if f[0] == "u" and f[1] == d and f[2] == s]
                if g[uidx[0]] < 0:
                    continue
                ud = ufun(Xp)[:, d]
                for i in uidx:
                    _, _, _, a, b = loc[i]
                    La, _ = leg(a, Xr[:, t1])
                    Lb, _ = leg(b, Xr[:, t2])
                    x[g[i]] = (2 * a + 1) * (2 * b + 1) * np.sum(W * ud * La[a] * Lb[b])
    return x


def field_dofs(mesh, pfun, ufun):
    """Per-element Legendre coefficients [p, u_x, u_y, u_z] (L^2 projection)."""
    p = mesh.p
    xq, wq = gauss01(p + 3)
    X = np.array([(xq[i], xq[j], xq[k]) for k in range(len(xq)) for j in range(len(xq))
                  for i in range(len(xq))])
    W = np.array([wq[i] * wq[j] * wq[k] for k in range(len(xq)) for j in range(len(xq))
                  for i in range(len(xq))])
    tabs = [leg(max(p - 1, 0), X[:, d])[0] for d in range(3)]
    out = np.zeros((mesh.n_elem, 4 * p ** 3), dtype=np.complex128)
    for e in range(mesh.n_elem):
        corner = mesh.x0 + np.asarray(mesh.elem_coord(e)) * mesh.h
        Xp = corner + X * mesh.h
        vals = [pfun(Xp)] + [ufun(Xp)[:, d] for d in range(3)]
        j = 0
        for comp in range(4):
            for c in range(p):
                for b in range(p):
                    for a in range(p):
                        phi = tabs[0][a] * tabs[1][b] * tabs[2][c]
                        out[e, j] = (2 * a + 1) * (2 * b + 1) * (2 * c + 1) * np.sum(W * vals[comp] * phi)
                        j += 1
    return out
