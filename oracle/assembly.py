"""Fine-grid DPG trace system: element loop and global assembly (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For every element: the DPG element matrix (``oracle.element.dpg_element``),
static condensation of the fields (Sec. 1.2), then the condensed matrices are
summed into the global Hermitian positive-definite trace system A x = b
(Sec. 6 notes that the condensed system is HPD).  The element data needed to
recover the fields afterwards is kept.
"""
import numpy as np
import scipy.sparse as sp

from .element import boundary_faces, condense, dpg_element, recover_fields
from .mesh import Mesh


class FineSystem:
    """Condensed element matrices, their global DOF maps and the assembled system."""

    def __init__(self, mesh, omega, wavespeed=None, load=None, elements=None):
        self.mesh = mesh
        self.omega = float(omega)
        self.load = load
        ne = mesh.n_elem
        self.c = np.ones(ne) if wavespeed is None else np.asarray(wavespeed, dtype=np.float64)
        p = mesh.p
        ntr = mesh.n_local()
        self.dofs = np.stack([mesh.elem_dofs(e) for e in range(ne)])
        self.Kc = np.zeros((ne, ntr, ntr), dtype=np.complex128)
        self.Fc = np.zeros((ne, ntr), dtype=np.complex128)
        self.K = [None] * ne
        self.F = [None] * ne
        self.bflags = [boundary_faces(mesh, e) for e in range(ne)]
        todo = range(ne) if elements is None else elements
        for e in todo:
            ec = mesh.elem_coord(e)
            corner = mesh.x0 + np.asarray(ec) * mesh.h
            K, F = dpg_element(p, mesh.h, corner, self.c[e], self.omega, self.bflags[e], load)
            self.K[e], self.F[e] = K, F
            self.Kc[e], self.Fc[e] = condense(p, K, F, self.bflags[e])

    def assemble(self):
        """Global sparse A (CSR) and dense b from the condensed element matrices."""
        rows, cols, vals = [], [], []
        b = np.zeros(self.mesh.n_dof, dtype=np.complex128)
        for e in range(self.mesh.n_elem):
            g = self.dofs[e]
            ok = np.nonzero(g >= 0)[0]
            gi = g[ok]
            R, C = np.meshgrid(gi, gi, indexing="ij")
            rows.append(R.ravel())
            cols.append(C.ravel())
            vals.append(self.Kc[e][np.ix_(ok, ok)].ravel())
            np.add.at(b, gi, self.Fc[e][ok])
        n = self.mesh.n_dof
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n)).tocsr()
        A.sum_duplicates()
        return A, b

    def fields(self, x):
        """Per-element field DOFs [p, u_x, u_y, u_z] from the global trace vector x."""
        p = self.mesh.p
        out = np.zeros((self.mesh.n_elem, 4 * p ** 3), dtype=np.complex128)
        for e in range(self.mesh.n_elem):
            g = self.dofs[e]
            xt = np.where(g >= 0, x[np.maximum(g, 0)], 0.0)
            out[e] = recover_fields(p, self.K[e], self.F[e], xt)
        return out


def build_fine(n, p, omega, wavespeed=None, load=None, x0=(0, 0, 0), x1=(1, 1, 1)):
    mesh = Mesh(n, p, x0, x1)
    return FineSystem(mesh, omega, wavespeed, load)
