"""Structured hexahedral meshes and the global trace-DOF numbering (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The trace unknowns of the broken ultraweak formulation (Sec. 2, "Broken
ultraweak formulation") live on the mesh skeleton: p-hat is the trace of an
H^1-conforming field of order p (vertex, edge and face functions), u-hat_n the
normal trace of an H(div)-conforming field of order p (face functions only).
Under the impedance reading used throughout, u-hat_n is eliminated on the
domain boundary Gamma, so boundary faces carry p-hat DOFs only.

Global numbering (entity-blocked, the same one the C-ABI documents):

  block V  vertices, 1 DOF each, vertex (i,j,k) -> i + (nx+1)(j + (ny+1)k)
  block E  edges along x, then y, then z; an edge along d has index extents
           n_e + (e != d); p-1 DOFs each (H^1 modes 2..p of that axis)
  block F  faces normal to x, then y, then z (p-hat); a face normal to d has
           extents n_e + (e == d); (p-1)^2 DOFs each, modes (m1, m2) of the two
           tangential axes in increasing axis order, index (m1-2) + (p-1)(m2-2)
  block U  interior faces only (u-hat_n), same face order with the boundary
           faces skipped; p^2 DOFs each, Legendre modes (a, b) of the
           tangential axes, index a + p b; the unknown is the flux in the
           +axis direction of the face normal.

Element-local trace ordering: first the p-hat functions phi_a(x) phi_b(y)
phi_c(z) for (a, b, c) in {0..p}^3 ordered by a + (p+1)(b + (p+1)c), keeping
the triples with at least one index in {0, 1}; then the u-hat functions of the
six faces in the order x-, x+, y-, y+, z-, z+, modes a + p b.

Parity: pinned by ``tests/test_oracle_mesh.py`` (closed-form DOF counts,
bijectivity, neighbour agreement of shared entities).
"""
import itertools

import numpy as np


def tangential(d):
    """The two axes tangential to a face normal to axis d, increasing order."""
    return [e for e in range(3) if e != d]


class Mesh:
    """Axis-aligned box split into nx x ny x nz equal hexahedra, trace order p."""

    def __init__(self, n, p, x0=(0.0, 0.0, 0.0), x1=(1.0, 1.0, 1.0)):
        self.n = tuple(int(v) for v in n)
        self.p = int(p)
        self.x0 = np.asarray(x0, dtype=np.float64)
        self.x1 = np.asarray(x1, dtype=np.float64)
        self.h = (self.x1 - self.x0) / np.asarray(self.n, dtype=np.float64)
        n0, n1, n2 = self.n
        self.n_elem = n0 * n1 * n2
        self.n_vert = (n0 + 1) * (n1 + 1) * (n2 + 1)
        self.edge_ext = [[self.n[e] + (e != d) for e in range(3)] for d in range(3)]
        self.face_ext = [[self.n[e] + (e == d) for e in range(3)] for d in range(3)]
        self.n_edge_d = [int(np.prod(x)) for x in self.edge_ext]
        self.n_face_d = [int(np.prod(x)) for x in self.face_ext]
        self.iface_ext = [[self.n[e] - (e == d) for e in range(3)] for d in range(3)]
        self.n_iface_d = [int(np.prod(x)) for x in self.iface_ext]
        p = self.p
        self.n_edge = sum(self.n_edge_d)
        self.n_face = sum(self.n_face_d)
        self.n_iface = sum(self.n_iface_d)
        self.off_E = self.n_vert
        self.off_F = self.off_E + self.n_edge * (p - 1)
        self.off_U = self.off_F + self.n_face * (p - 1) ** 2
        self.n_dof = self.off_U + self.n_iface * p * p
        self._local = local_trace_functions(p)

    # ---- entity indices -------------------------------------------------
    @staticmethod
    def _lin(c, ext):
        return c[0] + ext[0] * (c[1] + ext[1] * c[2])

    def vertex(self, c):
        return self._lin(c, [v + 1 for v in self.n])

    def edge(self, d, c):
        return sum(self.n_edge_d[:d]) + self._lin(c, self.edge_ext[d])

    def face(self, d, c):
        return sum(self.n_face_d[:d]) + self._lin(c, self.face_ext[d])

    def is_boundary_face(self, d, c):
        return c[d] == 0 or c[d] == self.n[d]

    def iface(self, d, c):
        cc = list(c)
        cc[d] -= 1
        return sum(self.n_iface_d[:d]) + self._lin(cc, self.iface_ext[d])

    # ---- element <-> global ---------------------------------------------
    def elem_coord(self, e):
        n0, n1, _ = self.n
        return (e % n0, (e // n0) % n1, e // (n0 * n1))

    def elem_index(self, c):
        return self._lin(c, self.n)

    def n_local(self):
        return len(self._local)

    def elem_dofs(self, e):
        """Global DOF of every element-local trace function (-1 if absent)."""
        p = self.p
        ec = self.elem_coord(e)
        out = np.full(len(self._local), -1, dtype=np.int64)
        for li, f in enumerate(self._local):
            if f[0] == "p":
                idx = f[1]
                vdims = [d for d in range(3) if idx[d] < 2]
                pos = [ec[d] + (idx[d] if idx[d] < 2 else 0) for d in range(3)]
                if len(vdims) == 3:
                    out[li] = self.vertex(pos)
                elif len(vdims) == 2:
                    d = [dd for dd in range(3) if dd not in vdims][0]
                    out[li] = self.off_E + self.edge(d, pos) * (p - 1) + (idx[d] - 2)
                else:
                    d = vdims[0]
                    t1, t2 = tangential(d)
                    out[li] = (self.off_F + self.face(d, pos) * (p - 1) ** 2
                               + (idx[t1] - 2) + (p - 1) * (idx[t2] - 2))
            else:
                _, d, s, a, b = f
                pos = list(ec)
                pos[d] += s
                if self.is_boundary_face(d, pos):
                    continue
                out[li] = self.off_U + self.iface(d, pos) * p * p + a + p * b
        return out

    def dof_table(self):
        """Per global DOF: (kind, doubled-coordinate entity centre, modes).

        kind is "v", "e", "f" (p-hat) or "u" (u-hat).  The centre of an entity
        is given in units of half an element, so vertex (i,j,k) sits at
        (2i, 2j, 2k) and the edge along x from it at (2i+1, 2j, 2k).
        """
        p = self.p
        tab = [None] * self.n_dof
        for c in itertools.product(*[range(v + 1) for v in self.n]):
            c = (c[0], c[1], c[2])
            tab[self.vertex(c)] = ("v", tuple(2 * v for v in c), ())
        for d in range(3):
            for c in itertools.product(*[range(v) for v in self.edge_ext[d]]):
                g = self.edge(d, c)
                ctr = [2 * v for v in c]
                ctr[d] += 1
                for m in range(2, p + 1):
                    tab[self.off_E + g * (p - 1) + m - 2] = ("e", tuple(ctr), (d, m))
        for d in range(3):
            t1, t2 = tangential(d)
            for c in itertools.product(*[range(v) for v in self.face_ext[d]]):
                ctr = [2 * v for v in c]
                ctr[t1] += 1
                ctr[t2] += 1
                g = self.face(d, c)
                for m2 in range(2, p + 1):
                    for m1 in range(2, p + 1):
                        tab[self.off_F + g * (p - 1) ** 2 + (m1 - 2) + (p - 1) * (m2 - 2)] = (
                            "f", tuple(ctr), (d, m1, m2))
                if not self.is_boundary_face(d, c):
                    r = self.iface(d, c)
                    for b in range(p):
                        for a in range(p):
                            tab[self.off_U + r * p * p + a + p * b] = ("u", tuple(ctr), (d, a, b))
        return tab


def local_trace_functions(p):
    """Element-local trace functions in the documented order.

    ("p", (a, b, c)) for p-hat = phi_a(x) phi_b(y) phi_c(z);
    ("u", d, s, a, b) for u-hat on face normal d at side s (0 low, 1 high),
    Legendre modes (a, b) of the tangential axes.
    """
    out = []
    for c in range(p + 1):
        for b in range(p + 1):
            for a in range(p + 1):
                if min(a, b, c) < 2:
                    out.append(("p", (a, b, c)))
    for d in range(3):
        for s in range(2):
            for b in range(p):
                for a in range(p):
                    out.append(("u", d, s, a, b))
    return out


def n_trace_local(p):
    return (p + 1) ** 3 - (p - 1) ** 3 + 6 * p * p
