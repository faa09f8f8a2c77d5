"""Pins of the oracle's mesh and global trace numbering (no GPU)."""
import itertools

import numpy as np
import pytest

from oracle.mesh import Mesh, n_trace_local


def closed_form_ndof(n, p):
    nx, ny, nz = n
    V = (nx + 1) * (ny + 1) * (nz + 1)
    E = nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz
    F = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)
    Fi = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    return V + E * (p - 1) + F * (p - 1) ** 2 + Fi * p * p


# DOF counts of the workload meshes (exact counts on structured grids)
@pytest.mark.parametrize("n,p,N", [((4, 4, 4), 2, 1241), ((4, 4, 4), 1, 269),
                                   ((16, 16, 16), 3, 188561), ((16, 16, 16), 2, 77921),
                                   ((8, 8, 8), 2, 9777), ((32, 32, 16), 3, 753905),
                                   ((8, 8, 4), 2, 4905), ((24, 24, 24), 4, 1175329)])
def test_dof_counts(n, p, N):
    m = Mesh(n, p)
    assert m.n_dof == N == closed_form_ndof(n, p)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_local_sizes(p):
    assert Mesh((1, 1, 1), p).n_local() == n_trace_local(p)
    assert n_trace_local(p) == {1: 14, 2: 50, 3: 110}[p]


@pytest.mark.parametrize("n,p", [((2, 3, 2), 2), ((3, 2, 2), 3), ((2, 2, 2), 1)])
def test_numbering_is_consistent(n, p):
    m = Mesh(n, p)
    dofs = np.stack([m.elem_dofs(e) for e in range(m.n_elem)])
    used = dofs[dofs >= 0]
    assert set(used.tolist()) == set(range(m.n_dof))         # every DOF reached
    for e in range(m.n_elem):
        assert len(set(dofs[e][dofs[e] >= 0].tolist())) == int(np.sum(dofs[e] >= 0))
    # multiplicity = number of elements adjacent to the entity
    tab = m.dof_table()
    count = np.bincount(used, minlength=m.n_dof)
    for g, (kind, ctr, _) in enumerate(tab):
        adj = 1
        for d in range(3):
            flat = ctr[d] % 2 == 0
            interior = 0 < ctr[d] < 2 * m.n[d]
            adj *= 2 if (flat and interior) else 1
        assert count[g] == adj
    # the element-local p-hat function (a,b,c) of neighbours agree on shared faces
    for e in range(m.n_elem):
        ec = m.elem_coord(e)
        for d in range(3):
            if ec[d] + 1 >= n[d]:
                continue
            nb = list(ec)
            nb[d] += 1
            f = m.elem_index(tuple(nb))
            loc = [x for x in __import__("oracle.mesh", fromlist=["x"]).local_trace_functions(p)]
            pos = {fn: i for i, fn in enumerate(loc)}
            for fn in loc:
                if fn[0] == "p" and fn[1][d] == 1:
                    other = list(fn[1])
                    other[d] = 0
                    assert dofs[e][pos[fn]] == dofs[f][pos[("p", tuple(other))]]
                if fn[0] == "u" and fn[1] == d and fn[2] == 1:
                    assert dofs[e][pos[fn]] == dofs[f][pos[("u", d, 0, fn[3], fn[4])]] >= 0
