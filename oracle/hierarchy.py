"""DPG-MG level hierarchy (oracle), Sec. 3 of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Levels are numbered 0 (coarsest) .. L (finest).  The finest mesh (n, p) is
first p-coarsened down to ``p_min``, then h-coarsened (n -> n/2) while levels
remain and every n is even (the paper builds its hierarchy by refinement,
Sec. 3 first paragraph and Sec. 4 "Uniform p-refinements"; this is the same
hierarchy read from the fine end).

Every level keeps element matrices of its operator A_l, so that each
transition is element-local:

* p-transition (same mesh, order p -> p-1): the hierarchical bases are nested,
  prolongation is injection of the lower-order modes and the restricted coarse
  operator P^* A P is the principal submatrix; smoothing acts on A_l itself.
* h-transition (mesh n -> n/2, Sec. 3 "Prolongation"): stage one condenses,
  per coarse element K, the fine DOFs interior to K (the macro grid): with A^K
  the sum of the 8 children's element matrices,
      M^K = A^K_SS - A^K_SI (A^K_II)^{-1} A^K_IS;
  stage two is the natural inclusion I (coarse trace functions written in the
  fine basis on the coarse skeleton, by constrained approximation: each
  coarse function is interpolated exactly on every fine subface); the coarse
  operator is the restriction A_c^K = I_K^* M^K I_K (Sec. 3 "Alternative
  construction", "restrict").  Smoothing acts on the macro operator
  M_l = sum_K M^K.

Smoother (Sec. 3 "V-cycle and smoother"): additive Schwarz with one block per
vertex w of the next coarser mesh; a DOF belongs to block w when every
(macro-)element adjacent to its entity has w as a corner (rule R1), or, as
an option, when w lies in the closure of the (macro-)entity carrying the DOF
(rule R2; the two differ only at the boundary).  Blocks
are inverted densely.  Damping theta = 1 / (1.05 lambda), lambda from 30
power iterations of S M started from a SplitMix64 vector (seed 12345).

Coarsest level: dense Cholesky factorisation of A_0 (the paper solves its
initial mesh directly with MUMPS, Sec. 4 list; option "none" is its "no
initial-grid solver during the iteration"; option "smooth" applies one damped
additive Schwarz step on level 0 instead, with the vertex patches of level 0's
own mesh and theta from the same power iteration).
"""
import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis import gauss01, h1, leg
from .mesh import Mesh, local_trace_functions
from .splitmix import complex_start_vector

THETA_SEED = 12345
POWER_ITERS = 30
THETA_SAFETY = 1.05


def level_specs(n, p, n_levels, p_min=2):
    """[(n, p)] from finest to coarsest and the transition kind below each level."""
    specs = [(tuple(n), p)]
    kinds = []
    while len(specs) < n_levels:
        cn, cp = specs[-1]
        if cp > p_min:
            specs.append((cn, cp - 1))
            kinds.append("p")
        elif all(v % 2 == 0 and v >= 2 for v in cn):
            specs.append((tuple(v // 2 for v in cn), cp))
            kinds.append("h")
        else:
            break
    return specs, kinds


def assemble(E, dofs, n):
    rows, cols, vals = [], [], []
    for e in range(E.shape[0]):
        g = dofs[e]
        ok = np.nonzero(g >= 0)[0]
        R, C = np.meshgrid(g[ok], g[ok], indexing="ij")
        rows.append(R.ravel())
        cols.append(C.ravel())
        vals.append(E[e][np.ix_(ok, ok)].ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


class Level:
    pass


def _p_selection(p):
    """Positions of the order-(p-1) local trace functions inside the order-p list."""
    fine = local_trace_functions(p)
    pos = {f: i for i, f in enumerate(fine)}
    return np.array([pos[f] for f in local_trace_functions(p - 1)])


def _dof_keys(mesh):
    return {(k, c, m): i for i, (k, c, m) in enumerate(mesh.dof_table())}


def _p_injection(fine_mesh, coarse_mesh):
    """inj[i_coarse] = fine DOF carrying the same entity and mode."""
    fk = _dof_keys(fine_mesh)
    return np.array([fk[key] for key in coarse_mesh.dof_table()], dtype=np.int64)


def _subface_fit(vals_coarse, basis_fine):
    """Coefficients c with basis_fine^T c = vals_coarse (exact interpolation)."""
    return np.linalg.solve(basis_fine.T, vals_coarse)


def _inclusion_element(coarse, fine, K, tab_f):
    """Natural inclusion of coarse element K: {fine DOF: {coarse local fn: coeff}}.

    Constrained approximation, done literally: on every fine subface of the six
    faces of K, sample the coarse trace function at (p+1)^2 points and solve for
    the coefficients of the fine subface functions (exact, the coarse function
    restricted to a subface is a polynomial of the fine space).
    """
    p = coarse.p
    Kc = np.asarray(coarse.elem_coord(K))
    Hc = coarse.h
    hf = fine.h
    loc_c = local_trace_functions(p)
    loc_f = local_trace_functions(p)
    out = {}
    xs = np.linspace(0.05, 0.95, p + 1)          # distinct sample abscissae
    for d in range(3):
        t1, t2 = [e for e in range(3) if e != d]
        for s in range(2):
            for a1 in range(2):
                for a2 in range(2):
                    # child element of K owning this subface
                    cc = [0, 0, 0]
                    cc[d] = s
                    cc[t1] = a1
                    cc[t2] = a2
                    ce = fine.elem_index(tuple(2 * Kc + np.asarray(cc)))
                    gdofs = fine.elem_dofs(ce)
                    # sample points in the child's reference coordinates
                    pts = []
                    for j in range(p + 1):
                        for i in range(p + 1):
                            x = np.zeros(3)
                            x[d] = s
                            x[t1] = xs[i]
                            x[t2] = xs[j]
                            pts.append(x)
                    Xf = np.array(pts)
                    # the same points in K's reference coordinates
                    Xc = (np.asarray(cc) + Xf) * hf / Hc
                    # p-hat: fine functions with index s along d
                    fidx = [i for i, f in enumerate(loc_f) if f[0] == "p" and f[1][d] == s]
                    Vf = np.array([_h1_eval(loc_f[i][1], Xf, p) for i in fidx])
                    for cj, fn in enumerate(loc_c):
                        if fn[0] != "p":
                            continue
                        vc = _h1_eval(fn[1], Xc, p)
                        if np.max(np.abs(vc)) < 1e-15:
                            continue
                        coef = _subface_fit(vc, Vf)
                        for i, cf in zip(fidx, coef):
                            if abs(cf) > 1e-14:
                                _put(out, gdofs[i], cj, cf)
                    # u-hat on the coarse face (d, s)
                    uidx = [i for i, f in enumerate(loc_f) if f[0] == "u" and f[1] == d and f[2] == s]
                    if gdofs[uidx[0]] < 0:
                        continue
                    ptsu = []
                    for j in range(p):
                        for i in range(p):
                            x = np.zeros(3)
                            x[d] = s
                            x[t1] = np.linspace(0.1, 0.9, p)[i] if p > 1 else 0.5
                            x[t2] = np.linspace(0.1, 0.9, p)[j] if p > 1 else 0.5
                            ptsu.append(x)
                    Xu = np.array(ptsu)
                    Xuc = (np.asarray(cc) + Xu) * hf / Hc
                    Vu = np.array([_leg2_eval(loc_f[i], Xu) for i in uidx])
                    for cj, fn in enumerate(loc_c):
                        if fn[0] != "u" or fn[1] != d or fn[2] != s:
                            continue
                        coef = _subface_fit(_leg2_eval(fn, Xuc), Vu)
                        for i, cf in zip(uidx, coef):
                            if abs(cf) > 1e-14:
                                _put(out, gdofs[i], cj, cf)
    return out


def _put(out, g, cj, val):
    row = out.setdefault(int(g), {})
    if cj in row:
        assert abs(row[cj] - val) < 1e-11, "inconsistent inclusion coefficient"
    row[cj] = val


def _h1_eval(idx, X, p):
    v = np.ones(X.shape[0])
    for d in range(3):
        V, _ = h1(p, X[:, d])
        v = v * V[idx[d]]
    return v


def _leg2_eval(fn, X):
    _, d, _, a, b = fn
    t1, t2 = [e for e in range(3) if e != d]
    La, _ = leg(a, X[:, t1])
    Lb, _ = leg(b, X[:, t2])
    return La[a] * Lb[b]


def _patch_rule_R1(lev_mesh, coarse_mesh, table, kind, smask):
    """Vertex patches (rule R1) of the smoothing space of a level.

    Returns a list over coarse vertices of sorted DOF index arrays.
    """
    H = 2 if kind == "p" else 4            # coarse element width, doubled fine units
    nco = coarse_mesh.n
    members = {}
    for i, (kd, ctr, _) in enumerate(table):
        if not smask[i]:
            continue
        # (macro-)elements whose closed box contains the entity centre
        adj = []
        for cand in itertools.product(*[
                [v for v in (ctr[d] // H - 1, ctr[d] // H) if 0 <= v < nco[d]] for d in range(3)]):
            if all(H * cand[d] <= ctr[d] <= H * cand[d] + H for d in range(3)):
                adj.append(cand)
        # coarse vertices that are a corner of every adjacent element
        for w in itertools.product(*[(adj[0][d], adj[0][d] + 1) for d in range(3)]):
            if all(all(w[d] in (E[d], E[d] + 1) for d in range(3)) for E in adj):
                members.setdefault(w, []).append(i)
    out = []
    for w in itertools.product(*[range(v + 1) for v in reversed(nco)]):
        w = (w[2], w[1], w[0])
        out.append(np.array(sorted(members.get(w, [])), dtype=np.int64))
    return out


def _patch_rule_R2(lev_mesh, coarse_mesh, table, kind, smask):
    """Vertex patches (rule R2) of the smoothing space of a level.

    A DOF belongs to block w when w lies in the closure of the coarse entity
    that carries it: on a p level the DOF's own entity, on an h level the
    coarse (macro) entity in whose relative interior the fine entity lies.
    Per axis that closure is the single coarse plane the entity centre lies
    on, or else the two coarse planes around it.  The two rules differ only on
    DOFs of boundary entities: R1 also gives those to the vertices one layer
    inside (the one adjacent element has them as corners), R2 does not.
    Returns a list over coarse vertices of sorted DOF index arrays.
    """
    H = 2 if kind == "p" else 4
    nco = coarse_mesh.n
    members = {}
    for i, (kd, ctr, _) in enumerate(table):
        if not smask[i]:
            continue
        span = [(ctr[d] // H,) if ctr[d] % H == 0 else (ctr[d] // H, ctr[d] // H + 1) for d in range(3)]
        for w in itertools.product(*span):
            members.setdefault(w, []).append(i)
    out = []
    for w in itertools.product(*[range(v + 1) for v in reversed(nco)]):
        w = (w[2], w[1], w[0])
        out.append(np.array(sorted(members.get(w, [])), dtype=np.int64))
    return out


PATCH_RULES = {"R1": _patch_rule_R1, "R2": _patch_rule_R2}


def build_hierarchy(fine_mesh, Kc, dofs, n_levels, p_min=2, coarsest="cholesky",
                    theta=None, stored=None, patch_rule="R1"):
    """All levels from the fine element matrices Kc (condensed) and DOF maps.

    Coarse operators are restricted (Sec. 3, A_c = I^* M I) unless ``stored``
    is given: stored(mesh) returns the condensed element matrices of the DPG
    system assembled directly on a coarser mesh (the paper's "stored"
    alternative), which then replace the restricted ones level by level.
    ``patch_rule`` picks the vertex-patch membership at the boundary ("R1",
    the default, or "R2"; the paper does not say which, Sec. 3 "V-cycle and
    smoother").
    """
    rule = PATCH_RULES[patch_rule]
    specs, kinds = level_specs(fine_mesh.n, fine_mesh.p, n_levels, p_min)
    levels = []
    top = Level()
    top.mesh = fine_mesh
    top.E = Kc
    top.dofs = dofs
    levels.append(top)
    for li, kind in enumerate(kinds):
        lev = levels[-1]
        lev.kind = kind
        cn, cp = specs[li + 1]
        cmesh = Mesh(cn, cp, lev.mesh.x0, lev.mesh.x1)
        crs = Level()
        crs.mesh = cmesh
        crs.dofs = np.stack([cmesh.elem_dofs(e) for e in range(cmesh.n_elem)])
        nf = lev.mesh.n_dof
        if kind == "p":
            sel = _p_selection(lev.mesh.p)
            crs.E = lev.E[:, sel][:, :, sel]
            lev.inj = _p_injection(lev.mesh, cmesh)
            lev.M = assemble(lev.E, lev.dofs, nf)
            lev.smask = np.ones(nf, dtype=bool)
        else:
            table = lev.mesh.dof_table()
            ntl = len(local_trace_functions(cp))
            crs.E = np.zeros((cmesh.n_elem, ntl, ntl), dtype=np.complex128)
            lev.S, lev.I, lev.Aii_inv, lev.T = [], [], [], []
            Mrows, Mcols, Mvals = [], [], []
            Irows, Icols, Ivals = [], [], []
            for K in range(cmesh.n_elem):
                Kc3 = np.asarray(cmesh.elem_coord(K))
                kids = [lev.mesh.elem_index(tuple(2 * Kc3 + np.asarray(o)))
                        for o in itertools.product((0, 1), repeat=3)]
                glob = sorted({int(g) for c in kids for g in lev.dofs[c] if g >= 0})
                pos = {g: i for i, g in enumerate(glob)}
                AK = np.zeros((len(glob), len(glob)), dtype=np.complex128)
                for c in kids:
                    g = lev.dofs[c]
                    ok = np.nonzero(g >= 0)[0]
                    li_ = np.array([pos[int(v)] for v in g[ok]])
                    AK[np.ix_(li_, li_)] += lev.E[c][np.ix_(ok, ok)]
                lo = 4 * Kc3
                on_bdry = np.array([any(table[g][1][d] in (lo[d], lo[d] + 4) for d in range(3))
                                    for g in glob])
                Sl = np.nonzero(on_bdry)[0]
                Il = np.nonzero(~on_bdry)[0]
                Aii = AK[np.ix_(Il, Il)]
                Aii_inv = np.linalg.inv(Aii)
                T = AK[np.ix_(Sl, Il)] @ Aii_inv
                MK = AK[np.ix_(Sl, Sl)] - T @ AK[np.ix_(Il, Sl)]
                Sg = np.array(glob)[Sl]
                Ig = np.array(glob)[Il]
                lev.S.append(Sg)
                lev.I.append(Ig)
                lev.Aii_inv.append(Aii_inv)
                lev.T.append(T)
                R, C = np.meshgrid(Sg, Sg, indexing="ij")
                Mrows.append(R.ravel())
                Mcols.append(C.ravel())
                Mvals.append(MK.ravel())
                # natural inclusion restricted to K, and the restricted operator
                inc = _inclusion_element(cmesh, lev.mesh, K, table)
                IK = np.zeros((len(Sg), ntl))
                spos = {int(g): i for i, g in enumerate(Sg)}
                for g, row in inc.items():
                    for cj, val in row.items():
                        IK[spos[g], cj] = val
                cg = crs.dofs[K]
                IK[:, cg < 0] = 0.0
                crs.E[K] = IK.T @ MK @ IK
                for g, row in inc.items():
                    for cj, val in row.items():
                        if cg[cj] >= 0:
                            Irows.append(g)
                            Icols.append(int(cg[cj]))
                            Ivals.append(val)
            lev.M = sp.coo_matrix((np.concatenate(Mvals), (np.concatenate(Mrows),
                                   np.concatenate(Mcols))), shape=(nf, nf)).tocsr()
            lev.M.sum_duplicates()
            # global inclusion: coefficients are identical from both sides of a
            # shared coarse face, keep one copy of each (row, col)
            seen = {}
            for r_, c_, v_ in zip(Irows, Icols, Ivals):
                if (r_, c_) in seen:
                    assert abs(seen[(r_, c_)] - v_) < 1e-11
                seen[(r_, c_)] = v_
            keys = list(seen.keys())
            lev.P = sp.coo_matrix(([seen[k] for k in keys], ([k[0] for k in keys], [k[1] for k in keys])),
                                  shape=(nf, cmesh.n_dof)).tocsr()
            lev.smask = np.zeros(nf, dtype=bool)
            for Sg in lev.S:
                lev.smask[Sg] = True
        if stored is not None:
            crs.E = stored(cmesh)
        lev.patches = rule(lev.mesh, cmesh, lev.mesh.dof_table(), kind, lev.smask)
        Md = lev.M
        lev.patch_inv = [np.linalg.inv(Md[idx][:, idx].toarray()) for idx in lev.patches]
        lev.theta = theta if theta is not None else estimate_theta(lev)
        levels.append(crs)
    levels[-1].kind = None
    c0 = levels[-1]
    c0.A = assemble(c0.E, c0.dofs, c0.mesh.n_dof).toarray()
    c0.coarsest = coarsest
    if coarsest == "cholesky" or len(levels) == 1:
        c0.coarsest = "cholesky"
        c0.chol = sla.cho_factor(c0.A, lower=True)
    elif coarsest == "smooth":
        # level 0 smoothed with the vertex patches of its own mesh (the p-level
        # rule with the level itself as the coarse mesh)
        c0.M = sp.csr_matrix(c0.A)
        c0.smask = np.ones(c0.mesh.n_dof, dtype=bool)
        c0.patches = rule(c0.mesh, c0.mesh, c0.mesh.dof_table(), "p", c0.smask)
        c0.patch_inv = [np.linalg.inv(c0.A[np.ix_(idx, idx)]) for idx in c0.patches]
        c0.theta = theta if theta is not None else estimate_theta(c0)
    levels.reverse()
    return levels


def smoother(lev, r):
    """Undamped additive Schwarz S r = sum_j R_j^T (R_j M R_j^T)^{-1} R_j r."""
    out = np.zeros_like(r)
    for idx, Ainv in zip(lev.patches, lev.patch_inv):
        out[idx] += Ainv @ r[idx]
    return out


def estimate_theta(lev):
    """theta = 1 / (1.05 lambda), lambda ~ largest eigenvalue of S M.

    Power iteration x <- S M x / ||S M x||_2 (30 steps) from a SplitMix64
    vector restricted to the smoothing space, then the Rayleigh quotient
    lambda = (M x, S M x) / (M x, x).
    """
    n = lev.M.shape[0]
    x = complex_start_vector(THETA_SEED, n)
    x[~lev.smask] = 0.0
    x /= np.linalg.norm(x)
    for _ in range(POWER_ITERS):
        y = smoother(lev, lev.M @ x)
        x = y / np.linalg.norm(y)
    Mx = lev.M @ x
    lam = np.vdot(smoother(lev, Mx), Mx).real / np.vdot(x, Mx).real
    return 1.0 / (THETA_SAFETY * lam)
