"""Builds oracle systems from the same workload dictionaries the library gets.

Test infrastructure: the tests drive both sides with identical seeded inputs
(``paper_2304_01728_gb300.workloads``) and compare element by element.
"""
import multiprocessing as mp
import os

import numpy as np

from oracle.assembly import FineSystem, build_fine
from oracle.element import condense, dpg_element
from oracle.mesh import Mesh
from oracle.hierarchy import build_hierarchy
from oracle.problem import GaussianSource, Manufactured, PlaneWave


def oracle_load(pk):
    src = pk.get("source", "gaussian")
    if src == "gaussian":
        return GaussianSource(pk.get("src_center", (0.5, 0.5, 0.5)), pk.get("src_width", 0.1), pk.get("src_amp", 1.0))
    if src == "plane_wave":
        return PlaneWave(pk["wave_dir"], pk["omega"], 1.0)
    return Manufactured(pk["mf_coeffs"], pk["omega"], pk.get("x0", (0, 0, 0)), pk.get("x1", (1, 1, 1)))


_CTX = {}


def _pinit(pk):
    _CTX.update(pk=pk, mesh=Mesh(pk["n"], pk["p"], pk.get("x0", (0, 0, 0)), pk.get("x1", (1, 1, 1))),
                load=oracle_load(pk))


def _pelem(e):
    """One element of the oracle's FineSystem, computed by the oracle's own
    dpg_element / condense exactly as FineSystem does."""
    pk, m = _CTX["pk"], _CTX["mesh"]
    from oracle.element import boundary_faces
    bf = boundary_faces(m, e)
    corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
    c = 1.0 if pk.get("wavespeed") is None else float(np.asarray(pk["wavespeed"]).ravel()[e])
    K, F = dpg_element(m.p, m.h, corner, c, pk["omega"], bf, _CTX["load"])
    Kc, Fc = condense(m.p, K, F, bf)
    return e, K, F, Kc, Fc


def build_fine_parallel(pk, workers=None):
    """The oracle's FineSystem with its element loop spread over processes
    (started with 'spawn', so that no GPU context is inherited); the same
    numbers as oracle.assembly.build_fine."""
    workers = workers or min(16, os.cpu_count() or 1)
    mesh = Mesh(pk["n"], pk["p"], pk.get("x0", (0, 0, 0)), pk.get("x1", (1, 1, 1)))
    fs = FineSystem(mesh, pk["omega"], pk.get("wavespeed"), oracle_load(pk), elements=[])
    with mp.get_context("spawn").Pool(workers, initializer=_pinit, initargs=(pk,)) as pool:
        for e, K, F, Kc, Fc in pool.imap_unordered(_pelem, range(mesh.n_elem), chunksize=2):
            fs.K[e], fs.F[e], fs.Kc[e], fs.Fc[e] = K, F, Kc, Fc
    return fs


def oracle_system(pk, ok, hierarchy=True, parallel=False):
    if parallel and np.prod(pk["n"]) >= 8 and (os.cpu_count() or 1) > 1:
        fs = build_fine_parallel(pk)
    else:
        fs = build_fine(pk["n"], pk["p"], pk["omega"], wavespeed=pk.get("wavespeed"), load=oracle_load(pk),
                        x0=pk.get("x0", (0, 0, 0)), x1=pk.get("x1", (1, 1, 1)))
    A, b = fs.assemble()
    levels = None
    if hierarchy:
        stored = None
        if ok.get("flags", 0) & 4:   # coarse operators assembled on each coarser mesh
            c = np.asarray(pk["wavespeed"]).ravel()[0] if pk.get("wavespeed") is not None else 1.0

            def stored(cmesh):
                cf = build_fine(cmesh.n, cmesh.p, pk["omega"], wavespeed=np.full(cmesh.n_elem, c),
                                load=oracle_load(pk), x0=cmesh.x0, x1=cmesh.x1)
                return cf.Kc
        levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, ok.get("n_levels", 2), ok.get("p_min", 2),
                                 coarsest=ok.get("coarsest", "cholesky"), stored=stored,
                                 patch_rule="R2" if ok.get("flags", 0) & 64 else "R1")
    return fs, A, b, levels


# Mixed path against the FP64 oracle.  Its V-cycle runs in complex64, and its
# patch factorisations (Cholesky, triangular inverse, L^-H L^-1) and macro
# condensations are computed in FP32 from complex64 blocks, so the V-cycle and
# the damping theta (estimated on the smoother the V-cycle applies) differ from
# the oracle's FP64 ones by the FP32 factorisation error: complex64 rounding
# (2^-24) amplified by the block condition numbers.  Measured: V-cycle up to
# 2.1e-5 and theta up to 4.1e-5 (order 5), 4e-6 on the 16^3, p = 3 workload.
# The solution itself is held to the parity bar (1e-7, iterations within 10%).
MIXED_VCYCLE_TOL = 1e-4
MIXED_THETA_TOL = 1e-4


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rand_vec(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)
