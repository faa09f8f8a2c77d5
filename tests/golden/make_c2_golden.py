"""Writes tests/golden/c2_oracle.json: full-size oracle reference values of the
16^3, p = 3, omega = 16 pi workload (FP64 V-cycle, 3 levels, tol 1e-8).

Calls only oracle/ (and the seeded workload generator).  The element loop is
distributed over processes; each element is computed by the oracle's own
dpg_element / condense, unchanged.  Run: python tests/golden/make_c2_golden.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

from oracle.assembly import FineSystem  # noqa: E402
from oracle.element import condense, dpg_element  # noqa: E402
from oracle.hierarchy import build_hierarchy  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from oracle.problem import GaussianSource  # noqa: E402
from oracle.solver import mg_pcg  # noqa: E402
from paper_2304_01728_gb300 import workloads  # noqa: E402

# random sketch of the solution: SKETCH_ROWS seeded +-1 projections, from which a
# test estimates the relative L2 error of a whole solution vector (its expected
# square is ||x - x_ref||^2 * SKETCH_ROWS)
SKETCH_SEED, SKETCH_ROWS = 4242, 128


def sketch(x):
    out = np.empty(SKETCH_ROWS, complex)
    for j0 in range(0, SKETCH_ROWS, 16):
        out[j0:j0 + 16] = workloads.rademacher_rows(SKETCH_SEED, j0, j0 + 16, x.size) @ x
    return out

_CTX = {}


def _init(pk):
    m = Mesh(pk["n"], pk["p"], pk.get("x0", (0, 0, 0)), pk.get("x1", (1, 1, 1)))
    _CTX.update(mesh=m, pk=pk, load=GaussianSource(pk["src_center"], pk["src_width"]))


def _elem(e):
    m, pk, ld = _CTX["mesh"], _CTX["pk"], _CTX["load"]
    from oracle.element import boundary_faces
    bf = boundary_faces(m, e)
    corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
    c = 1.0 if pk.get("wavespeed") is None else pk["wavespeed"][e]
    K, F = dpg_element(m.p, m.h, corner, c, pk["omega"], bf, ld)
    Kc, Fc = condense(m.p, K, F, bf)
    return e, Kc, Fc


def main():
    w = workloads.config2("fp64")
    pk, ok = w["problem"], w["opts"]
    t0 = time.time()
    mesh = Mesh(pk["n"], pk["p"])
    fs = FineSystem(mesh, pk["omega"], pk.get("wavespeed"), None, elements=[])
    with mp.get_context("spawn").Pool(int(os.environ.get("WORKERS", os.cpu_count())), initializer=_init,
                                      initargs=(pk,)) as pool:
        for e, Kc, Fc in pool.imap_unordered(_elem, range(mesh.n_elem), chunksize=16):
            fs.Kc[e], fs.Fc[e] = Kc, Fc
    t1 = time.time()
    A, b = fs.assemble()
    levels = build_hierarchy(mesh, fs.Kc, fs.dofs, ok["n_levels"], ok["p_min"])
    t2 = time.time()
    x, it, hist = mg_pcg(levels, A, b, tol=ok["tol"])
    t3 = time.time()
    rng = np.random.default_rng(2024)
    idx = sorted(rng.choice(A.shape[0], 64, replace=False).tolist())
    out = {
        "workload": w["name"], "n_dof": int(A.shape[0]), "nnz": int(A.nnz), "iters": int(it),
        "relres": float(hist[-1]), "true_relres": float(np.linalg.norm(b - A @ x) / np.linalg.norm(b)),
        "norm_b": float(np.linalg.norm(b)), "norm_x": float(np.linalg.norm(x)),
        "theta": [float(l.theta) for l in levels[1:]],
        "sample_idx": idx, "sample_x": [[float(x[i].real), float(x[i].imag)] for i in idx],
        "sketch_seed": SKETCH_SEED, "sketch_rows": SKETCH_ROWS,
        "sketch_x": [[float(v.real), float(v.imag)] for v in sketch(x)],
        "residual_history": [float(v) for v in hist],
        "oracle_seconds": {"elements": t1 - t0, "hierarchy": t2 - t1, "pcg": t3 - t2},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("iters", "relres", "theta", "oracle_seconds")}))


if __name__ == "__main__":
    main()
