"""Adds to tests/golden/c3_oracle.json the oracle's converged solution of the
layered-medium workload (the same FP64 hierarchy, PCG to relative residual
1e-12): its sign sketch and the relative L2 distance of the stored tol-1e-8
solution to it, i.e. how far the oracle's own iterate at the workload's
tolerance is from the discrete solution.

Calls only oracle/ (and the seeded workload generator); the element loop is
spread over processes as in make_c3_golden.py.  Run after make_c3_golden.py:
python tests/golden/make_c3_converged.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

from make_c2_golden import _elem, _init, sketch  # noqa: E402
from oracle.assembly import FineSystem  # noqa: E402
from oracle.hierarchy import build_hierarchy  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from oracle.solver import mg_pcg  # noqa: E402
from paper_2304_01728_gb300 import workloads  # noqa: E402

TOL_CONVERGED = 1e-12


def main():
    path = os.path.join(HERE, "c3_oracle.json")
    gold = json.load(open(path))
    w = workloads.config3("fp64")
    pk, ok = w["problem"], w["opts"]
    t0 = time.time()
    mesh = Mesh(pk["n"], pk["p"], pk["x0"], pk["x1"])
    fs = FineSystem(mesh, pk["omega"], np.asarray(pk["wavespeed"]), None, elements=[])
    with mp.get_context("spawn").Pool(int(os.environ.get("WORKERS", os.cpu_count())), initializer=_init,
                                      initargs=(pk,)) as pool:
        for e, Kc, Fc in pool.imap_unordered(_elem, range(mesh.n_elem), chunksize=16):
            fs.Kc[e], fs.Fc[e] = Kc, Fc
    A, b = fs.assemble()
    levels = build_hierarchy(mesh, fs.Kc, fs.dofs, ok["n_levels"], ok["p_min"])
    t1 = time.time()
    x8, it8, _ = mg_pcg(levels, A, b, tol=ok["tol"])
    xc, itc, hist = mg_pcg(levels, A, b, tol=TOL_CONVERGED, max_iter=5000)
    t2 = time.time()
    assert it8 == gold["iters"]
    gold.update({
        "converged_tol": TOL_CONVERGED, "converged_iters": int(itc), "converged_relres": float(hist[-1]),
        "converged_norm_x": float(np.linalg.norm(xc)),
        "converged_sketch_x": [[float(v.real), float(v.imag)] for v in sketch(xc)],
        "tol_solution_distance_to_converged": float(np.linalg.norm(x8 - xc) / np.linalg.norm(xc)),
        "converged_oracle_seconds": {"setup": t1 - t0, "pcg_both": t2 - t1},
    })
    with open(path, "w") as f:
        json.dump(gold, f, indent=1)
    print(json.dumps({k: gold[k] for k in ("converged_iters", "converged_relres",
                                           "tol_solution_distance_to_converged")}))


if __name__ == "__main__":
    main()
