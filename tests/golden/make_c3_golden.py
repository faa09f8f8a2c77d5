"""Writes tests/golden/c3_oracle.json: full-size oracle reference values of the
layered-medium workload ([0,2]x[0,2]x[0,1], 32x32x16 hexahedra, p = 3,
omega = 20 pi, 6 seeded layers, 4 levels p3 -> p2 -> h -> h, FP64 V-cycle,
tol 1e-8).

Calls only oracle/ (and the seeded workload generator).  The element loop is
distributed over processes; each element is computed by the oracle's own
dpg_element / condense, unchanged (the helpers are those of
make_c2_golden.py).  Run: python tests/golden/make_c3_golden.py
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

from make_c2_golden import SKETCH_ROWS, SKETCH_SEED, _elem, _init, sketch  # noqa: E402
from oracle.assembly import FineSystem  # noqa: E402
from oracle.hierarchy import build_hierarchy  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from oracle.solver import mg_pcg  # noqa: E402
from paper_2304_01728_gb300 import workloads  # noqa: E402


def main():
    w = workloads.config3("fp64")
    pk, ok = w["problem"], w["opts"]
    t0 = time.time()
    mesh = Mesh(pk["n"], pk["p"], pk["x0"], pk["x1"])
    fs = FineSystem(mesh, pk["omega"], np.asarray(pk["wavespeed"]), None, elements=[])
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
    rng = np.random.default_rng(2025)
    idx = sorted(rng.choice(A.shape[0], 64, replace=False).tolist())
    out = {
        "workload": w["name"], "n_dof": int(A.shape[0]), "nnz": int(A.nnz), "iters": int(it),
        "relres": float(hist[-1]), "true_relres": float(np.linalg.norm(b - A @ x) / np.linalg.norm(b)),
        "norm_b": float(np.linalg.norm(b)), "norm_x": float(np.linalg.norm(x)),
        "theta": [float(l.theta) for l in levels[1:]],
        "level_dofs": [int(l.mesh.n_dof) for l in levels],
        "sample_idx": idx, "sample_x": [[float(x[i].real), float(x[i].imag)] for i in idx],
        "sketch_seed": SKETCH_SEED, "sketch_rows": SKETCH_ROWS,
        "sketch_x": [[float(v.real), float(v.imag)] for v in sketch(x)],
        "residual_history": [float(v) for v in hist],
        "oracle_seconds": {"elements": t1 - t0, "hierarchy": t2 - t1, "pcg": t3 - t2},
    }
    with open(os.path.join(HERE, "c3_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("iters", "relres", "theta", "oracle_seconds")}))


if __name__ == "__main__":
    main()
