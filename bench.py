#!/usr/bin/env python3
"""Benchmark of the DPG-MG solver (MG-preconditioned CG on the condensed DPG trace system).

One step = one pass of the whole hot path through the C ABI: dpgmg_setup
(batched element DPG work, assembly, hierarchy, patch factorisations,
coarsest factor) + dpgmg_solve (PCG to relative residual 1e-8, field
recovery) + dpgmg_release.  Default workload: the layered medium, the
largest single-GPU configuration ([0,2]x[0,2]x[0,1], 32x32x16 hexahedra,
p = 3, omega = 20 pi, 6 seeded layers, 4 levels p3 -> p2 -> h -> h, mixed
V-cycle, FP64 CG); --config 2 runs the 16^3 unit cube instead.

value  = DOF-iterations per second of the PCG phase (N_dof * iterations /
         PCG device time), summed over ranks; ms_per_step is the whole step.
e2e    = the same metric with the end-to-end time of setup + solve through the
         public API with host input and output buffers (copies included).
roofline: the finest-level smoother product kernel, timed live with CUDA
         events on the library's stream inside the timed steps.
cpu_baseline: the FP64 oracle (test infrastructure) on a bounded sample of
         the same workload (a sub-box of its mesh around the source with the
         same h, p, omega, wavespeeds and hierarchy shape), PCG phase timed,
         on one core and as one replica per host core.
Extra keys: error of each precision option against the oracle's full-size
solution (tests/golden), the 16^3 workload's numbers, and bounded
serving/batching summaries.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
       [--config 2|3] [--precision mixed|fp64] [--no-extras]
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-iters/s of MG-PCG to rel. residual 1e-8"
UNIT = "DOF-iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys (oracle errors per option, the 16^3 workload, serving/batch)")
    ap.add_argument("--n", type=int, default=0, help="override the mesh size n^3 (profiling of a smaller case)")
    ap.add_argument("--cuda-cores", action="store_true",
                    help="coarsest complex64 factorisation on the FP32 CUDA cores (DPGMG_FLAG_CUDA_CORES) "
                         "instead of the tensor cores")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "sweep"],
                    help="step: the bench line; batch: independent uneven problems; serve: Poisson request stream; "
                         "sweep: iteration counts of the convergence studies (h, p, omega, smoothing steps)")
    ap.add_argument("--count", type=int, default=16, help="batch/serve: problems drawn from the seeded stream")
    ap.add_argument("--max-dofs", type=float, default=2.5e5, help="batch/serve: sample only problems up to this size")
    ap.add_argument("--slots", type=int, default=4, help="batch/serve: concurrent serving slots")
    ap.add_argument("--rate", type=float, default=0.0, help="serve: arrival rate in requests/s (0: all at t = 0)")
    ap.add_argument("--budget-gb", type=float, default=160.0, help="batch/serve: device-memory admission budget")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-steps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-all-cores", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload(cfg, precision):
    from paper_2304_01728_gb300 import workloads
    return {1: workloads.config1, 2: lambda: workloads.config2(precision),
            3: lambda: workloads.config3(precision)}[cfg]()


# ------------------------------------------------------------------ oracle
def oracle_sample_problem(w, cfg):
    """A sub-box of the workload mesh around the source, with the same element
    size, order, frequency, wavespeeds and hierarchy shape: 8x8x4 elements and
    4 levels (p3 -> p2 -> h -> h) for the layered medium, 4^3 elements and 3
    levels for the unit cube."""
    pk = dict(w["problem"])
    n = pk["n"]
    x0 = pk.get("x0", (0, 0, 0))
    x1 = pk.get("x1", (1, 1, 1))
    h = [(x1[d] - x0[d]) / n[d] for d in range(3)]
    sub = [min(8, n[0]), min(8, n[1]), min(4, n[2])] if cfg == 3 else [min(4, n[d]) for d in range(3)]
    lo, hi, start = [], [], []
    for d in range(3):
        c = int(round((pk["src_center"][d] - x0[d]) / h[d])) - sub[d] // 2
        c = max(0, min(n[d] - sub[d], c))
        start.append(c)
        lo.append(x0[d] + c * h[d])
        hi.append(x0[d] + (c + sub[d]) * h[d])
    ws = pk.get("wavespeed")
    wsub = None
    if ws is not None:
        wsub = [ws[(start[0] + kx) + n[0] * ((start[1] + ky) + n[1] * (start[2] + kz))]
                for kz in range(sub[2]) for ky in range(sub[1]) for kx in range(sub[0])]
    levels = min(w["opts"]["n_levels"], 4 if cfg == 3 else 3)
    return dict(n=tuple(sub), p=pk["p"], omega=pk["omega"], x0=tuple(lo), x1=tuple(hi), wavespeed=wsub,
                src_center=pk["src_center"], src_width=pk["src_width"]), dict(w["opts"], n_levels=levels)


_ORC = {}


def _orc_init(pk):
    from oracle.mesh import Mesh
    from oracle.problem import GaussianSource
    _ORC.update(pk=pk, mesh=Mesh(pk["n"], pk["p"], pk["x0"], pk["x1"]),
                load=GaussianSource(pk["src_center"], pk["src_width"]))


def _orc_elem(e):
    """One element of the oracle's FineSystem, by the oracle's own functions."""
    import numpy as np
    from oracle.element import boundary_faces, condense, dpg_element
    pk, m = _ORC["pk"], _ORC["mesh"]
    bf = boundary_faces(m, e)
    corner = m.x0 + np.asarray(m.elem_coord(e)) * m.h
    c = 1.0 if pk["wavespeed"] is None else pk["wavespeed"][e]
    K, F = dpg_element(m.p, m.h, corner, c, pk["omega"], bf, _ORC["load"])
    Kc, Fc = condense(m.p, K, F, bf)
    return e, Kc, Fc


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_run(args):
    """Runs in a fresh process without a GPU: the oracle's setup of the sample
    (untimed; its element loop over a spawned process pool), then its PCG
    phase timed on one core (--oracle-steps times), then, with
    --oracle-all-cores, once in each of one forked single-threaded replica per
    host core at the same time."""
    import multiprocessing as mp
    from oracle.assembly import FineSystem
    from oracle.hierarchy import build_hierarchy
    from oracle.mesh import Mesh
    from oracle.solver import mg_pcg
    w = workload(args.config, "fp64")
    pk, ok = oracle_sample_problem(w, args.config)
    t0 = time.perf_counter()
    mesh = Mesh(pk["n"], pk["p"], pk["x0"], pk["x1"])
    fs = FineSystem(mesh, pk["omega"], pk["wavespeed"], None, elements=[])
    ncpu = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(min(ncpu, 32), initializer=_orc_init, initargs=(pk,)) as pool:
        for e, Kc, Fc in pool.imap_unordered(_orc_elem, range(mesh.n_elem), chunksize=4):
            fs.Kc[e], fs.Fc[e] = Kc, Fc
    A, b = fs.assemble()
    levels = build_hierarchy(fs.mesh, fs.Kc, fs.dofs, ok["n_levels"], ok["p_min"])
    t_setup = time.perf_counter() - t0
    res = []
    for _ in range(args.oracle_steps):
        t1 = time.perf_counter()
        x, it, hist = mg_pcg(levels, A, b, tol=ok["tol"])
        res.append((time.perf_counter() - t1, it))
    n = A.shape[0]
    tot_t = sum(r[0] for r in res)
    tot_di = sum(n * r[1] for r in res)
    all_core = None
    if args.oracle_all_cores and ncpu > 1 and hasattr(os, "fork"):
        t1 = time.perf_counter()
        pids = []
        for _ in range(ncpu):
            pid = os.fork()
            if pid == 0:
                try:
                    mg_pcg(levels, A, b, tol=ok["tol"])
                    os._exit(0)
                except BaseException:
                    os._exit(1)
            pids.append(pid)
        ok_all = all(os.waitpid(pid, 0)[1] == 0 for pid in pids)
        wall = time.perf_counter() - t1
        if ok_all:
            all_core = dict(value=ncpu * n * res[-1][1] / wall, cores=ncpu, wall_s=wall)
    print(json.dumps(dict(value=tot_di / tot_t, n_dof=n, iters=res[-1][1], pcg_s=[r[0] for r in res],
                          setup_s=t_setup, all_core=all_core, nproc=ncpu, cpu_model=cpu_model(),
                          sample="%dx%dx%d-element sub-box [%s]-[%s] of the %s mesh (same h, p=%d, omega, "
                          "wavespeeds and source), %d levels, oracle setup untimed, PCG phase timed" % (
                              pk["n"][0], pk["n"][1], pk["n"][2], ",".join("%.4g" % v for v in pk["x0"]),
                              ",".join("%.4g" % v for v in pk["x1"]), "x".join(map(str, w["problem"]["n"])),
                              pk["p"], ok["n_levels"]))))


def oracle_subprocess(args, steps=1, timeout=900, all_cores=False):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--config", str(args.config),
           "--oracle-steps", str(steps)] + (["--oracle-all-cores"] if all_cores else [])
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def golden_for(cfg):
    """The oracle's full-size reference of a workload (tests/golden, written by
    oracle-only scripts), or None."""
    path = os.path.join(ROOT, "tests", "golden", {2: "c2_oracle.json", 3: "c3_oracle.json"}.get(cfg, "-"))
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def sketch_error(x, gold, key="sketch_x", norm_key="norm_x"):
    """Relative L2 distance of the trace vector x (complex128) to an oracle
    solution (its tolerance-1e-8 solve, or with key "converged_sketch_x" its
    solve to 1e-12), estimated from the stored seeded sign sketch."""
    import numpy as np
    from paper_2304_01728_gb300 import workloads
    if key not in gold:
        return None
    sk = np.empty(gold["sketch_rows"], complex)
    for j0 in range(0, gold["sketch_rows"], 16):
        sk[j0:j0 + 16] = workloads.rademacher_rows(gold["sketch_seed"], j0, j0 + 16, x.size) @ x
    skr = np.array([complex(*v) for v in gold[key]])
    return float(np.linalg.norm(sk - skr) / np.sqrt(gold["sketch_rows"]) / gold[norm_key])


def converged_distance(x, gold):
    return sketch_error(x, gold, "converged_sketch_x", "converged_norm_x")


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def reduce_ranks(dist, dof_iters, pcg_ms, total_ms, device):
    """Replicas only: work adds up over ranks, time is the slowest rank's."""
    import torch
    s = torch.tensor([dof_iters], dtype=torch.float64, device=device)
    m = torch.tensor([pcg_ms, total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(s[0]), float(m[0]), float(m[1])


# ------------------------------------------------------------------ gb300
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


def traffic_for(kernel, bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary (the captured
    launch's DRAM bytes per algorithmic byte, times this launch's algorithmic
    bytes), if the kernel source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except OSError:
        return None
    e = d.get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if e.get("source_sha") != sha:
        return None
    ratio = e.get("ratio_traffic_to_algorithmic")
    return ratio * bytes_per_launch if ratio else None


FP64_PEAK_TFLOPS = 1.20   # measured FP64 FMA rate of one GB300 (8 independent FMA chains per thread)


def element_line(acc, full_gflop):
    """Roofline line of the batched element stage (FP64 arithmetic): the
    fraction uses the flops the stage executed; with element classes that is
    far below the flops of the full per-element pipeline, reported beside it."""
    ms, gflop, n = acc
    if not n or ms <= 0:
        return None
    tf = gflop / (ms / 1e3) / 1e3
    return {"kernels": "k_elem_build/potrf/trsm/herk/condense/member_load", "bound": "alu", "achieved": tf,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
            "peak_source": "measured FP64 FMA rate (nominal 1.25)", "executed_gflop_per_setup": gflop / n,
            "full_pipeline_gflop_per_setup": full_gflop, "ms_per_setup": ms / n}


def full_pipeline_gflop(n_elem, p):
    """Algorithmic GFLOP of the element stage if every element ran the whole
    pipeline (the per-element counts of dpgmg_setup_profile)."""
    nt = (p + 2) ** 3 + 3 * (p + 2) * (p + 1) ** 2
    nf = 4 * p ** 3
    ntr = (p + 1) ** 3 - (p - 1) ** 3 + 6 * p * p
    m = nf + ntr
    mac = nt ** 3 / 6 + nt ** 2 * (m + 1) / 2 + (m + 1) ** 2 * nt / 2 + nf ** 3 / 6 + nf ** 2 * (ntr + 1) + \
        ntr * (ntr + 1) * nf
    return 8.0 * mac * n_elem / 1e9


def run_gb300(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2304_01728_gb300 import build as B
    B.build()
    from paper_2304_01728_gb300 import dpgmg as D

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = workload(args.config, args.precision)
    if args.n:
        w["problem"]["n"] = (args.n,) * 3
        w["name"] += " (mesh overridden to %d^3)" % args.n
    if args.cuda_cores:
        w["opts"]["flags"] = w["opts"].get("flags", 0) | D.FLAG_CUDA_CORES
        w["name"] += ", coarsest factor on CUDA cores"
    stream = torch.cuda.Stream()
    h = D.dpgmg_create(local_rank, 0, ctypes.c_void_p(stream.cuda_stream))
    pb, keep = D.make_problem(**w["problem"])
    op = D.make_opts(**w["opts"])
    n_dof, n_field, dev_bytes = D.dpgmg_query_sizes(pb, op)
    trace = torch.empty(2 * n_dof, dtype=torch.float64, device="cuda")
    fields = torch.empty(2 * n_field, dtype=torch.float64, device="cuda")

    tuned = {}
    elem_acc = [0.0, 0.0, 0]   # element-stage ms, GFLOP, setups
    phases = []                # device ms of each setup phase, per step
    patch_store = {}           # finest level: sum n_j^2, and over the real packed patches

    def step(prof=D.PROF_OFF):
        s = D.dpgmg_setup(h, pb, op)
        try:
            for l in range(1, w["opts"]["n_levels"]):
                try:
                    tuned["level%d" % l] = D.dpgmg_spmv_group(h, s, l)
                except D.DpgmgError:
                    break
            tuned["cg"] = D.dpgmg_spmv_group(h, s, -1)
            li = D.dpgmg_level_info(h, s, w["opts"]["n_levels"] - 1)
            patch_store.update(sum_patch_sq=int(li.sum_patch_sq), real_sq=int(li.patch_real_sq),
                               op_nnz=int(li.op_nnz), op_real_nnz=int(li.op_real_nnz))
            em, eg, _ = D.dpgmg_setup_profile(h, s)
            phases.append(D.dpgmg_setup_phases(h, s))
            elem_acc[0] += em
            elem_acc[1] += eg
            elem_acc[2] += 1
            if prof:
                D.dpgmg_profile(h, s, prof)
            code, st = D.dpgmg_solve(h, s, trace.data_ptr(), fields.data_ptr(), out_is_device=True)
            if code != D.DPGMG_OK:
                raise RuntimeError("solve status %s" % D.strerror(code))
            pr = D.dpgmg_profile_read(h, s) if prof else None
            return st, pr
        finally:
            D.dpgmg_release(h, s)

    for _ in range(args.warmup):
        step()
    elem_acc[:] = [0.0, 0.0, 0]
    phases.clear()
    clocks = Clocks(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = D.dpgmg_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats, prof_ms, prof_n, prof_b = [], 0.0, 0, 0
    # profiler range = the timed steps (ncu --profile-from-start off); no-op otherwise
    torch.cuda.profiler.start()
    for _ in range(args.steps):
        st, pr = step(D.PROF_SMOOTH_FINE)
        stats.append((st.iters, st.t_pcg_ms, st.t_setup_ms, st.true_relres, st.relres, st.bytes_per_iter))
        prof_ms += pr[0]
        prof_n += pr[1]
        prof_b = pr[2]
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    launches = D.dpgmg_launch_count() - l0
    elem_acc_timed = list(elem_acc)
    gold = golden_for(args.config) if not args.n else None
    err_main = sketch_error(trace.cpu().numpy().view(np.complex128), gold) if gold else None
    conv_main = converged_distance(trace.cpu().numpy().view(np.complex128), gold) if gold else None
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    dof_iters = float(sum(n_dof * s[0] for s in stats))
    pcg_ms = float(sum(s[1] for s in stats))
    if dist:
        dof_iters, pcg_ms, total_ms = reduce_ranks(dist, dof_iters, pcg_ms, total_ms, "cuda")
    value = dof_iters / (pcg_ms / 1e3)

    # ---- the other HBM-bound kernels of the iteration, one profiled step each
    kernels = []
    for prof, name in ((D.PROF_SPMV_FINE, "k_spmv (finest V-cycle SpMV, c64 values)"),
                       (D.PROF_SPMV_CG, "k_spmv_df (CG operator, c64 hi + lo values)")):
        _, pr = step(prof)
        ms = pr[0] / max(pr[1], 1)
        gbs = pr[2] / (ms / 1e3) / 1e9
        kernels.append({"kernel": name, "bytes_per_launch": pr[2], "launches": pr[1], "avg_launch_ms": ms,
                        "achieved": gbs, "unit": "GB/s",
                        "bytes_rule": "stored values read once: complex64 8 B per entry (CG operator: high + "
                                      "low parts, 16 B), real packed rows half of that",
                        "real_packed_fraction_of_entries": (patch_store["op_real_nnz"] / patch_store["op_nnz"]
                                                            if patch_store.get("op_nnz") else None)})

    # ---- end to end through the public API with host buffers
    e2e = None
    nelem = int(np.prod(w["problem"]["n"]))
    steps_e2e = 0 if args.no_e2e else args.steps
    c_host = np.ascontiguousarray(w["problem"].get("wavespeed") or np.ones(nelem), dtype=np.float64)
    c_pin = torch.from_numpy(c_host).pin_memory()
    pk2 = dict(w["problem"], wavespeed=None)
    pb2, keep2 = D.make_problem(**pk2)
    pb2.wavespeed = ctypes.cast(ctypes.c_void_p(c_pin.data_ptr()), ctypes.POINTER(ctypes.c_double))
    tr_h = torch.empty(2 * n_dof, dtype=torch.float64).pin_memory()
    fl_h = torch.empty(2 * n_field, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_di = 0.0
    for _ in range(steps_e2e):
        s = D.dpgmg_setup(h, pb2, op)
        code, st = D.dpgmg_solve(h, s, tr_h.data_ptr(), fl_h.data_ptr(), out_is_device=False)
        D.dpgmg_release(h, s)
        e2e_di += n_dof * st.iters
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    if steps_e2e:
        e2e = {"value": e2e_di / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(c_host.nbytes),
               "d2h_bytes_per_step": int(16 * (n_dof + n_field)), "ms_per_step": 1e3 * t_e2e / steps_e2e}

    # ---- FP64 V-cycle path on the same workload (one step, reported beside)
    def one(opts_kw):
        s = D.dpgmg_setup(h, pb, D.make_opts(**dict(w["opts"], **opts_kw)))
        code, st = D.dpgmg_solve(h, s, trace.data_ptr(), fields.data_ptr(), out_is_device=True)
        D.dpgmg_release(h, s)
        r = {"value": n_dof * st.iters / (st.t_pcg_ms / 1e3), "iters": st.iters, "pcg_ms": st.t_pcg_ms,
             "setup_ms": st.t_setup_ms, "true_relres": st.true_relres, "status": D.strerror(code)}
        if gold:
            r["rel_l2_error_vs_oracle"] = sketch_error(trace.cpu().numpy().view(np.complex128), gold)
            r["rel_l2_distance_to_converged"] = converged_distance(trace.cpu().numpy().view(np.complex128), gold)
        return r

    fp64 = None
    options = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        fp64 = one(dict(precision="fp64"))
        if not args.no_extras:
            # the CG operator's two forms (Sec. 3 runs CG on the FP64 condensed system):
            # double-float (the default, timed above) and complex128 on the FP64 pipe; the
            # FP64 V-cycle with the complex128 CG operator is complex128 throughout
            options = {"mixed_cg_double_float": {"rel_l2_error_vs_oracle": err_main,
                                                 "rel_l2_distance_to_converged": conv_main,
                                                 "pcg_ms": pcg_ms / args.steps, "iters": stats[-1][0]},
                       "mixed_cg_c128": one(dict(flags=D.FLAG_CG_C128)),
                       "fp64_cg_double_float": fp64,
                       "fp64_cg_c128": one(dict(precision="fp64", flags=D.FLAG_CG_C128)),
                       "mixed_patch_factors_fp64": one(dict(flags=D.FLAG_PATCH_FP64)),
                       "mixed_coarsest_cuda_cores": one(dict(flags=D.FLAG_CUDA_CORES)),
                       "mixed_all_complex64_storage": one(dict(flags=D.FLAG_COMPLEX_STORAGE))}
    D.dpgmg_destroy(h)


    if rank != 0:
        return None
    peak, peak_kind = peaks()
    per_launch_ms = prof_ms / max(prof_n, 1)
    achieved = prof_b / (per_launch_ms / 1e3) / 1e9
    it_last = stats[-1]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 V-cycle / c128 CG" if args.precision == "mixed" else "c128",
        "data": "synthetic (seeded Gaussian source; no dataset)",
        "config": {"workload": w["name"], "n": list(w["problem"]["n"]), "p": w["problem"]["p"],
                   "omega": w["problem"]["omega"], "levels": w["opts"]["n_levels"], "precision": args.precision,
                   "n_dof": n_dof, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "operators (GBs) exceed L2; no flush needed"},
        "iters": it_last[0], "pcg_ms": pcg_ms / args.steps, "setup_ms": sum(s[2] for s in stats) / args.steps,
        "true_relres": it_last[3], "relres": it_last[4], "bytes_per_iter": it_last[5],
        "pcg_GBps": it_last[5] * it_last[0] / (stats[-1][1] / 1e3) / 1e9,
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_patch_apply (finest smoother)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "bytes_per_launch": prof_b, "launches": prof_n, "avg_launch_ms": per_launch_ms,
                     "bytes_rule": "stored patch-inverse entries read once: 8 B per complex64 entry, 4 B per "
                                   "entry of a real packed block",
                     "real_packed_fraction_of_entries": (patch_store["real_sq"] / patch_store["sum_patch_sq"]
                                                         if patch_store.get("sum_patch_sq") else None),
                     "traffic": traffic_for("k_patch_apply", prof_b),
                     "traffic_source": "not measured in this run: ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                       "per algorithmic byte of the finest launches of one step of the "
                                       "32x32x16 layered workload (profiles/traffic.json) times this "
                                       "launch's algorithmic bytes; null once the kernel source has changed"},
        "clocks": clk, "e2e": e2e, "fp64_path": fp64,
        "rel_l2_error_vs_oracle": err_main,
        "rel_l2_distance_to_converged": conv_main,
        "oracle_reference": ({"iters": gold["iters"], "n_dof": gold["n_dof"],
                              "tol_solution_distance_to_converged": gold.get("tol_solution_distance_to_converged"),
                              "converged_iters": gold.get("converged_iters"),
                              "source": "tests/golden/%s (full-size FP64 oracle run; errors estimated from its "
                                        "128-row seeded sign sketch)" % {2: "c2_oracle.json", 3: "c3_oracle.json"}[
                                            args.config]} if gold else None),
        "precision_options": options,
        "kernels": [dict(k, frac=k["achieved"] / peak) for k in kernels],
        "spmv_group_tuned": tuned,
        "setup_phases_ms": ({k: sum(p[i] for p in phases) / len(phases) for i, k in enumerate(D.SETUP_PHASES)}
                            if phases else None),
        "element_stage": element_line(elem_acc_timed, full_pipeline_gflop(int(np.prod(w["problem"]["n"])),
                                                                          w["problem"]["p"])),
    }
    return out


# ------------------------------------------------------------------ batch / serve
def run_stream(args):
    """Independent problems through the serving loop (continuous batching).

    batch: the first --count problems of the seeded uneven batch stream, all
    submitted at t = 0.  serve: the first --count requests of the seeded
    serving stream, submitted at Poisson arrival times (--rate requests/s).
    Problems above --max-dofs are left out of the sample (stated in the output);
    requests whose footprint exceeds the memory budget are refused (NOMEM).
    """
    import numpy as np
    from paper_2304_01728_gb300 import build as B
    B.build()
    from paper_2304_01728_gb300 import dpgmg as D
    from paper_2304_01728_gb300 import workloads as WL
    prec = args.precision
    stream = WL.config4(64, prec) if args.mode == "batch" else WL.config5(max(args.count, 1), prec)
    drawn = stream[:args.count]
    h = D.dpgmg_create(0, int(args.budget_gb * 1e9))
    D.dpgmg_serve_start(h, args.slots)
    sample, skipped = [], 0
    for it in drawn:
        pb, keep = D.make_problem(**it["problem"])
        op = D.make_opts(**it["opts"])
        nt, nf, est = D.dpgmg_query_sizes(pb, op)
        if nt > args.max_dofs:
            skipped += 1
            continue
        sample.append((it, pb, op, keep, nt, nf))
    t_arr, t = [], 0.0
    for it, *_ in sample:
        t += (it.get("gap", 0.0) / args.rate) if (args.mode == "serve" and args.rate > 0) else 0.0
        t_arr.append(t)
    tickets, refused, per = [], 0, []
    t0 = time.perf_counter()
    for (it, pb, op, keep, nt, nf), ta in zip(sample, t_arr):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0005)
        rec = {"n": it["problem"]["n"][0], "p": it["problem"]["p"], "omega": round(it["problem"]["omega"], 3),
               "dofs": nt, "est_gb": round(D.dpgmg_query_sizes(pb, op)[2] / 1e9, 2)}
        per.append(rec)
        try:
            tickets.append((D.dpgmg_submit(h, pb, op), nt, nf, rec))
        except D.DpgmgError as e:
            if e.code != D.DPGMG_ERR_NOMEM:
                raise
            refused += 1
            rec["status"] = "refused (NOMEM)"
    lat, dof_iters, iters, fails = [], 0.0, [], 0
    for tk, nt, nf, rec in tickets:
        x = np.zeros(nt, dtype=np.complex128)
        f = np.zeros(nf, dtype=np.complex128)
        while True:
            code, st, l = D.dpgmg_poll(h, tk, x, f)
            if code != D.DPGMG_ERR_PENDING:
                break
            time.sleep(0.001)
        rec["status"] = D.strerror(code)
        if code != D.DPGMG_OK:
            fails += 1
            continue
        rec.update(iters=st.iters, latency_ms=round(l, 1), setup_ms=round(st.t_setup_ms, 1),
                   pcg_ms=round(st.t_pcg_ms, 2))
        lat.append(l)
        dof_iters += nt * st.iters
        iters.append(st.iters)
    wall = time.perf_counter() - t0
    D.dpgmg_destroy(h)
    done = len(lat)
    out = {"mode": args.mode, "metric": "solves/s", "value": done / wall, "unit": "solve/s",
           "dof_iters_per_s": dof_iters / wall, "p50_ms": float(np.percentile(lat, 50)) if lat else None,
           "p99_ms": float(np.percentile(lat, 99)) if lat else None, "completed": done, "failed": fails,
           "refused_nomem": refused, "drawn": len(drawn), "left_out_above_max_dofs": skipped,
           "max_dofs": args.max_dofs, "slots": args.slots, "rate_per_s": args.rate, "precision": prec,
           "budget_gb": args.budget_gb, "requests": per,
           "wall_s": wall, "iters_mean": float(np.mean(iters)) if iters else None,
           "sample": "first %d problems of the seeded %s stream, those with <= %g trace DOFs" % (
               len(drawn), "batch (n~U{8..24}, p~U{2,3,4})" if args.mode == "batch" else
               "serving (n~U{8..48}, p~U{2..5})", args.max_dofs)}
    print(json.dumps(out))


# ------------------------------------------------------------------ sweep
def run_sweep(args):
    """Iteration counts of the convergence studies (Sec. 4: h-robustness at
    fixed omega, growth with omega, p-robustness, smoothing steps), with
    restricted and stored coarse operators, on the unit cube with a Gaussian
    source (x0 = (0.45, 0.5, 0.55), sigma = 0.1), mixed V-cycle, tol 1e-8.
    Prints one JSON line with a row per solve (iterations, PCG and setup ms)."""
    from paper_2304_01728_gb300 import build as B
    B.build()
    from paper_2304_01728_gb300 import dpgmg as D
    pi = math.pi
    studies = []
    for n in (4, 8, 16):                               # h at fixed omega (2 elements per wavelength at n = 16)
        studies.append(("h", n, 3, 8 * pi, 1))
    for om in (4 * pi, 8 * pi, 12 * pi, 16 * pi):      # omega at fixed mesh
        studies.append(("omega", 16, 3, om, 1))
    for p in (2, 3, 4):                                # p at fixed mesh and omega
        studies.append(("p", 8, p, 8 * pi, 1))
    for nu in (1, 2, 3):                               # V(nu, nu)
        studies.append(("nu", 16, 3, 8 * pi, nu))
    rows = []
    for study, n, p, om, nu in studies:
        row = {"study": study, "n": n, "p": p, "omega": round(om, 4), "nu": nu}
        for name, flags in (("restricted", 0), ("stored", D.FLAG_STORE_COARSE)):
            pk = dict(n=(n, n, n), p=p, omega=om, src_center=(0.45, 0.5, 0.55), src_width=0.1)
            opts = dict(n_levels=3, p_min=2 if p > 2 else 1, precision="mixed", tol=1e-8, flags=flags,
                        nu_pre=nu, nu_post=nu, max_iter=3000)
            with D.Solver(pk, **opts) as s:
                x, f, st, code = s.solve(fields=False)
            row[name] = {"iters": st.iters, "pcg_ms": round(st.t_pcg_ms, 2), "setup_ms": round(st.t_setup_ms, 1),
                         "status": D.strerror(code)}
        rows.append(row)
    print(json.dumps({"mode": "sweep", "levels": 3, "precision": "mixed", "tol": 1e-8, "rows": rows}))



# ------------------------------------------------------------------ extras
def c2_summary(args, D):
    """The 16^3, p = 3, omega = 16 pi unit-cube workload on the same GPU:
    PCG DOF-iter/s, setup, end to end through the C ABI with host buffers,
    finest smoother bandwidth, and error against the oracle's full-size run."""
    import numpy as np
    import torch
    w = workload(2, "mixed")
    stream = torch.cuda.Stream()
    h = D.dpgmg_create(0, 0, ctypes.c_void_p(stream.cuda_stream))
    pb, keep = D.make_problem(**w["problem"])
    op = D.make_opts(**w["opts"])
    n_dof, n_field, _ = D.dpgmg_query_sizes(pb, op)
    tr = torch.empty(2 * n_dof, dtype=torch.float64).pin_memory()
    fl = torch.empty(2 * n_field, dtype=torch.float64).pin_memory()
    res = []
    for k in range(6):
        t0 = time.perf_counter()
        s = D.dpgmg_setup(h, pb, op)
        if k >= 3:
            D.dpgmg_profile(h, s, D.PROF_SMOOTH_FINE)
        code, st = D.dpgmg_solve(h, s, tr.data_ptr(), fl.data_ptr(), out_is_device=False)
        pr = D.dpgmg_profile_read(h, s) if k >= 3 else None
        D.dpgmg_release(h, s)
        torch.cuda.synchronize()
        if k >= 3:
            res.append((st.iters, st.t_pcg_ms, st.t_setup_ms, time.perf_counter() - t0, pr))
    D.dpgmg_destroy(h)
    peak, _ = peaks()
    ms = sum(r[4][0] for r in res) / max(sum(r[4][1] for r in res), 1)
    gold = golden_for(2)
    return {"workload": w["name"], "n_dof": n_dof, "iters": res[-1][0],
            "value": n_dof * sum(r[0] for r in res) / (sum(r[1] for r in res) / 1e3), "unit": UNIT,
            "pcg_ms": sum(r[1] for r in res) / len(res), "setup_ms": sum(r[2] for r in res) / len(res),
            "e2e": {"value": n_dof * sum(r[0] for r in res) / sum(r[3] for r in res), "unit": UNIT,
                    "ms_per_step": 1e3 * sum(r[3] for r in res) / len(res)},
            "smoother_frac_of_hbm": res[-1][4][2] / (ms / 1e3) / 1e9 / peak,
            "rel_l2_error_vs_oracle": sketch_error(tr.numpy().view(np.complex128), gold) if gold else None}


def multi_load_summary(args, D, k=4):
    """Several loads on the headline workload at once (dpgmg_solve_block):
    k Gaussian sources at seeded positions in the source box of the layered
    medium; their condensed loads come from systems set up for each source.
    Aggregate DOF-iter/s of the block solve against k single solves."""
    import numpy as np
    from paper_2304_01728_gb300 import workloads as WL
    w = workload(args.config, "mixed")
    pk, ok = dict(w["problem"]), dict(w["opts"])
    lo, hi = np.array([0.5, 0.5, 0.25]), np.array([1.5, 1.5, 0.75])
    centers = [tuple(lo + (hi - lo) * np.array([WL._u(7, 3 * j + d) for d in range(3)]))
               for j in range(k)]
    h = D.dpgmg_create(0)
    try:
        B, single = [], []
        for c in centers:
            pb, keep = D.make_problem(**dict(pk, src_center=c))
            s = D.dpgmg_setup(h, pb, D.make_opts(**ok))
            B.append(D.dpgmg_rhs(h, s, D.dpgmg_query_sizes(pb, D.make_opts(**ok))[0]))
            x = np.zeros_like(B[-1])
            code, st = D.dpgmg_solve(h, s, x, None)
            single.append((st.iters, st.t_pcg_ms))
            D.dpgmg_release(h, s)
        B = np.array(B)
        pb, keep = D.make_problem(**dict(pk, src_center=centers[0]))
        s = D.dpgmg_setup(h, pb, D.make_opts(**ok))
        runs = []
        for rep in range(3):
            code, X, stats = D.dpgmg_solve_block(h, s, B)
            runs.append((stats[0].t_pcg_ms, [st.iters for st in stats], [st.true_relres for st in stats]))
        D.dpgmg_release(h, s)
    finally:
        D.dpgmg_destroy(h)
    n = B.shape[1]
    t_blk = min(r[0] for r in runs)
    iters = runs[-1][1]
    t_single = sum(t for _, t in single)
    return {"loads": k, "sources": [list(map(float, c)) for c in centers], "n_dof": n,
            "iters": iters, "single_iters": [i for i, _ in single], "true_relres": runs[-1][2],
            "block_pcg_ms": t_blk, "single_pcg_ms_sum": t_single,
            "value": n * sum(iters) / (t_blk / 1e3), "unit": UNIT,
            "single_value": n * sum(i for i, _ in single) / (t_single / 1e3),
            "note": "aggregate over the k loads; block = one dpgmg_solve_block call (best of 3), single = "
                    "k dpgmg_solve calls"}


def element_full_pipeline(args, D):
    """The element stage with every element through the whole pipeline
    (DPGMG_ELEMENT_REUSE=0: no element classes), as on a general mesh: its
    time, executed GFLOP and fraction of the measured FP64 rate, on the
    headline workload (two setups, the second timed)."""
    w = workload(args.config, "mixed")
    old = os.environ.get("DPGMG_ELEMENT_REUSE")
    os.environ["DPGMG_ELEMENT_REUSE"] = "0"
    h = D.dpgmg_create(0)
    try:
        pb, keep = D.make_problem(**w["problem"])
        op = D.make_opts(**w["opts"])
        res = None
        for rep in range(2):
            s = D.dpgmg_setup(h, pb, op)
            res = D.dpgmg_setup_profile(h, s)
            D.dpgmg_release(h, s)
    finally:
        D.dpgmg_destroy(h)
        if old is None:
            os.environ.pop("DPGMG_ELEMENT_REUSE", None)
        else:
            os.environ["DPGMG_ELEMENT_REUSE"] = old
    ms, gflop, _ = res
    tf = gflop / (ms / 1e3) / 1e3
    return {"ms_per_setup": ms, "executed_gflop_per_setup": gflop, "achieved": tf, "unit": "TFLOP/s",
            "peak": FP64_PEAK_TFLOPS, "frac": tf / FP64_PEAK_TFLOPS,
            "note": "DPGMG_ELEMENT_REUSE=0: every element through Gram Cholesky, TRSM, HERK, condensation"}


def stream_run(D, items, rate, slots, budget_gb):
    """Submit the problems at the given arrival times (rate = requests/s,
    exponential gaps of the stream; 0: all at t = 0) to a serving handle and
    collect them; returns latencies (ms), solves/s, DOF-iter/s and statuses."""
    import numpy as np
    h = D.dpgmg_create(0, int(budget_gb * 1e9))
    D.dpgmg_serve_start(h, slots)
    keep, t_arr, t = [], [], 0.0
    for it in items:
        pb, k = D.make_problem(**it["problem"])
        op = D.make_opts(**it["opts"])
        nt, nf, _ = D.dpgmg_query_sizes(pb, op)
        keep.append((pb, op, k, nt, nf))
        t += it.get("gap", 1.0) / rate if rate > 0 else 0.0
        t_arr.append(t)
    tickets, refused = [], 0
    t0 = time.perf_counter()
    for (pb, op, k, nt, nf), ta in zip(keep, t_arr):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0005)
        try:
            tickets.append((D.dpgmg_submit(h, pb, op), nt, nf))
        except D.DpgmgError as e:
            if e.code != D.DPGMG_ERR_NOMEM:
                raise
            refused += 1
    lat, di, fails, codes = [], 0.0, 0, []
    for q, (tk, nt, nf) in enumerate(tickets):
        while True:
            code, st, l = D.dpgmg_poll(h, tk, None, None)
            if code != D.DPGMG_ERR_PENDING:
                break
            time.sleep(0.0005)
        if code != D.DPGMG_OK:
            fails += 1
            codes.append({"request": q, "status": D.strerror(code), "message": D.lib().dpgmg_last_error().decode(),
                          "iters": st.iters, "relres": st.relres, "n_dof": nt})
            continue
        lat.append(l)
        di += nt * st.iters
    wall = time.perf_counter() - t0
    D.dpgmg_destroy(h)
    return {"completed": len(lat), "failed": fails, "failures": codes, "refused_nomem": refused, "wall_s": wall,
            "solves_per_s": len(lat) / wall, "dof_iters_per_s": di / wall,
            "p50_ms": float(np.percentile(lat, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat else None}


def serve_summary(D, precision, count=120, max_dofs=5e4, load=0.8, slots=4):
    """Bounded serving experiment: the first `count` requests of the seeded
    serving stream with at most max_dofs trace DOFs; the single-stream
    capacity is measured first (8 of them one at a time), then all `count`
    arrive as a Poisson stream at load x that capacity."""
    from paper_2304_01728_gb300 import workloads as WL
    items = []
    for it in WL.config5(2000, precision):
        pb, k = D.make_problem(**it["problem"])
        if D.dpgmg_query_sizes(pb, D.make_opts(**it["opts"]))[0] <= max_dofs:
            items.append(it)
        if len(items) == count:
            break
    t0 = time.perf_counter()
    for it in items[:8]:
        with D.Solver(it["problem"], **it["opts"]) as s:
            s.solve(fields=False)
    capacity = 8 / (time.perf_counter() - t0)
    r = stream_run(D, items, load * capacity, slots, 160.0)
    r.update(precision=precision, requests=len(items), rate_per_s=load * capacity,
             single_stream_capacity_per_s=capacity, load=load, slots=slots,
             sample="first %d requests of the seeded serving stream (n~U{8..48}, p~U{2..5}, omega~U[4,32pi], "
                    "constant or 4-layer wavespeed) with <= %d trace DOFs; Poisson arrivals at %.1fx the "
                    "measured one-at-a-time capacity" % (len(items), max_dofs, load))
    return r


def batch_summary(D, count=24, max_dofs=1.5e5, slots=4):
    """Bounded batch: the first `count` problems of the seeded uneven batch
    stream with at most max_dofs trace DOFs, all submitted at t = 0 (mixed)."""
    from paper_2304_01728_gb300 import workloads as WL
    items = []
    for it in WL.config4(64, "mixed"):
        pb, k = D.make_problem(**it["problem"])
        if D.dpgmg_query_sizes(pb, D.make_opts(**it["opts"]))[0] <= max_dofs:
            items.append(it)
        if len(items) == count:
            break
    r = stream_run(D, items, 0.0, slots, 160.0)
    r.update(problems=len(items), slots=slots,
             sample="first %d problems of the seeded batch stream (n~U{8..24}, p~U{2,3,4}, omega~U[4,12pi]) "
                    "with <= %d trace DOFs, all submitted at t = 0" % (len(items), max_dofs))
    return r


# ------------------------------------------------------------------ main
def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_run(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm is the FP64 oracle (no reference implementation exists)
        t0 = time.perf_counter()
        r = oracle_subprocess(args, steps=args.warmup + args.steps, timeout=1800)
        pcg = r["pcg_s"][args.warmup:]
        value = r["n_dof"] * r["iters"] * len(pcg) / sum(pcg)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(pcg) / len(pcg),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": workload(args.config, args.precision)["name"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}))
        return
    if args.mode == "sweep":
        if rank == 0:
            run_sweep(args)
        return
    if args.mode != "step":
        if rank == 0:
            run_stream(args)
        return
    out = run_gb300(args, rank, world, local_rank)
    if out is None:
        return
    if world == 1 and not args.no_extras and args.mode == "step" and not args.n:
        from paper_2304_01728_gb300 import dpgmg as D
        if args.config != 2:
            out["unit_cube_16cubed"] = c2_summary(args, D)
        out["multi_load"] = multi_load_summary(args, D)
        if out.get("element_stage"):
            out["element_stage"]["full_pipeline"] = element_full_pipeline(args, D)
        out["serve"] = {"mixed": serve_summary(D, "mixed"), "fp64": serve_summary(D, "fp64")}
        out["batch"] = batch_summary(D)
    if not args.no_cpu_baseline and world == 1 or (not args.no_cpu_baseline and rank == 0):
        try:
            r = oracle_subprocess(args, steps=1, all_cores=True)
            ac = r.get("all_core")
            gold = golden_for(args.config)
            out["cpu_baseline"] = {
                "value": ac["value"] if ac else r["value"], "unit": UNIT, "cores": ac["cores"] if ac else 1,
                "kind": "oracle", "sample": r["sample"] + ("; one single-threaded replica per host core at once"
                                                           if ac else "; one core"),
                "n_dof": r["n_dof"], "iters": r["iters"], "nproc": r["nproc"], "cpu_model": r["cpu_model"],
                "single_core": {"value": r["value"], "cores": 1, "pcg_s": r["pcg_s"][-1]},
                "full_size_record": ({"n_dof": gold["n_dof"], "iters": gold["iters"],
                                      "pcg_s": gold["oracle_seconds"]["pcg"],
                                      "value": gold["n_dof"] * gold["iters"] / gold["oracle_seconds"]["pcg"],
                                      "cores": 1, "where": "the oracle run that wrote the golden file (one core "
                                      "of the build host, not this host)"} if gold else None)}
        except Exception as e:  # reported, never silently replaced
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": "failed: %s" % str(e)[:200]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
