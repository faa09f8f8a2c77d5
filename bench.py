#!/usr/bin/env python3
"""Benchmark of the DPG-MG solver (MG-preconditioned CG on the condensed DPG trace system).

One step = one pass of the whole hot path through the C ABI: dpgmg_setup
(batched element DPG work, assembly, hierarchy, patch factorisations,
coarsest factor) + dpgmg_solve (PCG to relative residual 1e-8, field
recovery) + dpgmg_release, on the 16^3, p = 3, omega = 16 pi unit-cube
workload with a 3-level h/p V(1,1)-cycle.

value  = DOF-iterations per second of the PCG phase (N_dof * iterations /
         PCG device time), summed over ranks; ms_per_step is the whole step.
e2e    = the same metric with the end-to-end time of setup + solve through the
         public API with host input and output buffers (copies included).
roofline: the finest-level smoother product kernel, timed live with CUDA
         events on the library's stream inside the timed steps.
cpu_baseline: the FP64 oracle (test infrastructure) on a bounded sample of
         the same workload (a 4^3-element sub-box of the 16^3 mesh around the
         source, same h, p, omega, 3 levels), PCG phase only, one core.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
       [--config 2] [--precision mixed|fp64]
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
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
    return ap.parse_args()


def workload(cfg, precision):
    from paper_2304_01728_gb300 import workloads
    return {1: workloads.config1, 2: lambda: workloads.config2(precision),
            3: lambda: workloads.config3(precision)}[cfg]()


# ------------------------------------------------------------------ oracle
def oracle_sample_problem(w):
    """A 4^3-element sub-box of the workload mesh that contains the source."""
    pk = dict(w["problem"])
    n = pk["n"]
    x0 = pk.get("x0", (0, 0, 0))
    x1 = pk.get("x1", (1, 1, 1))
    h = [(x1[d] - x0[d]) / n[d] for d in range(3)]
    sub = [min(4, n[d]) for d in range(3)]
    lo, hi = [], []
    for d in range(3):
        c = int(round((pk["src_center"][d] - x0[d]) / h[d])) - sub[d] // 2
        c = max(0, min(n[d] - sub[d], c))
        lo.append(x0[d] + c * h[d])
        hi.append(x0[d] + (c + sub[d]) * h[d])
    ws = pk.get("wavespeed")
    wsub = None
    if ws is not None:
        wsub = []
        for kz in range(sub[2]):
            for ky in range(sub[1]):
                for kx in range(sub[0]):
                    ix = int(round((lo[0] - x0[0]) / h[0])) + kx
                    iy = int(round((lo[1] - x0[1]) / h[1])) + ky
                    iz = int(round((lo[2] - x0[2]) / h[2])) + kz
                    wsub.append(ws[ix + n[0] * (iy + n[1] * iz)])
    levels = w["opts"]["n_levels"]
    return dict(n=tuple(sub), p=pk["p"], omega=pk["omega"], x0=tuple(lo), x1=tuple(hi), wavespeed=wsub,
                src_center=pk["src_center"], src_width=pk["src_width"]), dict(w["opts"], n_levels=min(levels, 3))


def oracle_sample_run(args):
    """Runs in a fresh single-threaded process: oracle setup (untimed), PCG (timed)."""
    import numpy as np  # noqa: F401
    from oracle.assembly import build_fine
    from oracle.hierarchy import build_hierarchy
    from oracle.problem import GaussianSource
    from oracle.solver import mg_pcg
    w = workload(args.config, "fp64")
    pk, ok = oracle_sample_problem(w)
    t0 = time.perf_counter()
    fs = build_fine(pk["n"], pk["p"], pk["omega"], wavespeed=pk["wavespeed"],
                    load=GaussianSource(pk["src_center"], pk["src_width"]), x0=pk["x0"], x1=pk["x1"])
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
    print(json.dumps(dict(value=tot_di / tot_t, n_dof=n, iters=res[-1][1], pcg_s=[r[0] for r in res],
                          setup_s=t_setup, sample="%dx%dx%d-element sub-box [%s]-[%s] of the %s mesh (same h, p=%d, "
                          "omega, source), %d levels, PCG phase only" % (
                              pk["n"][0], pk["n"][1], pk["n"][2], ",".join("%.4g" % v for v in pk["x0"]),
                              ",".join("%.4g" % v for v in pk["x1"]), "x".join(map(str, w["problem"]["n"])),
                              pk["p"], ok["n_levels"]))))


def oracle_subprocess(args, steps=1, timeout=600):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--config", str(args.config),
           "--oracle-steps", str(steps)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


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


def traffic_for(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel source is unchanged."""
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
    return e.get("traffic_bytes_per_launch")


FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of one GB300 (no measured FP64 figure is provided)


def element_line(acc):
    """Roofline line of the batched element stage (FP64 arithmetic)."""
    ms, gflop, n = acc
    if not n or ms <= 0:
        return None
    tf = gflop / (ms / 1e3) / 1e3
    return {"kernels": "k_elem_build/potrf/trsm/herk/condense", "bound": "alu", "achieved": tf,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
            "peak_source": "nominal FP64", "gflop_per_setup": gflop / n, "ms_per_setup": ms / n}


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

    def step(prof=D.PROF_OFF):
        s = D.dpgmg_setup(h, pb, op)
        try:
            for l in range(1, w["opts"]["n_levels"]):
                try:
                    tuned["level%d" % l] = D.dpgmg_spmv_group(h, s, l)
                except D.DpgmgError:
                    break
            tuned["cg"] = D.dpgmg_spmv_group(h, s, -1)
            em, eg, _ = D.dpgmg_setup_profile(h, s)
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
                        "achieved": gbs, "unit": "GB/s"})

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
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        op64 = D.make_opts(**dict(w["opts"], precision="fp64"))
        s = D.dpgmg_setup(h, pb, op64)
        code, st = D.dpgmg_solve(h, s, trace.data_ptr(), fields.data_ptr(), out_is_device=True)
        D.dpgmg_release(h, s)
        fp64 = {"value": n_dof * st.iters / (st.t_pcg_ms / 1e3), "iters": st.iters, "pcg_ms": st.t_pcg_ms,
                "setup_ms": st.t_setup_ms, "true_relres": st.true_relres}
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
                     "traffic": traffic_for("k_patch_apply")},
        "clocks": clk, "e2e": e2e, "fp64_path": fp64,
        "kernels": [dict(k, frac=k["achieved"] / peak) for k in kernels],
        "spmv_group_tuned": tuned,
        "element_stage": element_line(elem_acc_timed),
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
    if not args.no_cpu_baseline and world == 1 or (not args.no_cpu_baseline and rank == 0):
        try:
            r = oracle_subprocess(args, steps=1)
            out["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": r["sample"], "n_dof": r["n_dof"], "iters": r["iters"]}
        except Exception as e:  # reported, never silently replaced
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": "failed: %s" % str(e)[:200]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
