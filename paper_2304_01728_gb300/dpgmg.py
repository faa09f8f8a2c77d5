"""Thin ctypes binding of the C ABI in include/dpgmg.h (argument marshalling only).

Every computation runs in ``libdpgmg.so``; importing this module on a machine
without the built library raises immediately (there is no fallback).  The
functions carry the C names; ``Solver`` is a small convenience wrapper that
owns a handle and a system.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpgmg.so")

DPGMG_OK = 0
ERR = {-1: "ARG", -2: "NOMEM", -3: "NOT_HPD", -4: "BREAKDOWN", -5: "NOT_CONVERGED",
       -6: "TIMEOUT", -7: "PENDING", -8: "CUDA"}
DPGMG_ERR_ARG, DPGMG_ERR_NOMEM, DPGMG_ERR_NOT_HPD, DPGMG_ERR_BREAKDOWN = -1, -2, -3, -4
DPGMG_ERR_NOT_CONVERGED, DPGMG_ERR_TIMEOUT, DPGMG_ERR_PENDING, DPGMG_ERR_CUDA = -5, -6, -7, -8
SRC_GAUSSIAN, SRC_PLANE_WAVE, SRC_MANUFACTURED = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
COARSEST_CHOLESKY, COARSEST_NONE, COARSEST_AUTO, COARSEST_SMOOTH = 0, 1, 2, 3
FLAG_EAGER, FLAG_CUDA_CORES, FLAG_STORE_COARSE, FLAG_WARM_START, FLAG_CG_C128 = 1, 2, 4, 8, 16
FLAG_PATCH_FP64, FLAG_PATCH_R2, FLAG_RECOMPUTE_PATCHES, FLAG_COMPLEX_STORAGE = 32, 64, 128, 256
FLAG_FAULT_NOT_HPD, FLAG_FAULT_TC_WAIT = 1 << 28, 1 << 29
OP_A, OP_SMOOTH, OP_VCYCLE, OP_RESTRICT, OP_PROLONG, OP_CONDENSE, OP_COARSE, OP_AFULL = range(8)


class DpgmgError(RuntimeError):
    def __init__(self, code, where, msg=""):
        self.code = code
        super().__init__("%s: %s (%d) %s" % (where, ERR.get(code, "?"), code, msg))


class dpgmg_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3),
                ("p", ctypes.c_int), ("dp", ctypes.c_int), ("omega", ctypes.c_double),
                ("wavespeed", ctypes.POINTER(ctypes.c_double)), ("source", ctypes.c_int),
                ("src_center", ctypes.c_double * 3), ("src_width", ctypes.c_double),
                ("src_amp", ctypes.c_double), ("wave_dir", ctypes.c_double * 3),
                ("mf_order", ctypes.c_int), ("mf_coeffs", ctypes.POINTER(ctypes.c_double)),
                ("u0_samples", ctypes.POINTER(ctypes.c_double))]


class dpgmg_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("n_levels", ctypes.c_int), ("p_min", ctypes.c_int),
                ("precision", ctypes.c_int), ("coarsest", ctypes.c_int), ("flags", ctypes.c_int),
                ("theta", ctypes.c_double)]


class dpgmg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("t_pcg_ms", ctypes.c_double),
                ("bytes_per_iter", ctypes.c_longlong), ("n_dof", ctypes.c_longlong),
                ("dev_bytes_peak", ctypes.c_longlong)]


class dpgmg_level_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("p", ctypes.c_int), ("n_dof", ctypes.c_longlong),
                ("n_smooth", ctypes.c_longlong), ("kind", ctypes.c_int), ("n_patches", ctypes.c_longlong),
                ("patch_max", ctypes.c_longlong), ("sum_patch_sq", ctypes.c_longlong),
                ("op_nnz", ctypes.c_longlong), ("theta", ctypes.c_double), ("patch_stored", ctypes.c_longlong),
                ("patch_real_sq", ctypes.c_longlong), ("op_real_nnz", ctypes.c_longlong)]


_lib = None
EXPORTS = ["dpgmg_create", "dpgmg_destroy", "dpgmg_query_sizes", "dpgmg_default_opts", "dpgmg_setup",
           "dpgmg_solve", "dpgmg_release", "dpgmg_strerror", "dpgmg_last_error", "dpgmg_level_info",
           "dpgmg_element_matrix", "dpgmg_rhs", "dpgmg_apply", "dpgmg_launch_count", "dpgmg_profile",
           "dpgmg_profile_read", "dpgmg_smooth_noalloc", "dpgmg_serve_start", "dpgmg_submit", "dpgmg_poll",
           "dpgmg_spmv_group", "dpgmg_setup_profile", "dpgmg_error_indicator", "dpgmg_setup_phases",
           "dpgmg_dof_map", "dpgmg_boundary_points", "dpgmg_solve_block"]
PROF_OFF, PROF_SMOOTH_FINE, PROF_SPMV_FINE, PROF_SPMV_CG = 0, 1, 2, 3


def lib():
    """Load libdpgmg.so (built by ``paper_2304_01728_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdpgmg.so is not built (run paper_2304_01728_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    dptr = ctypes.POINTER(ctypes.c_double)
    L.dpgmg_create.argtypes = [ctypes.POINTER(vp), i, ctypes.c_size_t, vp]
    L.dpgmg_destroy.argtypes = [vp]
    L.dpgmg_destroy.restype = None
    L.dpgmg_query_sizes.argtypes = [ctypes.POINTER(dpgmg_problem), ctypes.POINTER(dpgmg_opts),
                                    ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(ctypes.c_size_t)]
    L.dpgmg_default_opts.argtypes = [ctypes.POINTER(dpgmg_opts)]
    L.dpgmg_default_opts.restype = None
    L.dpgmg_setup.argtypes = [vp, ctypes.POINTER(dpgmg_problem), ctypes.POINTER(dpgmg_opts), ctypes.POINTER(vp)]
    L.dpgmg_solve.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(dpgmg_stats)]
    L.dpgmg_release.argtypes = [vp, vp]
    L.dpgmg_release.restype = None
    L.dpgmg_strerror.argtypes = [i]
    L.dpgmg_strerror.restype = ctypes.c_char_p
    L.dpgmg_last_error.argtypes = []
    L.dpgmg_last_error.restype = ctypes.c_char_p
    L.dpgmg_level_info.argtypes = [vp, vp, i, ctypes.POINTER(dpgmg_level_desc)]
    L.dpgmg_element_matrix.argtypes = [vp, vp, i, ll, dptr, dptr]
    L.dpgmg_rhs.argtypes = [vp, vp, dptr]
    L.dpgmg_apply.argtypes = [vp, vp, i, i, dptr, dptr]
    L.dpgmg_serve_start.argtypes = [vp, i]
    L.dpgmg_serve_start.restype = i
    L.dpgmg_submit.argtypes = [vp, ctypes.POINTER(dpgmg_problem), ctypes.POINTER(dpgmg_opts), ctypes.POINTER(ll)]
    L.dpgmg_submit.restype = i
    L.dpgmg_poll.argtypes = [vp, ll, vp, vp, ctypes.POINTER(dpgmg_stats), ctypes.POINTER(d)]
    L.dpgmg_poll.restype = i
    L.dpgmg_smooth_noalloc.argtypes = [vp, vp, i, vp, vp]
    L.dpgmg_smooth_noalloc.restype = i
    L.dpgmg_launch_count.argtypes = []
    L.dpgmg_launch_count.restype = ll
    L.dpgmg_profile.argtypes = [vp, vp, i]
    L.dpgmg_spmv_group.argtypes = [vp, vp, i, i, ctypes.POINTER(i)]
    L.dpgmg_spmv_group.restype = i
    L.dpgmg_setup_profile.argtypes = [vp, vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
    L.dpgmg_setup_profile.restype = i
    L.dpgmg_setup_phases.argtypes = [vp, vp, ctypes.POINTER(d), i]
    L.dpgmg_setup_phases.restype = i
    L.dpgmg_dof_map.argtypes = [ctypes.POINTER(dpgmg_problem), ll, ctypes.POINTER(i)]
    L.dpgmg_dof_map.restype = i
    L.dpgmg_boundary_points.argtypes = [ctypes.POINTER(dpgmg_problem), ctypes.POINTER(ll),
                                        ctypes.POINTER(ctypes.c_double)]
    L.dpgmg_boundary_points.restype = i
    L.dpgmg_solve_block.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i, ctypes.c_void_p, ctypes.c_void_p, i,
                                    ctypes.POINTER(dpgmg_stats)]
    L.dpgmg_solve_block.restype = i
    L.dpgmg_error_indicator.argtypes = [vp, vp, dptr, dptr]
    L.dpgmg_error_indicator.restype = i
    L.dpgmg_profile_read.argtypes = [vp, vp, ctypes.POINTER(d), ctypes.POINTER(ll), ctypes.POINTER(ll)]
    for f in ["dpgmg_create", "dpgmg_query_sizes", "dpgmg_setup", "dpgmg_solve", "dpgmg_level_info",
              "dpgmg_element_matrix", "dpgmg_rhs", "dpgmg_apply", "dpgmg_profile", "dpgmg_profile_read"]:
        getattr(L, f).restype = i
    _lib = L
    return L


def _check(code, where):
    if code != DPGMG_OK:
        raise DpgmgError(code, where, lib().dpgmg_last_error().decode())
    return code


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(n, p, omega, x0=(0, 0, 0), x1=(1, 1, 1), wavespeed=None, source="gaussian",
                 src_center=(0.5, 0.5, 0.5), src_width=0.1, src_amp=1.0, wave_dir=(1, 0, 0),
                 mf_coeffs=None, u0_samples=None):
    """Fill a dpgmg_problem; returns (struct, keep-alive list of arrays)."""
    pb = dpgmg_problem()
    keep = []
    for k in range(3):
        pb.n[k] = int(n[k])
        pb.x0[k] = float(x0[k])
        pb.x1[k] = float(x1[k])
        pb.src_center[k] = float(src_center[k])
        pb.wave_dir[k] = float(wave_dir[k])
    pb.p, pb.dp, pb.omega = int(p), 1, float(omega)
    if wavespeed is not None:
        c = np.ascontiguousarray(wavespeed, dtype=np.float64)
        keep.append(c)
        pb.wavespeed = _dptr(c)
    pb.source = {"gaussian": SRC_GAUSSIAN, "plane_wave": SRC_PLANE_WAVE, "manufactured": SRC_MANUFACTURED}[source]
    pb.src_width, pb.src_amp = float(src_width), float(src_amp)
    if mf_coeffs is not None:
        C = np.ascontiguousarray(np.asarray(mf_coeffs, dtype=np.complex128))
        keep.append(C)
        pb.mf_order = C.shape[1]
        pb.mf_coeffs = C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if u0_samples is not None:
        U = np.ascontiguousarray(np.asarray(u0_samples, dtype=np.complex128))
        keep.append(U)
        pb.u0_samples = U.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return pb, keep


def make_opts(**kw):
    op = dpgmg_opts()
    lib().dpgmg_default_opts(ctypes.byref(op))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[v]
        if k == "coarsest" and isinstance(v, str):
            v = {"cholesky": COARSEST_CHOLESKY, "none": COARSEST_NONE, "auto": COARSEST_AUTO,
                 "smooth": COARSEST_SMOOTH}[v]
        setattr(op, k, v)
    return op


def dpgmg_create(device=0, mem_budget_bytes=0, cuda_stream=None):
    h = ctypes.c_void_p()
    _check(lib().dpgmg_create(ctypes.byref(h), int(device), int(mem_budget_bytes), cuda_stream), "dpgmg_create")
    return h


def dpgmg_destroy(h):
    lib().dpgmg_destroy(h)


def dpgmg_query_sizes(pb, op):
    nt, nf, nb = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t()
    _check(lib().dpgmg_query_sizes(ctypes.byref(pb), ctypes.byref(op), ctypes.byref(nt), ctypes.byref(nf),
                                   ctypes.byref(nb)), "dpgmg_query_sizes")
    return nt.value, nf.value, nb.value


def dpgmg_setup(h, pb, op):
    s = ctypes.c_void_p()
    _check(lib().dpgmg_setup(h, ctypes.byref(pb), ctypes.byref(op), ctypes.byref(s)), "dpgmg_setup")
    return s


def dpgmg_solve(h, s, trace_out=None, field_out=None, out_is_device=False):
    """trace_out / field_out: numpy complex128 arrays (host) or device pointers (ints)."""
    st = dpgmg_stats()
    tp = trace_out.ctypes.data if isinstance(trace_out, np.ndarray) else trace_out
    fp = field_out.ctypes.data if isinstance(field_out, np.ndarray) else field_out
    code = lib().dpgmg_solve(h, s, tp, fp, int(bool(out_is_device)), ctypes.byref(st))
    if code not in (DPGMG_OK, DPGMG_ERR_NOT_CONVERGED):
        _check(code, "dpgmg_solve")
    return code, st


def dpgmg_solve_block(h, s, rhs, trace_out=None, on_device=False, k=None):
    """k right-hand sides at once.  rhs: numpy complex128 [k, n] (host) or a
    device pointer (int, then k is required); trace_out likewise (host arrays
    are allocated when None).  Returns (code, x, [stats per column])."""
    if isinstance(rhs, np.ndarray):
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        k = rhs.shape[0]
        if trace_out is None:
            trace_out = np.zeros_like(rhs)
    stats = (dpgmg_stats * k)()
    rp = rhs.ctypes.data if isinstance(rhs, np.ndarray) else rhs
    tp = trace_out.ctypes.data if isinstance(trace_out, np.ndarray) else trace_out
    code = lib().dpgmg_solve_block(h, s, int(k), rp, tp, int(bool(on_device)), stats)
    if code not in (DPGMG_OK, DPGMG_ERR_NOT_CONVERGED):
        _check(code, "dpgmg_solve_block")
    return code, trace_out, list(stats)


def dpgmg_release(h, s):
    lib().dpgmg_release(h, s)


def dpgmg_level_info(h, s, level):
    d = dpgmg_level_desc()
    _check(lib().dpgmg_level_info(h, s, int(level), ctypes.byref(d)), "dpgmg_level_info")
    return d


def dpgmg_element_matrix(h, s, level, e, nloc, with_load=False):
    M = np.zeros((nloc, nloc), dtype=np.complex128)
    F = np.zeros(nloc, dtype=np.complex128) if with_load else None
    _check(lib().dpgmg_element_matrix(h, s, int(level), int(e), _dptr(M), _dptr(F) if with_load else None),
           "dpgmg_element_matrix")
    return (M, F) if with_load else M


def dpgmg_rhs(h, s, n):
    b = np.zeros(n, dtype=np.complex128)
    _check(lib().dpgmg_rhs(h, s, _dptr(b)), "dpgmg_rhs")
    return b


def dpgmg_apply(h, s, op, level, x, nout):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.zeros(nout, dtype=np.complex128)
    _check(lib().dpgmg_apply(h, s, int(op), int(level), _dptr(x), _dptr(y)), "dpgmg_apply")
    return y


def dpgmg_serve_start(h, slots):
    _check(lib().dpgmg_serve_start(h, int(slots)), "dpgmg_serve_start")


def dpgmg_submit(h, pb, op):
    """Queue a solve; returns the ticket (raises DpgmgError with NOMEM when refused)."""
    t = ctypes.c_longlong()
    _check(lib().dpgmg_submit(h, ctypes.byref(pb), ctypes.byref(op), ctypes.byref(t)), "dpgmg_submit")
    return t.value


def dpgmg_poll(h, ticket, trace_out=None, field_out=None):
    """(status, stats, latency_ms); status DPGMG_ERR_PENDING while not finished."""
    st = dpgmg_stats()
    lat = ctypes.c_double()
    tp = trace_out.ctypes.data if isinstance(trace_out, np.ndarray) else trace_out
    fp = field_out.ctypes.data if isinstance(field_out, np.ndarray) else field_out
    code = lib().dpgmg_poll(h, ctypes.c_longlong(ticket), tp, fp, ctypes.byref(st), ctypes.byref(lat))
    return code, st, lat.value


def dpgmg_dof_map(pb, n_trace):
    """Per global trace DOF: (kind, cx, cy, cz, axis, m1, m2) as an int array [n_trace, 7]."""
    out = np.zeros((n_trace, 7), dtype=np.int32)
    _check(lib().dpgmg_dof_map(ctypes.byref(pb), n_trace, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
           "dpgmg_dof_map")
    return out


def dpgmg_boundary_points(pb):
    """Points [n, 3] at which a caller's impedance load u0 is sampled (problem u0_samples)."""
    n = ctypes.c_longlong(0)
    _check(lib().dpgmg_boundary_points(ctypes.byref(pb), ctypes.byref(n), None), "dpgmg_boundary_points")
    out = np.zeros((n.value, 3))
    _check(lib().dpgmg_boundary_points(ctypes.byref(pb), ctypes.byref(n),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "dpgmg_boundary_points")
    return out


def dpgmg_launch_count():
    return int(lib().dpgmg_launch_count())


def dpgmg_error_indicator(h, s, x, nelem):
    """eta_K^2 of every element for the trace vector x (complex128)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    eta2 = np.zeros(int(nelem), dtype=np.float64)
    _check(lib().dpgmg_error_indicator(h, s, _dptr(x), eta2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "dpgmg_error_indicator")
    return eta2


SETUP_PHASES = ("element stage", "operators", "smoothers", "coarsest (side stream)", "coarsest wait",
                "solve preparation")


def dpgmg_setup_phases(h, s):
    """Device ms of each setup phase, in the order of SETUP_PHASES."""
    out = (ctypes.c_double * len(SETUP_PHASES))()
    _check(lib().dpgmg_setup_phases(h, s, out, len(SETUP_PHASES)), "dpgmg_setup_phases")
    return list(out)


def dpgmg_setup_profile(h, s):
    """(element-stage ms, element-stage GFLOP, setup ms)"""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().dpgmg_setup_profile(h, s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "dpgmg_setup_profile")
    return a.value, b.value, c.value


def dpgmg_spmv_group(h, s, level, set_to=0):
    g = ctypes.c_int()
    _check(lib().dpgmg_spmv_group(h, s, int(level), int(set_to), ctypes.byref(g)), "dpgmg_spmv_group")
    return g.value


def dpgmg_profile(h, s, which):
    _check(lib().dpgmg_profile(h, s, int(which)), "dpgmg_profile")


def dpgmg_profile_read(h, s):
    """(summed device ms, launches, algorithmic bytes per launch) since the last read."""
    ms, n, b = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().dpgmg_profile_read(h, s, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)), "dpgmg_profile_read")
    return ms.value, n.value, b.value


def dpgmg_smooth_noalloc(h, s, level, r_dev, y_dev):
    """y = theta S r on device pointers (ints), allocation-free; see include/dpgmg.h."""
    _check(lib().dpgmg_smooth_noalloc(h, s, int(level), ctypes.c_void_p(r_dev), ctypes.c_void_p(y_dev)),
           "dpgmg_smooth_noalloc")


def strerror(code):
    return lib().dpgmg_strerror(int(code)).decode()


class Solver:
    """One handle + one system: setup on construction, solve() on demand."""

    def __init__(self, problem_kw, device=0, mem_budget_bytes=0, **opts):
        self.h = dpgmg_create(device, mem_budget_bytes)
        self.pb, self._keep = make_problem(**problem_kw)
        self.op = make_opts(**opts)
        self.n_trace, self.n_field, self.dev_bytes = dpgmg_query_sizes(self.pb, self.op)
        try:
            self.s = dpgmg_setup(self.h, self.pb, self.op)
        except Exception:
            dpgmg_destroy(self.h)
            raise

    def solve(self, fields=True):
        x = np.zeros(self.n_trace, dtype=np.complex128)
        f = np.zeros(self.n_field, dtype=np.complex128) if fields else None
        code, st = dpgmg_solve(self.h, self.s, x, f)
        return x, f, st, code

    def level(self, l):
        return dpgmg_level_info(self.h, self.s, l)

    def close(self):
        if self.s is not None:
            dpgmg_release(self.h, self.s)
            self.s = None
        if self.h is not None:
            dpgmg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
