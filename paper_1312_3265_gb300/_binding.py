"""ctypes marshalling for the C ABI (include/sw_cgne.h)."""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from .build import lib_path as _lib_path

SW_OK = 0
SW_NOT_CONVERGED = 1
SW_OP_STAGGERED_WILSON = 0
SW_OP_WILSON = 1
SW_OP_WILSON_EVEN_ODD = 2
SW_PREC_F64 = 0
SW_PREC_F32_RELIABLE = 1
SW_PREC_F16_RELIABLE = 2
SW_PARAM_CHUNK = 0
SW_PARAM_RELIABLE_DELTA = 1
SW_PARAM_NS_SW = 2
SW_PARAM_NS_WILSON = 3
SW_PARAM_GRAPHS = 4
SW_PARAM_SITE_BLOCKING = 5
SW_PARAM_GROUP_FAST = 6
SW_PARAM_RELIABLE_DELTA_F16 = 9
SW_PARAM_PERSISTENT = 10
SW_PARAM_WILSON_LEAN = 11
SW_SITE_SHAPES = 6  # SW_PARAM_SITE_BLOCKING values: 0 lexicographic, 1..5 site-block shapes


class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("t_antiperiodic", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("status", ctypes.c_int),
                ("precision", ctypes.c_int), ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("engines_live", ctypes.c_int), ("engines_created", ctypes.c_int), ("engines_retired", ctypes.c_int),
                ("requests_waited_for_memory", ctypes.c_longlong), ("requests_waiting", ctypes.c_longlong),
                ("bytes_charged", ctypes.c_ulonglong), ("budget", ctypes.c_ulonglong)]


@dataclass
class SolveInfo:
    iters: int
    reliable_updates: int
    status: int
    precision: int
    true_rel_resid: float
    seconds: float
    lambda_min: float = 0.0
    lambda_max: float = 0.0

    @property
    def kappa(self):
        return self.lambda_max / self.lambda_min if self.lambda_min > 0 else float("nan")

    @staticmethod
    def from_c(c):
        return SolveInfo(c.iters, c.reliable_updates, c.status, c.precision, c.true_rel_resid, c.seconds,
                         c.lambda_min, c.lambda_max)


class SWError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = f"{where}: {sw_status_string(code)} (status {code})"
        if code == -4:
            msg += f" [{sw_last_cuda_error()}]"
        super().__init__(msg)


def lib_path():
    return _lib_path()


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        p = _lib_path()
        if not os.path.exists(p):
            raise ImportError(f"CUDA library {p} is missing: build it first with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(p)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lat = ctypes.POINTER(Lattice)
        L.sw_hypercube_build.argtypes = [lat, vp, vp, vp]
        L.sw_dslash_apply.argtypes = [lat, vp, vp, vp, vp, d, d, i, vp]
        L.wilson_dslash_apply.argtypes = [lat, vp, vp, vp, d, d, i, vp]
        L.cgne_solve.argtypes = [lat, i, vp, vp, vp, vp, d, d, d, i, i, ctypes.POINTER(_Info), vp]
        L.cgne_solve_batch.argtypes = [lat, i, vp, vp, i, vp, vp, ctypes.POINTER(ctypes.c_double), d, d, i, i,
                                       ctypes.POINTER(_Info), vp]
        L.dslash_apply_inner.argtypes = [lat, i, vp, vp, i, vp, vp, ctypes.POINTER(ctypes.c_double), d, i, i, vp]
        L.dslash_apply_inner.restype = i
        L.cgne_solve_noalloc.argtypes = [lat, i, vp, vp, vp, vp, d, d, d, i, ctypes.POINTER(_Info), vp]
        L.cgne_solve_noalloc.restype = i
        srv = ctypes.c_void_p
        L.sw_server_create.argtypes = [ctypes.c_size_t, ctypes.POINTER(srv)]
        L.sw_server_add_engine.argtypes = [srv, lat, i, vp, d, i, i, ctypes.POINTER(i)]
        L.sw_server_submit.argtypes = [srv, i, vp, vp, d, d, i, ctypes.POINTER(ctypes.c_longlong)]
        L.sw_server_add_field.argtypes = [srv, lat, vp, i, ctypes.POINTER(i)]
        L.sw_server_submit_field.argtypes = [srv, i, i, d, i, vp, vp, d, d, i, ctypes.POINTER(ctypes.c_longlong)]
        L.sw_server_stats.argtypes = [srv, ctypes.POINTER(_ServerStats)]
        L.sw_server_poll.argtypes = [srv, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_Info),
                                     ctypes.POINTER(i)]
        L.sw_server_drain.argtypes = [srv, d]
        L.sw_server_destroy.argtypes = [srv]
        for f in ("sw_server_create", "sw_server_add_engine", "sw_server_submit", "sw_server_poll",
                  "sw_server_drain", "sw_server_destroy", "sw_server_add_field", "sw_server_submit_field",
                  "sw_server_stats"):
            getattr(L, f).restype = i
        L.sw_autotune.argtypes = [lat, i, vp, vp, i, i, d, i, ctypes.POINTER(d), ctypes.POINTER(i), vp]
        L.sw_autotune.restype = i
        L.sw_autotune_layout.argtypes = [lat, i, vp, vp, i, i, d, i, ctypes.POINTER(d), ctypes.POINTER(i),
                                         ctypes.POINTER(i), vp]
        L.sw_autotune_layout.restype = i
        L.sw_set_param.argtypes = [i, d]
        L.sw_get_param.argtypes = [i, ctypes.POINTER(d)]
        L.sw_set_param.restype = i
        L.sw_get_param.restype = i
        L.sw_measure_fp64_peak.argtypes = [ctypes.POINTER(d), vp]
        L.sw_measure_fp64_peak.restype = i
        L.sw_kernel_launches.argtypes = []
        L.sw_kernel_launches.restype = ctypes.c_longlong
        L.sw_workspace_reserved.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.sw_workspace_reserved.restype = i
        L.sw_trim_workspace.argtypes = []
        L.sw_trim_workspace.restype = i
        L.sw_profile_enable.argtypes = [i]
        L.sw_profile_reset.argtypes = []
        L.sw_profile_count.argtypes = []
        L.sw_profile_entry.argtypes = [i, ctypes.c_char_p, i, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
        for f in ("sw_profile_enable", "sw_profile_reset", "sw_profile_count", "sw_profile_entry"):
            getattr(L, f).restype = i
        L.sw_status_string.argtypes = [i]
        L.sw_status_string.restype = ctypes.c_char_p
        L.sw_last_cuda_error.argtypes = []
        L.sw_last_cuda_error.restype = ctypes.c_char_p
        for f in ("sw_hypercube_build", "sw_dslash_apply", "wilson_dslash_apply", "cgne_solve", "cgne_solve_batch"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


def sw_status_string(code):
    return lib().sw_status_string(int(code)).decode()


def sw_last_cuda_error():
    return lib().sw_last_cuda_error().decode()


def _lat(dims, t_antiperiodic):
    return ctypes.byref(Lattice((ctypes.c_int * 4)(*[int(v) for v in dims]), int(bool(t_antiperiodic))))


def _ptr(t):
    """Device pointer of a torch tensor (or a raw integer address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(code, where):
    if code < 0:
        raise SWError(code, where)
    return code


def sw_hypercube_build(dims, U, W, t_antiperiodic=False, stream=None):
    _check(lib().sw_hypercube_build(_lat(dims, t_antiperiodic), _ptr(U), _ptr(W), _stream(stream)),
           "sw_hypercube_build")


def sw_dslash_apply(dims, U, W, inp, out, mass, r=1.0, dagger=False, t_antiperiodic=False, stream=None):
    _check(lib().sw_dslash_apply(_lat(dims, t_antiperiodic), _ptr(U), _ptr(W), _ptr(inp), _ptr(out),
                                 float(mass), float(r), int(bool(dagger)), _stream(stream)), "sw_dslash_apply")


def wilson_dslash_apply(dims, U, inp, out, mass, r=1.0, dagger=False, t_antiperiodic=False, stream=None):
    _check(lib().wilson_dslash_apply(_lat(dims, t_antiperiodic), _ptr(U), _ptr(inp), _ptr(out),
                                     float(mass), float(r), int(bool(dagger)), _stream(stream)),
           "wilson_dslash_apply")


def dslash_apply_inner(dims, op, U, W, inp, out, masses, r=1.0, dagger=False, precision=SW_PREC_F32_RELIABLE,
                       t_antiperiodic=False, stream=None):
    """(D+m) or (D+m)^+ on len(masses) systems back to back, in the inner precision
    of the mixed-mode iterations (by the CG iteration kernels), returned in FP64."""
    n = len(masses)
    m = (ctypes.c_double * n)(*[float(v) for v in masses])
    _check(lib().dslash_apply_inner(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), n, _ptr(inp), _ptr(out), m,
                                    float(r), int(bool(dagger)), int(precision), _stream(stream)),
           "dslash_apply_inner")


def cgne_solve(dims, op, U, W, chi, x, mass, r=1.0, tol=1e-8, max_iter=100000, precision=SW_PREC_F64,
               t_antiperiodic=False, stream=None):
    """Solve (D+m)^+(D+m) x = (D+m)^+ chi; x holds the initial guess on entry.
    Returns SolveInfo; raises SWError on negative status (not on SW_NOT_CONVERGED)."""
    info = _Info()
    rc = lib().cgne_solve(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), _ptr(chi), _ptr(x),
                          float(mass), float(r), float(tol), int(max_iter), int(precision),
                          ctypes.byref(info), _stream(stream))
    _check(rc, "cgne_solve")
    return SolveInfo.from_c(info)


def cgne_solve_batch(dims, op, U, W, chi, x, masses, r=1.0, tol=1e-8, max_iter=100000, precision=SW_PREC_F64,
                     t_antiperiodic=False, stream=None):
    """Batched CGNE over nsys = len(masses) systems; chi and x hold the systems
    back to back.  Returns (status, [SolveInfo]); raises SWError on negative status."""
    n = len(masses)
    m = (ctypes.c_double * n)(*[float(v) for v in masses])
    infos = (_Info * n)()
    rc = lib().cgne_solve_batch(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), n, _ptr(chi), _ptr(x), m,
                                float(r), float(tol), int(max_iter), int(precision), infos, _stream(stream))
    _check(rc, "cgne_solve_batch")
    return rc, [SolveInfo.from_c(infos[i]) for i in range(n)]


def sw_profile_enable(on=True):
    lib().sw_profile_enable(int(bool(on)))


def sw_profile_reset():
    lib().sw_profile_reset()


def sw_profile_read():
    """{class: {"launches", "ms", "bytes", "flops", "issued"}} accumulated since the last reset
    (launches, ms, bytes, flops: the timed launches; issued: every launch while enabled)."""
    out = {}
    L = lib()
    for i in range(L.sw_profile_count()):
        name = ctypes.create_string_buffer(64)
        n, ms, by, fl = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(L.sw_profile_entry(i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                  ctypes.byref(fl)), "sw_profile_entry")
        iss = ctypes.c_longlong()
        _check(L.sw_profile_issued(i, ctypes.byref(iss)), "sw_profile_issued")
        out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value,
                                    "issued": iss.value}
    return out


def sw_measure_fp64_peak(stream=None):
    """FP64 FMA throughput of the current device, TFLOP/s (measured by the library)."""
    v = ctypes.c_double()
    _check(lib().sw_measure_fp64_peak(ctypes.byref(v), _stream(stream)), "sw_measure_fp64_peak")
    return v.value


def sw_kernel_launches():
    return int(lib().sw_kernel_launches())


def sw_workspace_reserved():
    """Device bytes the library's workspace pool on the current device holds (in use or cached)."""
    v = ctypes.c_ulonglong()
    _check(lib().sw_workspace_reserved(ctypes.byref(v)), "sw_workspace_reserved")
    return int(v.value)


def sw_trim_workspace():
    """Hand the cached, unused device workspace of the current device back to the driver."""
    _check(lib().sw_trim_workspace(), "sw_trim_workspace")


def cgne_solve_noalloc(dims, op, U, W, chi, x, mass, r=1.0, tol=1e-8, max_iter=100000, t_antiperiodic=False,
                       stream=None):
    """FP64 CGNE with the library's static device scratch (no allocation)."""
    info = _Info()
    rc = lib().cgne_solve_noalloc(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), _ptr(chi), _ptr(x),
                                  float(mass), float(r), float(tol), int(max_iter), ctypes.byref(info),
                                  _stream(stream))
    _check(rc, "cgne_solve_noalloc")
    return SolveInfo.from_c(info)


def sw_set_param(key, value):
    _check(lib().sw_set_param(int(key), float(value)), "sw_set_param")


def sw_get_param(key):
    v = ctypes.c_double()
    _check(lib().sw_get_param(int(key), ctypes.byref(v)), "sw_get_param")
    return v.value


def _host_ptr(a):
    """Address of a host buffer: a numpy array or a CPU torch tensor (contiguous)."""
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be contiguous")
        return a.ctypes.data
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("host buffer must be a contiguous CPU tensor")
    return a.data_ptr()


class Server:
    """Continuous-batching solve server (see sw_server_* in include/sw_cgne.h).

    Host buffers handed to submit() are kept referenced here until their
    request is returned by poll()."""

    def __init__(self, hbm_budget_bytes):
        self._h = ctypes.c_void_p()
        _check(lib().sw_server_create(int(hbm_budget_bytes), ctypes.byref(self._h)), "sw_server_create")
        self._keep = {}

    def add_engine(self, dims, op, U, r=1.0, precision=SW_PREC_F32_RELIABLE, slots=8, t_antiperiodic=False):
        eng = ctypes.c_int()
        _check(lib().sw_server_add_engine(self._h, _lat(dims, t_antiperiodic), int(op), _ptr(U), float(r),
                                          int(precision), int(slots), ctypes.byref(eng)), "sw_server_add_engine")
        return eng.value

    def submit(self, engine, chi_host, x_host, mass, tol=1e-8, max_iter=100000):
        rid = ctypes.c_longlong()
        _check(lib().sw_server_submit(self._h, int(engine), _host_ptr(chi_host), _host_ptr(x_host), float(mass),
                                      float(tol), int(max_iter), ctypes.byref(rid)), "sw_server_submit")
        self._keep[rid.value] = (chi_host, x_host)
        return rid.value

    def add_field(self, dims, U, slots=8, t_antiperiodic=False):
        """Resident gauge field for submit_field; returns its index."""
        f = ctypes.c_int()
        _check(lib().sw_server_add_field(self._h, _lat(dims, t_antiperiodic), _ptr(U), int(slots), ctypes.byref(f)),
               "sw_server_add_field")
        return f.value

    def submit_field(self, field, op, chi_host, x_host, mass, precision=SW_PREC_F32_RELIABLE, r=1.0, tol=1e-8,
                     max_iter=100000):
        """Queue a solve on a resident field; the server admits it by device memory."""
        rid = ctypes.c_longlong()
        _check(lib().sw_server_submit_field(self._h, int(field), int(op), float(r), int(precision), _host_ptr(chi_host),
                                            _host_ptr(x_host), float(mass), float(tol), int(max_iter),
                                            ctypes.byref(rid)), "sw_server_submit_field")
        self._keep[rid.value] = (chi_host, x_host)
        return rid.value

    def stats(self):
        st = _ServerStats()
        _check(lib().sw_server_stats(self._h, ctypes.byref(st)), "sw_server_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def poll(self, max_n=1024):
        ids = (ctypes.c_longlong * max_n)()
        infos = (_Info * max_n)()
        n = ctypes.c_int()
        _check(lib().sw_server_poll(self._h, max_n, ids, infos, ctypes.byref(n)), "sw_server_poll")
        out = []
        for k in range(n.value):
            self._keep.pop(ids[k], None)
            out.append((ids[k], SolveInfo.from_c(infos[k])))
        return out

    def drain(self, timeout_s=600.0):
        _check(lib().sw_server_drain(self._h, float(timeout_s)), "sw_server_drain")

    def close(self):
        if self._h:
            lib().sw_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sw_autotune(dims, op, U, W, nsys, precision=SW_PREC_F32_RELIABLE, r=1.0, iters=48, t_antiperiodic=False,
                stream=None):
    """Time register-blocking widths 1, 2, 4 and keep the fastest; returns (best, {width: ms})."""
    ms = (ctypes.c_double * 3)()
    best = ctypes.c_int()
    _check(lib().sw_autotune(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), int(nsys), int(precision),
                             float(r), int(iters), ms, ctypes.byref(best), _stream(stream)), "sw_autotune")
    return best.value, {1: ms[0], 2: ms[1], 4: ms[2]}


def sw_autotune_layout(dims, op, U, W, nsys, precision=SW_PREC_F32_RELIABLE, r=1.0, iters=48,
                       t_antiperiodic=False, stream=None):
    """Time register-blocking widths 1, 2, 4 x site orders 0..SW_SITE_SHAPES-1
    (lexicographic, then the site-block shapes) and keep the fastest pair;
    returns ((ns, shape), {(ns, shape): ms})."""
    ms = (ctypes.c_double * (3 * SW_SITE_SHAPES))()
    bns, bshape = ctypes.c_int(), ctypes.c_int()
    _check(lib().sw_autotune_layout(_lat(dims, t_antiperiodic), int(op), _ptr(U), _ptr(W), int(nsys),
                                    int(precision), float(r), int(iters), ms, ctypes.byref(bns),
                                    ctypes.byref(bshape), _stream(stream)), "sw_autotune_layout")
    return (bns.value, bshape.value), {(w, b): ms[k * SW_SITE_SHAPES + b] for k, w in enumerate((1, 2, 4))
                                        for b in range(SW_SITE_SHAPES)}
