"""Python binding of the phiks C ABI (include/phiks.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libphiks.so.  Device buffers are torch tensors (their data_ptr is
passed through), streams are torch.cuda.Stream objects (their cuda_stream
handle is passed through).  If the library is missing or fails to load this
module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "PHIKS_FP64", "PHIKS_TF32", "PHIKS_TF32X3", "PHIKS_BF16X3", "PHIKS_FP64_EMU", "PHIKS_C128",
    "PHIKS_RULE_GLL",
    "PHIKS_RULE_GL",
    "PhiksError", "Options", "lib", "library_path", "load",
    "phiks_plan", "phiks_apply", "phiks_apply_ex", "phiks_workspace_size",
    "phiks_select_params", "phiks_choose_params", "phiks_last_params", "phiks_tucker", "phiks_expm",
    "phiks_profile_enable", "phiks_profile_read", "phiks_kernel_launches", "phiks_tucker_noalloc",
    "phiks_device_status", "phiks_serve_trace", "phiks_integrate", "phiks_integrate_blocks",
    "phiks_plan_shape", "phiks_destroy", "phiks_last_error", "Plan", "Batch",
    "phiks_debug_fail_alloc", "phiks_debug_live_allocations", "phiks_debug_wait_timeout",
    "Tuning", "phiks_get_tuning", "phiks_set_tuning", "phiks_autotune",
    "EXPORTED",
]

PHIKS_FP64, PHIKS_TF32, PHIKS_TF32X3, PHIKS_BF16X3, PHIKS_FP64_EMU, PHIKS_C128 = 0, 1, 2, 3, 4, 5
PHIKS_RULE_GLL, PHIKS_RULE_GL = 0, 1
DTYPES = {"fp64": PHIKS_FP64, "tf32": PHIKS_TF32, "tf32x3": PHIKS_TF32X3, "bf16x3": PHIKS_BF16X3,
          "fp64emu": PHIKS_FP64_EMU, "c128": PHIKS_C128}
STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "UNSUPPORTED", 4: "NO_PARAMS", 5: "CUDA", 6: "TIMEOUT"}

# every symbol include/phiks.h declares
EXPORTED = [
    "phiks_options_init", "phiks_plan", "phiks_apply", "phiks_apply_ex", "phiks_workspace_size",
    "phiks_select_params", "phiks_choose_params", "phiks_last_params", "phiks_tucker", "phiks_expm",
    "phiks_profile_enable", "phiks_profile_read", "phiks_kernel_launches", "phiks_tucker_noalloc",
    "phiks_device_status", "phiks_batch_create", "phiks_batch_destroy", "phiks_batch_apply",
    "phiks_batch_capture", "phiks_graph_launch", "phiks_graph_destroy", "phiks_serve_trace",
    "phiks_integrate", "phiks_integrate_blocks", "phiks_plan_shape", "phiks_destroy", "phiks_last_error",
    "phiks_debug_fail_alloc", "phiks_debug_live_allocations", "phiks_debug_wait_timeout",
    "phiks_get_tuning", "phiks_set_tuning", "phiks_autotune",
]

HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(HERE, "libphiks.so")


class Tuning(ctypes.Structure):
    _fields_ = [
        ("fused", ctypes.c_int),
        ("fused_rows", ctypes.c_int),
        ("fp64_tile", ctypes.c_int),
        ("mode_order", ctypes.c_int * 8),
        ("emu_cols", ctypes.c_int),
        ("split_ntiles", ctypes.c_int),
        ("reserved", ctypes.c_int * 8),
    ]

    def as_dict(self, d=None):
        order = list(self.mode_order)
        if d is not None:
            order = order[:d]
        return {"fused": self.fused, "fused_rows": self.fused_rows, "fp64_tile": self.fp64_tile,
                "mode_order": order, "emu_cols": self.emu_cols, "split_ntiles": self.split_ntiles}


class Options(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("nscales", ctypes.c_int),
        ("rule", ctypes.c_int),
        ("qmin", ctypes.c_int),
        ("qmax", ctypes.c_int),
        ("skip_phi0", ctypes.c_int),
        ("force_s", ctypes.c_int),
        ("force_q", ctypes.c_int),
        ("vnorms", ctypes.POINTER(ctypes.c_double)),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("no_cache", ctypes.c_int),
        ("graph", ctypes.c_int),
        ("reserved", ctypes.c_int * 6),
    ]


class ApplyArgs(ctypes.Structure):
    _fields_ = [
        ("plan", ctypes.c_void_p),
        ("tau", ctypes.c_double),
        ("p", ctypes.c_int),
        ("nv", ctypes.c_int),
        ("v", ctypes.POINTER(ctypes.c_void_p)),
        ("out", ctypes.c_void_p),
        ("nscales", ctypes.c_int),
        ("skip_phi0", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("vnorms", ctypes.POINTER(ctypes.c_double)),
    ]


class Request(ctypes.Structure):
    _fields_ = [("napply", ctypes.c_int), ("apply", ApplyArgs * 2)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("poll_us", ctypes.c_int),
                ("graphs", ctypes.c_int)]


class Nonlinear(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double)]


PHIKS_EXP_EULER, PHIKS_ETD2RK, PHIKS_EXPRK3, PHIKS_EXPRK4S5, PHIKS_EXPRK4S6 = 0, 1, 2, 3, 4
PHIKS_NL_ADR_EXACT, PHIKS_NL_ALLEN_CAHN, PHIKS_NL_BRUSSELATOR = 0, 1, 2
SCHEMES = {"expeuler": PHIKS_EXP_EULER, "etd2rk": PHIKS_ETD2RK, "exprk3": PHIKS_EXPRK3,
           "exprk4s5": PHIKS_EXPRK4S5, "exprk4s6": PHIKS_EXPRK4S6}


class PhiksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("phiks %s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libphiks.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libphiks.so is not built; run __graft_entry__.build() or "
                              "python paper_2210_07667_gb300/_build.py")
        from . import _build
        _build.build()
    L = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.phiks_options_init.argtypes = [ctypes.POINTER(Options)]
    L.phiks_options_init.restype = None
    L.phiks_plan.argtypes = [i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p), i,
                             ctypes.POINTER(vp)]
    L.phiks_apply.argtypes = [vp, d, i, ctypes.POINTER(vp), i, vp, vp]
    L.phiks_apply_ex.argtypes = [vp, d, i, ctypes.POINTER(vp), i, ctypes.POINTER(Options), vp, vp]
    L.phiks_workspace_size.argtypes = [vp, i, i, i, ctypes.POINTER(sz)]
    L.phiks_select_params.argtypes = [vp, d, i, i, ctypes.POINTER(d), ctypes.POINTER(Options),
                                      ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.phiks_choose_params.argtypes = [i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p),
                                      d, i, i, ctypes.POINTER(d), ctypes.POINTER(Options),
                                      ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.phiks_last_params.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                    ctypes.POINTER(i)]
    L.phiks_tucker.argtypes = [vp, vp, vp, ctypes.POINTER(vp), vp]
    L.phiks_expm.argtypes = [i, i, vp, vp, vp]
    L.phiks_profile_enable.argtypes = [vp, i]
    L.phiks_profile_enable.restype = ctypes.c_int
    L.phiks_profile_read.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(d)]
    L.phiks_profile_read.restype = ctypes.c_int
    L.phiks_kernel_launches.argtypes = []
    L.phiks_kernel_launches.restype = ctypes.c_uint64
    L.phiks_batch_create.argtypes = [i, ctypes.POINTER(vp)]
    L.phiks_batch_create.restype = ctypes.c_int
    L.phiks_batch_destroy.argtypes = [vp]
    L.phiks_batch_destroy.restype = None
    bargs = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(d), ctypes.POINTER(i), ctypes.POINTER(vp),
             ctypes.POINTER(i), ctypes.POINTER(Options), ctypes.POINTER(vp), vp]
    L.phiks_batch_apply.argtypes = bargs
    L.phiks_batch_apply.restype = ctypes.c_int
    L.phiks_batch_capture.argtypes = bargs + [ctypes.POINTER(vp)]
    L.phiks_batch_capture.restype = ctypes.c_int
    L.phiks_graph_launch.argtypes = [vp, vp]
    L.phiks_graph_launch.restype = ctypes.c_int
    L.phiks_graph_destroy.argtypes = [vp]
    L.phiks_graph_destroy.restype = None
    L.phiks_serve_trace.argtypes = [ctypes.POINTER(ServeConfig), i, ctypes.POINTER(Request),
                                    ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                                    ctypes.POINTER(d)]
    L.phiks_serve_trace.restype = ctypes.c_int
    L.phiks_integrate.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i, i, ctypes.POINTER(Nonlinear),
                                  d, d, i, vp, vp]
    L.phiks_integrate.restype = ctypes.c_int
    L.phiks_integrate_blocks.argtypes = [i, ctypes.POINTER(vp), i, ctypes.POINTER(Nonlinear), d, d, i, vp,
                                         ctypes.POINTER(Options), vp]
    L.phiks_integrate_blocks.restype = ctypes.c_int
    L.phiks_plan_shape.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_int64)]
    L.phiks_plan_shape.restype = ctypes.c_int
    L.phiks_device_status.argtypes = [vp, vp]
    L.phiks_device_status.restype = ctypes.c_int
    L.phiks_tucker_noalloc.argtypes = [i, ctypes.POINTER(ctypes.c_int64), vp, vp, ctypes.POINTER(vp), vp]
    L.phiks_tucker_noalloc.restype = ctypes.c_int
    L.phiks_destroy.argtypes = [vp]
    L.phiks_destroy.restype = None
    L.phiks_debug_fail_alloc.argtypes = [i]
    L.phiks_debug_fail_alloc.restype = None
    L.phiks_debug_live_allocations.argtypes = []
    L.phiks_debug_live_allocations.restype = ctypes.c_int64
    L.phiks_debug_wait_timeout.argtypes = [vp, d, vp]
    L.phiks_debug_wait_timeout.restype = ctypes.c_int
    L.phiks_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.phiks_get_tuning.restype = ctypes.c_int
    L.phiks_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
    L.phiks_set_tuning.restype = ctypes.c_int
    L.phiks_autotune.argtypes = [vp, d, i, i, ctypes.POINTER(Options), i, vp, ctypes.POINTER(Tuning),
                                 ctypes.POINTER(d)]
    L.phiks_autotune.restype = ctypes.c_int
    L.phiks_last_error.argtypes = []
    L.phiks_last_error.restype = ctypes.c_char_p
    for name in ["phiks_plan", "phiks_apply", "phiks_apply_ex", "phiks_workspace_size",
                 "phiks_select_params", "phiks_choose_params", "phiks_last_params", "phiks_tucker",
                 "phiks_expm"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def lib() -> ctypes.CDLL:
    return load()


def phiks_last_error() -> str:
    return load().phiks_last_error().decode()


def _check(st: int):
    if st != 0:
        raise PhiksError(st, phiks_last_error())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_options(**kw) -> Options:
    o = Options()
    load().phiks_options_init(ctypes.byref(o))
    vn = kw.pop("vnorms", None)
    for k, v in kw.items():
        setattr(o, k, v)
    if vn is not None:
        arr = (ctypes.c_double * len(vn))(*[float(x) for x in vn])
        o.vnorms = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        o._keep = arr
    return o


def phiks_plan(A: Sequence[np.ndarray], dtype: int = PHIKS_FP64) -> int:
    """Plan for K = A_d (+) ... (+) A_1; A_mu host arrays (any order, copied
    to column-major doubles)."""
    d = len(A)
    edt = np.complex128 if int(dtype) == PHIKS_C128 else np.float64
    mats = [np.asfortranarray(np.asarray(a, dtype=edt)) for a in A]
    n = (ctypes.c_int64 * d)(*[m.shape[0] for m in mats])
    ptrs = (ctypes.c_void_p * d)(*[m.ctypes.data for m in mats])
    out = ctypes.c_void_p()
    _check(load().phiks_plan(d, n, ptrs, int(dtype), ctypes.byref(out)))
    return out.value


def _vptrs(vs):
    arr = (ctypes.c_void_p * len(vs))(*[_ptr(v) for v in vs])
    return arr


def phiks_apply(plan: int, tau: float, p: int, vs, out, stream=None):
    _check(load().phiks_apply(plan, float(tau), int(p), _vptrs(vs), len(vs), _ptr(out), _stream(stream)))


def phiks_apply_ex(plan: int, tau: float, p: int, vs, out, stream=None, opts: Optional[Options] = None,
                   **kw):
    o = opts if opts is not None else make_options(**kw)
    _check(load().phiks_apply_ex(plan, float(tau), int(p), _vptrs(vs), len(vs), ctypes.byref(o),
                                 _ptr(out), _stream(stream)))


def phiks_workspace_size(plan: int, p: int, nv: int, nscales: int = 1) -> int:
    b = ctypes.c_size_t()
    _check(load().phiks_workspace_size(plan, p, nv, nscales, ctypes.byref(b)))
    return b.value


def phiks_select_params(plan: int, tau: float, p: int, vnorms: Sequence[float], **kw):
    o = make_options(**kw)
    vn = (ctypes.c_double * len(vnorms))(*[float(x) for x in vnorms])
    s, q, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().phiks_select_params(plan, float(tau), int(p), len(vnorms), vn, ctypes.byref(o),
                                      ctypes.byref(s), ctypes.byref(q), ctypes.byref(t)))
    return s.value, q.value, t.value


def phiks_choose_params(A: Sequence[np.ndarray], tau: float, p: int, vnorms: Sequence[float], **kw):
    """(s, q, T#) of Sec. 3.3 on the host, without a plan or a GPU (real A)."""
    d = len(A)
    mats = [np.asfortranarray(np.asarray(a, dtype=np.float64)) for a in A]
    n = (ctypes.c_int64 * d)(*[m.shape[0] for m in mats])
    ptrs = (ctypes.c_void_p * d)(*[m.ctypes.data for m in mats])
    o = make_options(**kw)
    vn = (ctypes.c_double * len(vnorms))(*[float(x) for x in vnorms])
    s, q, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().phiks_choose_params(d, n, ptrs, float(tau), int(p), len(vnorms), vn, ctypes.byref(o),
                                      ctypes.byref(s), ctypes.byref(q), ctypes.byref(t)))
    return s.value, q.value, t.value


def phiks_last_params(plan: int):
    s, q, t, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().phiks_last_params(plan, ctypes.byref(s), ctypes.byref(q), ctypes.byref(t),
                                    ctypes.byref(k)))
    return s.value, q.value, t.value, k.value


def phiks_tucker(plan: int, V, W, Ls, stream=None):
    _check(load().phiks_tucker(plan, _ptr(V), _ptr(W), _vptrs(Ls), _stream(stream)))


def phiks_expm(X, E, stream=None):
    """X, E: device tensors of shape (batch, n, n) holding column-major
    matrices (i.e. each [k] is the transpose in torch's row-major view)."""
    batch, n = int(X.shape[0]), int(X.shape[-1])
    _check(load().phiks_expm(batch, n, _ptr(X), _ptr(E), _stream(stream)))


def phiks_profile_enable(plan: int, enable: bool = True):
    _check(load().phiks_profile_enable(plan, int(bool(enable))))


def phiks_profile_read(plan: int):
    """(milliseconds, launches, flops) of the mu-mode products since the last read."""
    ms, n, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(load().phiks_profile_read(plan, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
    return ms.value, n.value, fl.value


def phiks_kernel_launches() -> int:
    return int(load().phiks_kernel_launches())


def phiks_device_status(plan: int, stream=None):
    """Raise PhiksError(TIMEOUT) if a bounded device-side wait gave up."""
    _check(load().phiks_device_status(plan, _stream(stream)))


def phiks_tucker_noalloc(dims: Sequence[int], V, W, Ls, stream=None):
    """FP64 Tucker operator without any allocation (N <= 1,048,576): its
    intermediates live in a fixed device array inside the library."""
    d = len(dims)
    n = (ctypes.c_int64 * d)(*[int(m) for m in dims])
    _check(load().phiks_tucker_noalloc(d, n, _ptr(V), _ptr(W), _vptrs(Ls), _stream(stream)))


class Batch:
    """Independent applies spread over worker streams (phiks_batch_*).

    instances: list of (plan handle, tau, p, [vectors], out, Options)."""

    def __init__(self, nstreams: int = 16):
        h = ctypes.c_void_p()
        _check(load().phiks_batch_create(int(nstreams), ctypes.byref(h)))
        self.handle = h.value

    @staticmethod
    def _marshal(instances):
        n = len(instances)
        plans = (ctypes.c_void_p * n)(*[x[0] for x in instances])
        taus = (ctypes.c_double * n)(*[float(x[1]) for x in instances])
        ps = (ctypes.c_int * n)(*[int(x[2]) for x in instances])
        flat = [_ptr(v) for x in instances for v in x[3]]
        vs = (ctypes.c_void_p * max(len(flat), 1))(*flat)
        nvs = (ctypes.c_int * n)(*[len(x[3]) for x in instances])
        opts = (Options * n)(*[x[5] for x in instances])
        outs = (ctypes.c_void_p * n)(*[_ptr(x[4]) for x in instances])
        return n, plans, taus, ps, vs, nvs, opts, outs

    def apply(self, instances, stream=None):
        n, plans, taus, ps, vs, nvs, opts, outs = self._marshal(instances)
        _check(load().phiks_batch_apply(self.handle, n, plans, taus, ps, vs, nvs, opts, outs,
                                        _stream(stream)))

    def capture(self, instances, stream):
        n, plans, taus, ps, vs, nvs, opts, outs = self._marshal(instances)
        g = ctypes.c_void_p()
        _check(load().phiks_batch_capture(self.handle, n, plans, taus, ps, vs, nvs, opts, outs,
                                          _stream(stream), ctypes.byref(g)))
        return g.value

    @staticmethod
    def launch(graph, stream):
        _check(load().phiks_graph_launch(graph, _stream(stream)))

    @staticmethod
    def destroy_graph(graph):
        load().phiks_graph_destroy(graph)

    def close(self):
        if self.handle:
            load().phiks_batch_destroy(self.handle)
            self.handle = None


def phiks_serve_trace(requests, arrivals, slots=8, hbm_budget=0, poll_us=0, graphs=1):
    """requests: list of lists of applies, each apply a dict with keys plan
    (handle), tau, p, v (list of tensors), out, vnorms, and optionally
    nscales, skip_phi0, tol.  Returns (latency_ms, queue_ms, makespan_s)."""
    n = len(requests)
    keep = []
    arr = (Request * n)()
    for k, apps in enumerate(requests):
        arr[k].napply = len(apps)
        for a, x in enumerate(apps):
            vp = (ctypes.c_void_p * len(x["v"]))(*[_ptr(t) for t in x["v"]])
            vn = (ctypes.c_double * len(x["vnorms"]))(*[float(t) for t in x["vnorms"]])
            keep += [vp, vn]
            arr[k].apply[a] = ApplyArgs(x["plan"], float(x["tau"]), int(x["p"]), len(x["v"]),
                                        ctypes.cast(vp, ctypes.POINTER(ctypes.c_void_p)), _ptr(x["out"]),
                                        int(x.get("nscales", 1)), int(x.get("skip_phi0", 0)),
                                        float(x.get("tol", 0.0)),
                                        ctypes.cast(vn, ctypes.POINTER(ctypes.c_double)))
    at = (ctypes.c_double * n)(*[float(t) for t in arrivals])
    lat = (ctypes.c_double * n)()
    qd = (ctypes.c_double * n)()
    mk = ctypes.c_double()
    cfg = ServeConfig(int(slots), int(hbm_budget), int(poll_us), int(graphs))
    _check(load().phiks_serve_trace(ctypes.byref(cfg), n, arr, at, lat, qd, ctypes.byref(mk)))
    return list(lat), list(qd), mk.value


def phiks_integrate(plan: int, dims, scheme: int, kind: int, eps: float, alpha: float, t0: float,
                    T: float, steps: int, u, stream=None):
    """Advance u in place with an exponential Runge-Kutta scheme (see include/phiks.h)."""
    n = (ctypes.c_int64 * len(dims))(*[int(m) for m in dims])
    nl = Nonlinear(int(kind), float(eps), float(alpha), 0.0, 0.0)
    _check(load().phiks_integrate(plan, n, len(dims), int(scheme), ctypes.byref(nl), float(t0), float(T),
                                  int(steps), _ptr(u), _stream(stream)))


def phiks_integrate_blocks(plans, scheme: int, kind: int, t0: float, T: float, steps: int, w,
                           eps: float = 0.0, alpha: float = 0.0, a: float = 0.0, b: float = 0.0,
                           stream=None, **opts):
    """Advance w in place for a block-diagonal K = diag(plans) (see include/phiks.h)."""
    arr = (ctypes.c_void_p * len(plans))(*[p.handle if hasattr(p, "handle") else p for p in plans])
    nl = Nonlinear(int(kind), float(eps), float(alpha), float(a), float(b))
    o = make_options(**opts) if opts else None
    _check(load().phiks_integrate_blocks(len(plans), arr, int(scheme), ctypes.byref(nl), float(t0), float(T),
                                         int(steps), _ptr(w), ctypes.byref(o) if o is not None else None,
                                         _stream(stream)))


def phiks_plan_shape(plan: int):
    d = ctypes.c_int()
    n = (ctypes.c_int64 * 8)()
    _check(load().phiks_plan_shape(plan, ctypes.byref(d), n))
    return tuple(int(n[k]) for k in range(d.value))


def phiks_debug_fail_alloc(after: int):
    """Make the library's device allocation after `after` more successes
    fail as out of memory (once); a negative value cancels it."""
    load().phiks_debug_fail_alloc(int(after))


def phiks_debug_live_allocations() -> int:
    """Device allocations the library holds now (all plans)."""
    return int(load().phiks_debug_live_allocations())


def phiks_debug_wait_timeout(plan: int, limit_ms: float, stream=None):
    """Launch the bounded-wait check (a wait nothing ends, limit_ms)."""
    _check(load().phiks_debug_wait_timeout(plan, float(limit_ms), _stream(stream)))


def phiks_get_tuning(plan: int) -> Tuning:
    t = Tuning()
    _check(load().phiks_get_tuning(plan, ctypes.byref(t)))
    return t


def phiks_set_tuning(plan: int, t: Tuning = None, **kw):
    """Set the plan's tuning: a Tuning, or the current one with fields from kw
    (mode_order as a sequence)."""
    if t is None:
        t = phiks_get_tuning(plan)
    for k, v in kw.items():
        if k == "mode_order":
            for j in range(8):
                t.mode_order[j] = int(v[j]) if j < len(v) else -1
        else:
            setattr(t, k, int(v))
    _check(load().phiks_set_tuning(plan, ctypes.byref(t)))
    return t


def phiks_autotune(plan: int, tau: float, p: int, nv: int, reps: int = 5, stream=None, **kw):
    """Time the candidate tunings on this call shape, set and return the
    fastest: (Tuning, ms per apply)."""
    o = make_options(**kw)
    t = Tuning()
    ms = ctypes.c_double()
    _check(load().phiks_autotune(plan, float(tau), int(p), int(nv), ctypes.byref(o), int(reps),
                                 _stream(stream), ctypes.byref(t), ctypes.byref(ms)))
    return t, ms.value


def phiks_destroy(plan: int):
    if plan:
        load().phiks_destroy(plan)


class Plan:
    """Owning wrapper: Plan(A_list, dtype).apply(...)."""

    def __init__(self, A: Sequence[np.ndarray], dtype: int = PHIKS_FP64):
        self.n = [int(np.asarray(a).shape[0]) for a in A]
        self.N = int(np.prod(self.n))
        self.dtype = dtype
        self.handle = phiks_plan(A, dtype)

    def apply(self, tau, p, vs, out, stream=None, **kw):
        if kw:
            phiks_apply_ex(self.handle, tau, p, vs, out, stream, **kw)
        else:
            phiks_apply(self.handle, tau, p, vs, out, stream)
        return out

    def last_params(self):
        return phiks_last_params(self.handle)

    def select_params(self, tau, p, vnorms, **kw):
        return phiks_select_params(self.handle, tau, p, vnorms, **kw)

    def close(self):
        if self.handle:
            phiks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
