"""Python binding of the EngineCL-style package-scheduling engine (libecl.so).

The functions keep the names of the C ABI in include/ecl.h and only marshal
arguments: handles are ctypes pointers, buffers are torch CUDA tensors
(device memory) or numpy arrays / CPU tensors (host memory, copied by the
engine), and a non-OK status raises :class:`EclError` carrying the engine's
latched error text.  Every computation runs in the CUDA kernels of the
library; there is no Python or CPU fallback, and importing a function that
needs the library fails loudly when libecl.so has not been built.

The ``Engine`` and ``Program`` classes are a convenience layer over the
same calls, mirroring the Tier-1 API of the paper (Sec. 6, Listings 1-2).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libecl.so")

ECL_OK, ECL_ERR_ARG, ECL_ERR_SIZE, ECL_ERR_BUFFER, ECL_ERR_SCHED, ECL_ERR_KERNEL, \
    ECL_ERR_CUDA, ECL_ERR_TIMEOUT, ECL_ERR_STATE = range(9)
STATUS_NAMES = ["ECL_OK", "ECL_ERR_ARG", "ECL_ERR_SIZE", "ECL_ERR_BUFFER", "ECL_ERR_SCHED",
                "ECL_ERR_KERNEL", "ECL_ERR_CUDA", "ECL_ERR_TIMEOUT", "ECL_ERR_STATE"]
ECL_STATIC, ECL_STATIC_REV, ECL_DYNAMIC, ECL_HGUIDED, ECL_MONOLITHIC = range(5)
SCHEDULERS = {"static": ECL_STATIC, "static_rev": ECL_STATIC_REV, "dynamic": ECL_DYNAMIC,
              "hguided": ECL_HGUIDED, "monolithic": ECL_MONOLITHIC}
ECL_ARG_BUF_IN, ECL_ARG_BUF_OUT, ECL_ARG_BUF_OUT_OPT, ECL_ARG_I32, ECL_ARG_I64, ECL_ARG_F32 = range(6)
ECL_DEBUG_SPIN_LIMIT, ECL_DEBUG_WITHHOLD = 1, 2

PKG_STAT_DTYPE = np.dtype([("off_wg", "<u8"), ("len_wg", "<u8"), ("t0_ns", "<u8"), ("t1_ns", "<u8"),
                           ("pkg", "<u4"), ("device", "<u4"), ("cta", "<u4"), ("smid", "<u4")])
WORKER_STAT_DTYPE = np.dtype([("t_first_ns", "<u8"), ("t_last_ns", "<u8"), ("busy_ns", "<u8"),
                              ("cta", "<u4"), ("device", "<u4"), ("smid", "<u4"), ("chunks", "<u4")])


class EclError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message) if message else name)


_lib = None
_vp = ctypes.c_void_p
_st = ctypes.c_int


def lib():
    """Loads libecl.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libecl.so is not built: run __graft_entry__.build() "
                               "(or python paper_1805_02755_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "ecl_engine_create": (_st, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
            "ecl_engine_destroy": (None, [_vp]),
            "ecl_engine_set_stream": (_st, [_vp, _vp]),
            "ecl_engine_copy_streams": (_st, [_vp, _vp, _vp, ctypes.c_int]),
            "ecl_engine_kernel_events": (_st, [_vp, _vp, _vp]),
            "ecl_work_items": (_st, [_vp, ctypes.c_uint64, ctypes.c_uint32]),
            "ecl_scheduler": (_st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
            "ecl_workers": (_st, [_vp, ctypes.c_int, ctypes.c_int]),
            "ecl_engine_program": (_st, [_vp, _vp]),
            "ecl_run": (_st, [_vp]),
            "ecl_synchronize": (_st, [_vp]),
            "ecl_stats": (_st, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "ecl_worker_stats": (_st, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "ecl_set_coverage": (_st, [_vp, _vp, ctypes.c_uint64]),
            "ecl_debug": (_st, [_vp, ctypes.c_int, ctypes.c_int64]),
            "ecl_plan_info": (_st, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                    ctypes.POINTER(ctypes.c_uint32)]),
            "ecl_plan": (_st, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_uint64,
                               ctypes.c_uint64, ctypes.c_uint32, _vp, _vp, _vp, ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_size_t), ctypes.c_char_p, ctypes.c_size_t]),
            "ecl_last_error": (ctypes.c_char_p, [_vp]),
            "ecl_error_count": (ctypes.c_int, [_vp]),
            "ecl_clear_errors": (None, [_vp]),
            "ecl_kernel_occupancy": (_st, [ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
            "ecl_program_create": (_st, [ctypes.POINTER(_vp), ctypes.c_char_p]),
            "ecl_program_destroy": (None, [_vp]),
            "ecl_program_in": (_st, [_vp, _vp, ctypes.c_size_t]),
            "ecl_program_out": (_st, [_vp, _vp, ctypes.c_size_t]),
            "ecl_program_out_pattern": (_st, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
            "ecl_program_arg": (_st, [_vp, ctypes.c_int, _vp, ctypes.c_size_t]),
            "ecl_program_local": (_st, [_vp, ctypes.c_int, ctypes.c_size_t]),
            "ecl_kernel_arg": (_st, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_char_p)]),
            "ecl_nbody_energy_noalloc": (_st, [_vp, ctypes.c_int32, ctypes.c_float, _vp, _vp]),
            "ecl_kernel_count": (ctypes.c_int, []),
            "ecl_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    """Names of the C ABI functions the binding declares."""
    lib()
    return sorted(n for n in dir(_lib) if n.startswith("ecl_"))


def _check(status: int, engine=None):
    if status != ECL_OK:
        msg = ""
        if engine is not None:
            msg = (lib().ecl_last_error(engine) or b"").decode()
        raise EclError(status, msg)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ raw calls
def ecl_engine_create(device_ordinal: int = 0, cuda_stream=None):
    h = _vp()
    _check(lib().ecl_engine_create(ctypes.byref(h), device_ordinal, _vp(_stream_handle(cuda_stream))))
    return h


def ecl_engine_destroy(e) -> None:
    lib().ecl_engine_destroy(e)


def ecl_engine_set_stream(e, cuda_stream) -> None:
    _check(lib().ecl_engine_set_stream(e, _vp(_stream_handle(cuda_stream))), e)


def ecl_engine_copy_streams(e, h2d_stream=None, d2h_stream=None, asynchronous: bool = True) -> None:
    h2d = 0 if h2d_stream is None else _stream_handle(h2d_stream)  # None: the engine's own stream
    d2h = 0 if d2h_stream is None else _stream_handle(d2h_stream)
    _check(lib().ecl_engine_copy_streams(e, _vp(h2d), _vp(d2h), 1 if asynchronous else 0), e)


def _event_handle(ev) -> int:
    if ev is None:
        return 0
    if isinstance(ev, int):
        return ev
    return ev.cuda_event  # torch.cuda.Event (created with enable_timing=True)


def ecl_engine_kernel_events(e, begin=None, end=None) -> None:
    _check(lib().ecl_engine_kernel_events(e, _vp(_event_handle(begin)), _vp(_event_handle(end))), e)


def ecl_work_items(e, gws: int, lws: int) -> None:
    _check(lib().ecl_work_items(e, gws, lws), e)


def ecl_scheduler(e, kind, params: Sequence[float] = ()) -> None:
    if isinstance(kind, str):
        kind = SCHEDULERS[kind]
    arr = (ctypes.c_double * max(1, len(params)))(*params)
    _check(lib().ecl_scheduler(e, int(kind), arr, len(params)), e)


def ecl_workers(e, devices: int = 0, ctas_per_device: int = 0) -> None:
    _check(lib().ecl_workers(e, devices, ctas_per_device), e)


def ecl_engine_program(e, p) -> None:
    _check(lib().ecl_engine_program(e, p), e)


def ecl_run(e) -> None:
    _check(lib().ecl_run(e), e)


def ecl_synchronize(e) -> None:
    _check(lib().ecl_synchronize(e), e)


def ecl_stats(e, cap: int = 1 << 20) -> np.ndarray:
    out = np.zeros(cap, dtype=PKG_STAT_DTYPE)
    n = ctypes.c_size_t()
    _check(lib().ecl_stats(e, out.ctypes.data, cap, ctypes.byref(n)), e)
    return out[: n.value].copy()


def ecl_worker_stats(e, cap: int = 1 << 16) -> np.ndarray:
    out = np.zeros(cap, dtype=WORKER_STAT_DTYPE)
    n = ctypes.c_size_t()
    _check(lib().ecl_worker_stats(e, out.ctypes.data, cap, ctypes.byref(n)), e)
    return out[: n.value].copy()


def ecl_set_coverage(e, counts) -> None:
    if counts is None:
        _check(lib().ecl_set_coverage(e, None, 0), e)
    else:
        _check(lib().ecl_set_coverage(e, _vp(counts.data_ptr()), counts.numel()), e)


def ecl_debug(e, kind: int, value: int) -> None:
    _check(lib().ecl_debug(e, int(kind), int(value)), e)


def chrome_trace(stats: np.ndarray, path: Optional[str] = None, name: str = "ecl") -> dict:
    """Per-package records (``ecl_stats``) as a Chrome trace (chrome://tracing,
    Perfetto): one complete event per package, process = device, thread = the
    CTA that fetched it, times in microseconds from the first fetch.  Written
    to ``path`` when given; the trace dict is returned either way."""
    events = []
    t0 = int(stats["t0_ns"].min()) if len(stats) else 0
    for r in stats:
        events.append({"name": "pkg %d" % int(r["pkg"]), "cat": name, "ph": "X",
                       "ts": (int(r["t0_ns"]) - t0) / 1e3, "dur": max(0, int(r["t1_ns"]) - int(r["t0_ns"])) / 1e3,
                       "pid": int(r["device"]), "tid": int(r["cta"]),
                       "args": {"off_wg": int(r["off_wg"]), "len_wg": int(r["len_wg"]), "smid": int(r["smid"])}})
    trace = {"traceEvents": events, "displayTimeUnit": "ns"}
    if path:
        import json
        with open(path, "w") as f:
            json.dump(trace, f)
    return trace


def ecl_plan_info(e) -> dict:
    G = ctypes.c_uint64()
    P = ctypes.c_uint64()
    D = ctypes.c_uint32()
    C = ctypes.c_uint32()
    N = ctypes.c_uint32()
    _check(lib().ecl_plan_info(e, ctypes.byref(G), ctypes.byref(P), ctypes.byref(D), ctypes.byref(C),
                               ctypes.byref(N)), e)
    return dict(G=G.value, packages=P.value, devices=D.value, ctas_per_device=C.value, ctas=N.value)


def ecl_plan(kind, params: Sequence[float], G: int, grain: int = 1, devices: int = 1):
    """Host-side package plan: arrays (off_wg, len_wg, device) in hand-out order."""
    if isinstance(kind, str):
        kind = SCHEDULERS[kind]
    arr = (ctypes.c_double * max(1, len(params)))(*params)
    n = ctypes.c_size_t()
    err = ctypes.create_string_buffer(512)
    L = lib()
    st = L.ecl_plan(int(kind), arr, len(params), G, grain, devices, None, None, None, 0,
                    ctypes.byref(n), err, 512)
    if st not in (ECL_OK, ECL_ERR_SIZE):
        raise EclError(st, err.value.decode())
    cap = n.value
    off = np.zeros(cap, dtype=np.uint64)
    ln = np.zeros(cap, dtype=np.uint64)
    dev = np.zeros(cap, dtype=np.uint32)
    st = L.ecl_plan(int(kind), arr, len(params), G, grain, devices, off.ctypes.data, ln.ctypes.data,
                    dev.ctypes.data, cap, ctypes.byref(n), err, 512)
    if st != ECL_OK:
        raise EclError(st, err.value.decode())
    return off, ln, dev


def ecl_last_error(e) -> str:
    return (lib().ecl_last_error(e) or b"").decode()


def ecl_error_count(e) -> int:
    return lib().ecl_error_count(e)


def ecl_clear_errors(e) -> None:
    lib().ecl_clear_errors(e)


def ecl_kernel_occupancy(kernel_name: str, device_ordinal: int = 0):
    sms = ctypes.c_int()
    per = ctypes.c_int()
    _check(lib().ecl_kernel_occupancy(device_ordinal, kernel_name.encode(), ctypes.byref(sms),
                                      ctypes.byref(per)))
    return sms.value, per.value


def ecl_program_create(kernel_name: str):
    h = _vp()
    _check(lib().ecl_program_create(ctypes.byref(h), kernel_name.encode()))
    return h


def ecl_program_destroy(p) -> None:
    lib().ecl_program_destroy(p)


def _addr_bytes(buf):
    """(address, bytes, keepalive) of a torch tensor or numpy array."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous")
        return buf.ctypes.data, buf.nbytes, buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return buf.data_ptr(), buf.numel() * buf.element_size(), buf
    raise TypeError("buffer must be a torch tensor or a numpy array")


def ecl_program_in(p, buf) -> None:
    a, n, _ = _addr_bytes(buf)
    _check(lib().ecl_program_in(p, _vp(a), n))


def ecl_program_out(p, buf) -> None:
    a, n, _ = _addr_bytes(buf)
    _check(lib().ecl_program_out(p, _vp(a), n))


def ecl_program_out_pattern(p, outs: int, work_items: int) -> None:
    _check(lib().ecl_program_out_pattern(p, outs, work_items))


def ecl_kernel_arg(kernel_name: str, index: int):
    kind = ctypes.c_int()
    name = ctypes.c_char_p()
    st = lib().ecl_kernel_arg(kernel_name.encode(), index, ctypes.byref(kind), ctypes.byref(name))
    if st != ECL_OK:
        return None
    return kind.value, name.value.decode()


def _noalloc_check(pos4, n: int, out_energy) -> None:
    """The C entry point sees bare addresses and cannot check buffer sizes:
    pos4 must be a contiguous float32 tensor of at least 4 n values and
    out_energy a contiguous float64 tensor of at least one value, both on the
    current CUDA device.  Raises ValueError otherwise."""
    import torch
    for name, t, dt, need in (("pos4", pos4, torch.float32, 4 * max(int(n), 0)),
                              ("out_energy", out_energy, torch.float64, 1)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != dt:
            raise ValueError("%s must be %s, not %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() < need:
            raise ValueError("%s holds %d values, %d needed" % (name, t.numel(), need))
    for name, t in (("pos4", pos4), ("out_energy", out_energy)):
        if t.device.type != "cuda" or t.device.index != torch.cuda.current_device():
            raise ValueError("%s must be on the current CUDA device" % name)


def ecl_nbody_energy_noalloc(pos4, n: int, eps2: float, out_energy, cuda_stream=None) -> None:
    """Potential energy into out_energy (device double[1]) without allocating;
    see include/ecl.h for the limits (n <= 524288, one shared scratch array).
    The tensors are checked first (dtype, contiguity, size, device)."""
    _noalloc_check(pos4, n, out_energy)
    _check(lib().ecl_nbody_energy_noalloc(_vp(pos4.data_ptr()), n, eps2, _vp(out_energy.data_ptr()),
                                          _vp(_stream_handle(cuda_stream))))


def ecl_kernel_count() -> int:
    return lib().ecl_kernel_count()


def ecl_kernel_name(i: int) -> Optional[str]:
    r = lib().ecl_kernel_name(i)
    return r.decode() if r is not None else None


def ecl_kernel_names():
    L = lib()
    return [L.ecl_kernel_name(i).decode() for i in range(L.ecl_kernel_count())]


def ecl_program_arg(p, index: int, value, kind: int) -> None:
    """Sets argument `index` from a Python value of the declared ECL_ARG_* kind."""
    if kind in (ECL_ARG_BUF_IN, ECL_ARG_BUF_OUT, ECL_ARG_BUF_OUT_OPT):
        addr = 0 if value is None else _addr_bytes(value)[0]
        c = ctypes.c_void_p(addr)
    elif kind == ECL_ARG_I32:
        c = ctypes.c_int32(int(value))
    elif kind == ECL_ARG_I64:
        c = ctypes.c_int64(int(value))
    elif kind == ECL_ARG_F32:
        c = ctypes.c_float(float(value))
    else:
        raise ValueError("unknown argument kind %r" % kind)
    _check(lib().ecl_program_arg(p, index, ctypes.byref(c), ctypes.sizeof(c)))


def ecl_program_local(p, index: int, nbytes: int) -> None:
    _check(lib().ecl_program_local(p, index, nbytes))


# ------------------------------------------------------------------ classes
class Program:
    """A kernel with its buffers, arguments and output pattern (Listing 1)."""

    def __init__(self, kernel_name: str):
        self.kernel = kernel_name
        self.h = ecl_program_create(kernel_name)
        self.kinds = []
        i = 0
        while True:
            r = ecl_kernel_arg(kernel_name, i)
            if r is None:
                break
            self.kinds.append(r)
            i += 1
        self._keep = []
        self._next = 0
        self.owned = False

    def in_(self, buf):
        ecl_program_in(self.h, buf)
        self._keep.append(buf)
        return self

    def out(self, buf):
        ecl_program_out(self.h, buf)
        self._keep.append(buf)
        return self

    def out_pattern(self, outs: int, work_items: int):
        ecl_program_out_pattern(self.h, outs, work_items)
        return self

    def arg(self, index: Optional[int], value):
        """Positional (index given) or aggregate (index None) argument."""
        i = self._next if index is None else index
        if i >= len(self.kinds):
            raise EclError(ECL_ERR_ARG, "%s takes %d arguments" % (self.kernel, len(self.kinds)))
        ecl_program_arg(self.h, i, value, self.kinds[i][0])
        if value is not None and not isinstance(value, (int, float)):
            self._keep.append(value)
        self._next = i + 1
        return self

    def args(self, *values):
        for v in values:
            self.arg(None, v)
        return self

    def __del__(self):
        try:
            if not self.owned and self.h:
                ecl_program_destroy(self.h)
        except Exception:
            pass


def current_device(device: Optional[int] = None) -> int:
    """`device`, or torch's current CUDA device when it is None (the GPU this
    process was given, e.g. LOCAL_RANK's under torchrun)."""
    if device is not None:
        return int(device)
    import torch
    return torch.cuda.current_device()


class Engine:
    """Engine bound to one GPU and one stream (the Tier-1 EngineCL object).
    `device` None: torch's current CUDA device."""

    def __init__(self, device: Optional[int] = None, stream=None):
        self.h = ecl_engine_create(current_device(device), stream)
        self.program_obj = None

    def close(self):
        if self.h:
            ecl_engine_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def work_items(self, gws: int, lws: int):
        ecl_work_items(self.h, gws, lws)
        return self

    def scheduler(self, kind, params: Sequence[float] = ()):
        ecl_scheduler(self.h, kind, params)
        return self

    def workers(self, devices: int = 0, ctas_per_device: int = 0):
        ecl_workers(self.h, devices, ctas_per_device)
        return self

    def program(self, prog: Program):
        ecl_engine_program(self.h, prog.h)
        prog.owned = True
        self.program_obj = prog  # keeps its buffers alive
        return self

    def set_stream(self, stream):
        ecl_engine_set_stream(self.h, stream)
        return self

    def copy_streams(self, h2d=None, d2h=None, asynchronous: bool = True):
        """Host-buffer copies on their own streams, event-ordered around the
        launch; with asynchronous=True run() returns at once and
        synchronize() waits for the results (include/ecl.h)."""
        ecl_engine_copy_streams(self.h, h2d, d2h, asynchronous)
        return self

    def kernel_events(self, begin=None, end=None):
        """Events recorded right before and after each later run's main
        kernel (include/ecl.h); None, None clears them."""
        ecl_engine_kernel_events(self.h, begin, end)
        self._kernel_events = (begin, end)  # kept alive with the engine
        return self

    def run(self):
        ecl_run(self.h)
        trace_dir = os.environ.get("ECL_TRACE")
        if trace_dir:  # debugging aid: every run's packages as a Chrome trace (synchronises)
            os.makedirs(trace_dir, exist_ok=True)
            Engine._traces = getattr(Engine, "_traces", 0) + 1
            kernel = self.program_obj.kernel if self.program_obj is not None else "run"
            self.trace(os.path.join(trace_dir, "ecl_%s_%04d.json" % (kernel, Engine._traces)))
        return self

    def synchronize(self):
        ecl_synchronize(self.h)
        return self

    def stats(self) -> np.ndarray:
        return ecl_stats(self.h)

    def worker_stats(self) -> np.ndarray:
        return ecl_worker_stats(self.h)

    def plan_info(self) -> dict:
        return ecl_plan_info(self.h)

    def set_coverage(self, counts):
        ecl_set_coverage(self.h, counts)
        return self

    def debug(self, kind: int, value: int):
        ecl_debug(self.h, kind, value)
        return self

    def trace(self, path: Optional[str] = None) -> dict:
        """The last run's packages as a Chrome trace (see chrome_trace).  With the
        environment variable ECL_TRACE set to a directory, every run writes one."""
        return chrome_trace(self.stats(), path)

    def last_error(self) -> str:
        return ecl_last_error(self.h)

    def has_errors(self) -> bool:
        return ecl_error_count(self.h) > 0

    def clear_errors(self):
        ecl_clear_errors(self.h)
        return self
