"""CPU oracle for the EngineCL hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library (``paper_1805_02755_gb300``)
never does, and this package imports nothing from it: the two meet only
through the seeded input arrays of ``workloads``.

``oracle.c`` holds the arithmetic (double precision except the FP32
Mandelbrot count, which the method fixes); this module builds it with gcc,
loads it with ctypes and splits large cases into independent unit ranges
run on host threads (ctypes releases the GIL during the foreign call).
``schedule.py`` holds the package sequences of the three schedulers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

from . import schedule  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f32 = ctypes.c_float
_f64 = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.ecl_oracle_mandelbrot.argtypes = [_p, _i64, _i64, _f32, _f32, _f32, _f32, _i32, _i64, _i64]
            L.ecl_oracle_gaussian.argtypes = [_p, _i64, _i64, _p, _i32, _p, _i64, _i64]
            L.ecl_oracle_gaussian_direct.argtypes = [_p, _i64, _i64, _p, _i32, _p]
            L.ecl_oracle_nbody_acc.argtypes = [_p, _i64, _f64, _p, _i64, _i64]
            L.ecl_oracle_nbody_step.argtypes = [_p, _p, _i64, _f64, _f64, _p, _p, _i64, _i64]
            L.ecl_oracle_nbody_energy.argtypes = [_p, _i64, _f64, _i64, _i64]
            L.ecl_oracle_nbody_energy.restype = _f64
            L.ecl_oracle_nbody_energy_row.argtypes = [_p, _i64, _f64, _i64, _p]
            L.ecl_oracle_nbody_energy_row.restype = _f64
            L.ecl_oracle_nbody_energy_grad.argtypes = [_p, _i64, _f64, _p, _i64, _i64]
            L.ecl_oracle_nbody_potential.argtypes = [_p, _i64, _f64, _p, _i64, _i64]
            L.ecl_oracle_binomial.argtypes = [_p, _p, _p, _p, _p, _f64, _i32, _i64, _i64, _p, _p, _p]
            L.ecl_oracle_bf16_round.argtypes = [_f32]
            L.ecl_oracle_bf16_round.restype = _f32
            L.ecl_oracle_bf16_round_array.argtypes = [_p, _p, _i64]
            L.ecl_oracle_gemm_entries.argtypes = [_p, _p, _i64, _i64, _i64, _i32, _p, _p, _i64, _p]
            L.ecl_oracle_ray.argtypes = [_p, _i32, _i32, _i64, _i64, _f32, _f32, _f32, _f32, _i32, _p, _i64, _i64]
            _lib = L
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _split(begin: int, end: int, parts: int):
    n = end - begin
    parts = max(1, min(parts, n)) if n > 0 else 1
    step = -(-n // parts) if n > 0 else 0
    return [(b, min(end, b + step)) for b in range(begin, end, step)] if n > 0 else []


def _run(fn, begin: int, end: int, threads: Optional[int]):
    threads = threads or default_threads()
    ranges = _split(begin, end, threads * 4)
    if threads == 1 or len(ranges) <= 1:
        return [fn(b, e) for b, e in ranges]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda r: fn(*r), ranges))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- Mandelbrot
def mandelbrot(width: int, height: int, x0: float, y0: float, dx: float, dy: float,
               max_iter: int, rows=None, threads: Optional[int] = None) -> np.ndarray:
    """Escape counts (uint32, height x width); ``rows`` = (begin, end) limits work."""
    L = lib()
    out = np.zeros((height, width), dtype=np.uint32)
    b, e = rows if rows is not None else (0, height)
    _run(lambda r0, r1: L.ecl_oracle_mandelbrot(_ptr(out), width, height, x0, y0, dx, dy,
                                                max_iter, r0, r1), b, e, threads)
    return out


# ---------------------------------------------------------------- Gaussian
def gaussian(img: np.ndarray, w: np.ndarray, rows=None, threads: Optional[int] = None) -> np.ndarray:
    """Separable clamp-to-edge blur in FP64 (rows outside ``rows`` stay 0)."""
    L = lib()
    img = _c(img, np.float32)
    w = _c(w, np.float32)
    H, W = img.shape
    out = np.zeros((H, W), dtype=np.float64)
    b, e = rows if rows is not None else (0, H)
    _run(lambda r0, r1: L.ecl_oracle_gaussian(_ptr(img), W, H, _ptr(w), len(w), _ptr(out), r0, r1),
         b, e, threads)
    return out


def gaussian_direct(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    L = lib()
    img = _c(img, np.float32)
    w = _c(w, np.float32)
    H, W = img.shape
    out = np.zeros((H, W), dtype=np.float64)
    L.ecl_oracle_gaussian_direct(_ptr(img), W, H, _ptr(w), len(w), _ptr(out))
    return out


# ---------------------------------------------------------------- NBody
def nbody_acc(pos4: np.ndarray, eps2: float, bodies=None, threads: Optional[int] = None) -> np.ndarray:
    """FP64 accelerations (n x 3); ``bodies`` = (begin, end) limits the rows computed."""
    L = lib()
    pos4 = _c(pos4, np.float32)
    n = pos4.shape[0]
    acc = np.zeros((n, 3), dtype=np.float64)
    b, e = bodies if bodies is not None else (0, n)
    _run(lambda i0, i1: L.ecl_oracle_nbody_acc(_ptr(pos4), n, eps2, _ptr(acc), i0, i1), b, e, threads)
    return acc


def nbody_step(pos4, vel4, dt: float, eps2: float, threads: Optional[int] = None):
    L = lib()
    pos4 = _c(pos4, np.float32)
    vel4 = _c(vel4, np.float32)
    n = pos4.shape[0]
    po = np.zeros((n, 4), dtype=np.float64)
    vo = np.zeros((n, 4), dtype=np.float64)
    _run(lambda i0, i1: L.ecl_oracle_nbody_step(_ptr(pos4), _ptr(vel4), n, dt, eps2,
                                                _ptr(po), _ptr(vo), i0, i1), 0, n, threads)
    return po, vo


def nbody_energy(pos4: np.ndarray, eps2: float, threads: Optional[int] = None, rows=None) -> float:
    """E = -sum_{i<j} m_i m_j (r_ij^2 + eps2)^(-1/2), partial sums added in FP64.

    rows=(b, e) sums only the terms of rows i in [b, e) (all j > i)."""
    L = lib()
    pos4 = _c(pos4, np.float32)
    n = pos4.shape[0]
    b, e = rows if rows is not None else (0, n)
    parts = _run(lambda i0, i1: L.ecl_oracle_nbody_energy(_ptr(pos4), n, eps2, i0, i1), b, e, threads)
    return float(sum(parts))


def nbody_energy_row(pos4: np.ndarray, eps2: float, i: int, q) -> float:
    L = lib()
    pos4 = _c(pos4, np.float32)
    q = _c(q, np.float64)
    return L.ecl_oracle_nbody_energy_row(_ptr(pos4), pos4.shape[0], eps2, int(i), _ptr(q))


def nbody_energy_grad(pos4: np.ndarray, eps2: float, bodies=None,
                      threads: Optional[int] = None) -> np.ndarray:
    L = lib()
    pos4 = _c(pos4, np.float32)
    n = pos4.shape[0]
    g = np.zeros((n, 3), dtype=np.float64)
    b, e = bodies if bodies is not None else (0, n)
    _run(lambda i0, i1: L.ecl_oracle_nbody_energy_grad(_ptr(pos4), n, eps2, _ptr(g), i0, i1),
         b, e, threads)
    return g


def nbody_potential(pos4: np.ndarray, eps2: float, bodies=None,
                    threads: Optional[int] = None) -> np.ndarray:
    """phi_i = sum_{j != i} m_j / sqrt(r_ij^2 + eps2) (so dE/dm_i = -phi_i)."""
    L = lib()
    pos4 = _c(pos4, np.float32)
    n = pos4.shape[0]
    phi = np.zeros(n, dtype=np.float64)
    b, e = bodies if bodies is not None else (0, n)
    _run(lambda i0, i1: L.ecl_oracle_nbody_potential(_ptr(pos4), n, eps2, _ptr(phi), i0, i1), b, e, threads)
    return phi


def nbody_fd_energy_grad(pos4: np.ndarray, eps2: float, idx, comp, h: float):
    """Central differences of the oracle energy in coordinate (idx[t], comp[t]).

    The perturbed coordinate is rounded to FP32 like the input positions, and
    the denominator is the actual FP32 distance between the two placements.
    """
    pos4 = _c(pos4, np.float32)
    out = np.zeros(len(idx), dtype=np.float64)
    for t, (i, c) in enumerate(zip(idx, comp)):
        q = pos4[i, :3].astype(np.float64)
        xp = np.float32(pos4[i, c] + np.float32(h))
        xm = np.float32(pos4[i, c] - np.float32(h))
        qp = q.copy()
        qm = q.copy()
        qp[c] = float(xp)
        qm[c] = float(xm)
        out[t] = (nbody_energy_row(pos4, eps2, i, qp) - nbody_energy_row(pos4, eps2, i, qm)) / \
            (float(xp) - float(xm))
    return out


# ---------------------------------------------------------------- Binomial
def binomial(S, K, T, sigma, steps, r: float, put: bool = False, options=None,
             threads: Optional[int] = None):
    """(price, delta, vega) in FP64 for a CRR European option lattice."""
    L = lib()
    S = _c(S, np.float32)
    K = _c(K, np.float32)
    T = _c(T, np.float32)
    sigma = _c(sigma, np.float32)
    steps = _c(steps, np.int32)
    n = S.shape[0]
    price = np.zeros(n)
    delta = np.zeros(n)
    vega = np.zeros(n)
    b, e = options if options is not None else (0, n)
    _run(lambda o0, o1: L.ecl_oracle_binomial(_ptr(S), _ptr(K), _ptr(T), _ptr(sigma), _ptr(steps),
                                              r, int(put), o0, o1, _ptr(price), _ptr(delta),
                                              _ptr(vega)), b, e, threads)
    return price, delta, vega


# ---------------------------------------------------------------- GEMM
def bf16_round(x: np.ndarray) -> np.ndarray:
    L = lib()
    x = _c(x, np.float32)
    out = np.empty_like(x)
    L.ecl_oracle_bf16_round_array(_ptr(x), _ptr(out), x.size)
    return out


GEMM_BF16, GEMM_FP32_EXACT, GEMM_SPLIT3 = 0, 1, 2


def gemm_entries(A: np.ndarray, Bt: np.ndarray, mode: int, ii, jj,
                 threads: Optional[int] = None) -> np.ndarray:
    """Entries C[ii[t], jj[t]] of A @ Bt.T in FP64 (see oracle.c for the modes)."""
    L = lib()
    A = _c(A, np.float32)
    Bt = _c(Bt, np.float32)
    ii = _c(ii, np.int64)
    jj = _c(jj, np.int64)
    M, K = A.shape
    N = Bt.shape[0]
    out = np.zeros(len(ii), dtype=np.float64)

    def part(t0, t1):
        L.ecl_oracle_gemm_entries(_ptr(A), _ptr(Bt), M, N, K, mode,
                                  _ptr(ii) + 8 * t0, _ptr(jj) + 8 * t0, t1 - t0, _ptr(out) + 8 * t0)
    _run(part, 0, len(ii), threads)
    return out


def gemm(A: np.ndarray, Bt: np.ndarray, mode: int, threads: Optional[int] = None) -> np.ndarray:
    """Full FP64 product for small shapes (every entry through gemm_entries)."""
    M = A.shape[0]
    N = Bt.shape[0]
    ii, jj = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    return gemm_entries(A, Bt, mode, ii.ravel(), jj.ravel(), threads).reshape(M, N)


# ---------------------------------------------------------------- Ray
def ray(scene: np.ndarray, nspheres: int, nlights: int, width: int, height: int, ka: float, bg, max_depth: int,
        rows=None, threads: Optional[int] = None) -> np.ndarray:
    """Whitted ray tracer in FP32 (see oracle.c): (height, width, 4) = r, g, b, rays traced."""
    L = lib()
    scene = _c(scene, np.float32)
    assert scene.size >= 12 * nspheres + 8 * nlights
    out = np.zeros((height, width, 4), dtype=np.float32)
    b, e = rows if rows is not None else (0, height)
    _run(lambda r0, r1: L.ecl_oracle_ray(_ptr(scene), nspheres, nlights, width, height, np.float32(ka),
                                         np.float32(bg[0]), np.float32(bg[1]), np.float32(bg[2]), max_depth,
                                         _ptr(out), r0, r1), b, e, threads)
    return out
