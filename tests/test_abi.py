"""The C ABI library builds, loads and exports every symbol include/ecl.h declares.

Only host-side calls run here (no GPU): program creation, argument checks and
the package planner.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KERNELS = ["mandelbrot", "gaussian", "gaussian_batch", "mandelbrot_batch", "nbody", "nbody_acc", "nbody_adjoint", "nbody_energy", "nbody_fd", "binomial", "binomial_batch", "binomial_full", "gemm_bf16", "gemm_split3", "gemm_split6", "cast_bf16", "ray", "fp32_probe"]


@pytest.fixture(scope="module")
def E():
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ecl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ecl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["ecl_engine_create", "ecl_engine_destroy", "ecl_program_create", "ecl_program_in",
              "ecl_program_out", "ecl_program_out_pattern", "ecl_program_arg", "ecl_program_local",
              "ecl_engine_program", "ecl_work_items", "ecl_scheduler", "ecl_workers", "ecl_run",
              "ecl_stats", "ecl_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(E):
    L = ctypes.CDLL(E.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_uses_the_same_names(E):
    for n in declared_functions():
        assert hasattr(E, n), n


def test_builtin_kernels(E):
    assert E.ecl_kernel_names() == KERNELS
    # Table 2: Mandelbrot takes 8 arguments
    kinds = []
    i = 0
    while E.ecl_kernel_arg("mandelbrot", i) is not None:
        kinds.append(E.ecl_kernel_arg("mandelbrot", i))
        i += 1
    assert len(kinds) == 8 and kinds[0] == (E.ECL_ARG_BUF_OUT, "out")


def test_program_errors_without_gpu(E):
    with pytest.raises(E.EclError) as ei:
        E.ecl_program_create("no_such_kernel")
    assert ei.value.status == E.ECL_ERR_KERNEL
    p = E.ecl_program_create("mandelbrot")
    try:
        L = E.lib()
        v = ctypes.c_int32(5)
        assert L.ecl_program_arg(p, 8, ctypes.byref(v), 4) == E.ECL_ERR_ARG      # past the last arg
        assert L.ecl_program_arg(p, 1, ctypes.byref(v), 8) == E.ECL_ERR_ARG      # wrong size
        assert L.ecl_program_arg(p, 1, ctypes.byref(v), 4) == E.ECL_OK
        assert L.ecl_program_arg(p, -1, ctypes.byref(v), 4) == E.ECL_OK          # aggregate: index 2
        assert L.ecl_program_local(p, 3, 1024) == E.ECL_ERR_ARG                  # no local args
        assert L.ecl_program_out_pattern(p, 0, 1) == E.ECL_ERR_ARG
        assert L.ecl_program_in(p, None, 16) == E.ECL_ERR_ARG
    finally:
        E.ecl_program_destroy(p)


def test_null_handles(E):
    L = E.lib()
    assert L.ecl_run(None) == E.ECL_ERR_ARG
    assert L.ecl_work_items(None, 1, 1) == E.ECL_ERR_ARG
    assert L.ecl_synchronize(None) == E.ECL_ERR_ARG
    assert L.ecl_engine_create(None, 0, None) == E.ECL_ERR_ARG
    L.ecl_engine_destroy(None)
    assert L.ecl_last_error(None) == b"NULL engine"
    assert L.ecl_engine_kernel_events(None, None, None) == E.ECL_ERR_ARG


def _table2():
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_properties.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, lws, rw, outp, nargs = line.split()
            r, w = (int(v) for v in rw.split(":"))
            rows[name] = dict(lws=int(lws), reads=r, writes=w, out=outp, args=int(nargs))
    return rows


def _kernel_args(E, name):
    out = []
    while E.ecl_kernel_arg(name, len(out)) is not None:
        out.append(E.ecl_kernel_arg(name, len(out)))
    return out


@pytest.mark.parametrize("name", ["gaussian", "ray", "mandelbrot", "nbody"])
def test_table2_argument_and_buffer_counts(E, name):
    """The built-in kernels of these benchmarks take Table 2's number of
    arguments and of read and written buffers."""
    want = _table2()[name]
    args = _kernel_args(E, name)
    reads = sum(1 for k, _ in args if k == E.ECL_ARG_BUF_IN)
    writes = sum(1 for k, _ in args if k in (E.ECL_ARG_BUF_OUT, E.ECL_ARG_BUF_OUT_OPT))
    assert (len(args), reads, writes) == (want["args"], want["reads"], want["writes"])


def test_table2_binomial_differs_as_documented(E):
    """Table 2's binomial prices one fixed-depth lattice per 255-wide
    work-group (5 arguments, 1:1 buffers, out 1:255); this one prices a batch
    of options of uneven depth (1..2048), one warp each, with delta and vega:
    9 arguments, 5 read buffers (S, K, T, sigma, depth), price and greeks
    written."""
    want = _table2()["binomial"]
    args = _kernel_args(E, "binomial")
    reads = sum(1 for k, _ in args if k == E.ECL_ARG_BUF_IN)
    writes = sum(1 for k, _ in args if k in (E.ECL_ARG_BUF_OUT, E.ECL_ARG_BUF_OUT_OPT))
    assert (len(args), reads, writes) == (9, 5, 2)
    assert (len(args), reads, writes) != (want["args"], want["reads"], want["writes"])


@pytest.mark.parametrize("case", ["pos_dtype", "pos_short", "pos_strided", "pos_numpy", "out_dtype", "out_empty",
                                  "on_host"])
def test_noalloc_energy_wrapper_rejects_bad_tensors(E, case):
    # The no-allocation energy call hands bare addresses to C, which cannot
    # see sizes: the binding checks dtype, contiguity, size and device before
    # any CUDA call (these run on the CPU and never reach the library).
    import numpy as np
    import torch
    n = 8
    pos = torch.zeros((n, 4), dtype=torch.float32)
    out = torch.zeros(1, dtype=torch.float64)
    msg = "current CUDA device"
    if case == "pos_dtype":
        pos, msg = pos.double(), "pos4 must be torch.float32"
    elif case == "pos_short":
        pos, msg = torch.zeros((n - 1, 4)), "pos4 holds 28 values, 32 needed"
    elif case == "pos_strided":
        pos, msg = torch.zeros((n, 8))[:, :4], "pos4 must be contiguous"
    elif case == "pos_numpy":
        pos, msg = np.zeros((n, 4), np.float32), "pos4 must be a torch tensor"
    elif case == "out_dtype":
        out, msg = out.float(), "out_energy must be torch.float64"
    elif case == "out_empty":
        out, msg = torch.zeros(0, dtype=torch.float64), "out_energy holds 0 values, 1 needed"
    with pytest.raises(ValueError, match=msg):
        E.ecl_nbody_energy_noalloc(pos, n, 1e-3, out)
