"""Batched launches and CUDA-graph replay.

Many instances of one program, of uneven size, run as ONE concatenated
NDRange in one persistent launch: a device table (layouts in include/ecl.h)
gives every instance its first work-group, and a work-group finds its
instance by binary search.  The package schedulers cut the concatenated
NDRange like any other (Sec. 5.3), so a package may span instances.

* ``BinomialBatch``: option batches ("binomial_batch", one work-group per
  option).
* ``MandelbrotBatch``: views of any size, window and iteration count
  ("mandelbrot_batch", 1024 pixels per work-group).
* ``GaussianBatch``: 31-tap images of any size with their own weights
  ("gaussian_batch", one 32 x 224 output tile per work-group).

A tuned configuration (``autotune.autotune(...)["config"]``) sets the
batch's scheduler and workers through ``autotune.apply``.  ``capture_graph``
records an engine's run into a CUDA graph (after one eager run has uploaded
the package plan, so the captured work is the kernel launch alone) for
replay without host launch overhead.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import Engine, Program, current_device

VIEW_DTYPE = np.dtype([("out", "<u8"), ("W", "<i4"), ("H", "<i4"), ("x0", "<f4"), ("y0", "<f4"), ("dx", "<f4"),
                       ("dy", "<f4"), ("max_iter", "<i4"), ("pad", "<i4"), ("first", "<i8"), ("wgs", "<i8")])
assert VIEW_DTYPE.itemsize == 56
IMAGE_DTYPE = np.dtype([("in", "<u8"), ("out", "<u8"), ("w", "<u8"), ("W", "<i4"), ("H", "<i4"),
                        ("first", "<i8"), ("tiles", "<i8")])
assert IMAGE_DTYPE.itemsize == 48

INSTANCE_DTYPE = np.dtype([("S", "<u8"), ("K", "<u8"), ("T", "<u8"), ("sigma", "<u8"), ("steps", "<u8"),
                           ("price", "<u8"), ("greeks", "<u8"), ("first", "<i8"), ("n", "<i8"),
                           ("r", "<f4"), ("pad", "<i4")])
assert INSTANCE_DTYPE.itemsize == 80


def _ptr(t: Optional[torch.Tensor]) -> int:
    return 0 if t is None else t.data_ptr()


class BinomialBatch:
    """Many binomial batches, one launch.

    ``batches``: sequence of dicts with CUDA tensors S, K, T, sigma (float32),
    steps (int32), price (float32 out), optional greeks (float32 (n, 2) out)
    and a float r.
    """

    def __init__(self, batches: Sequence[Dict], with_greeks: bool = True, device: Optional[int] = None,
                 scheduler=("hguided", (2.0, 1.0)), workers=(8, 0), stream=None, config: Optional[Dict] = None):
        self.batches = list(batches)
        tab = np.zeros(len(self.batches), dtype=INSTANCE_DTYPE)
        first = 0
        for i, b in enumerate(self.batches):
            n = int(b["S"].numel())
            tab[i] = (_ptr(b["S"]), _ptr(b["K"]), _ptr(b["T"]), _ptr(b["sigma"]), _ptr(b["steps"]),
                      _ptr(b["price"]), _ptr(b.get("greeks")), first, n, float(b["r"]), 0)
            first += n
        self.total = first
        device = current_device(device)
        self.table = torch.from_numpy(tab.view(np.uint8).copy()).to(f"cuda:{device}")
        self.engine = Engine(device, stream)
        self.program = Program("binomial_batch").in_(self.table).args(self.table, len(self.batches), self.total,
                                                                      1 if with_greeks else 0)
        self.engine.work_items(self.total * 32, 32).scheduler(*scheduler).workers(*workers)
        if config is not None:
            from .autotune import apply
            apply(self.engine, config)
        self.engine.program(self.program)

    def run(self):
        self.engine.run()
        return self

    def close(self):
        self.engine.close()


def _check_dev(t: torch.Tensor, dtype, numel: int, name: str, align: int = 4) -> None:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor" % (name, dtype))
    if t.numel() < numel:
        raise ValueError("%s holds %d values, %d needed" % (name, t.numel(), numel))
    if t.data_ptr() % align:
        raise ValueError("%s must be %d-byte aligned" % (name, align))


class _TableBatch:
    """One persistent launch over a device table of instances."""

    kernel = ""
    lws = 256

    def _finish(self, tab: np.ndarray, total: int, device: Optional[int], scheduler, workers, stream,
                config) -> None:
        self.total = total
        device = current_device(device)
        self.table = torch.from_numpy(tab.view(np.uint8).copy()).to(f"cuda:{device}")
        self.engine = Engine(device, stream)
        self.program = Program(self.kernel).in_(self.table).args(self.table, len(tab), total)
        self.engine.work_items(total * self.lws, self.lws).scheduler(*scheduler).workers(*workers)
        if config is not None:
            from .autotune import apply
            apply(self.engine, config)
        self.engine.program(self.program)

    def make_program(self):
        """A fresh program over the same table (for the autotuner)."""
        return Program(self.kernel).in_(self.table).args(self.table, len(self.table) // self.entry, self.total)

    def run(self):
        self.engine.run()
        return self

    def close(self):
        self.engine.close()


class MandelbrotBatch(_TableBatch):
    """Many Mandelbrot views, one launch.

    ``views``: sequence of dicts with ``out`` (CUDA int32/uint32 tensor of
    W*H values, 16-byte aligned), ``W``, ``H``, ``x0``, ``y0``, ``dx``,
    ``dy`` and ``max_iter``.
    """

    kernel = "mandelbrot_batch"
    lws = 256
    entry = VIEW_DTYPE.itemsize

    @staticmethod
    def workgroups(W: int, H: int) -> int:
        return -(-(W * H) // (4 * 256))

    def __init__(self, views: Sequence[Dict], device: Optional[int] = None, scheduler=("hguided", (2.0, 1.0)),
                 workers=(0, 0), stream=None, config: Optional[Dict] = None):
        self.views = list(views)
        tab = np.zeros(len(self.views), dtype=VIEW_DTYPE)
        first = 0
        for i, v in enumerate(self.views):
            W, H = int(v["W"]), int(v["H"])
            if W <= 0 or H <= 0:
                raise ValueError("view %d: width and height must be positive" % i)
            if v["max_iter"] < 0:
                raise ValueError("view %d: max_iter must be >= 0" % i)
            _check_dev(v["out"], v["out"].dtype, W * H, "view %d out" % i, 16)
            if v["out"].element_size() != 4:
                raise ValueError("view %d out must hold 32-bit counts" % i)
            n = self.workgroups(W, H)
            tab[i] = (v["out"].data_ptr(), W, H, v["x0"], v["y0"], v["dx"], v["dy"], int(v["max_iter"]), 0, first, n)
            first += n
        self._finish(tab, first, device, scheduler, workers, stream, config)


class GaussianBatch(_TableBatch):
    """Many 31-tap Gaussian images, one launch.

    ``images``: sequence of dicts with ``in`` and ``out`` (CUDA float32
    tensors of W*H values, ``out`` 16-byte aligned), ``w`` (CUDA float32
    tensor of 31 weights), ``W`` and ``H``.
    """

    kernel = "gaussian_batch"
    lws = 256
    entry = IMAGE_DTYPE.itemsize

    @staticmethod
    def tiles(W: int, H: int) -> int:
        return -(-H // 32) * -(-W // 224)

    def __init__(self, images: Sequence[Dict], device: Optional[int] = None, scheduler=("hguided", (2.0, 1.0)),
                 workers=(0, 0), stream=None, config: Optional[Dict] = None):
        self.images = list(images)
        tab = np.zeros(len(self.images), dtype=IMAGE_DTYPE)
        first = 0
        for i, im in enumerate(self.images):
            W, H = int(im["W"]), int(im["H"])
            if W <= 0 or H <= 0:
                raise ValueError("image %d: width and height must be positive" % i)
            _check_dev(im["in"], torch.float32, W * H, "image %d in" % i)
            _check_dev(im["out"], torch.float32, W * H, "image %d out" % i, 16)
            _check_dev(im["w"], torch.float32, 31, "image %d weights" % i)
            n = self.tiles(W, H)
            tab[i] = (im["in"].data_ptr(), im["out"].data_ptr(), im["w"].data_ptr(), W, H, first, n)
            first += n
        self._finish(tab, first, device, scheduler, workers, stream, config)


def capture_graph(engine: Engine, stream: Optional[torch.cuda.Stream] = None) -> torch.cuda.CUDAGraph:
    """Records one ``engine.run()`` into a CUDA graph and returns it.

    The engine runs once eagerly on the capture stream first, so the package
    plan (and any workspace) already exists and the captured work is the
    persistent launch alone; the device queue resets itself at the end of
    every run, so the graph can be replayed any number of times.
    """
    s = stream or torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    engine.set_stream(s)
    with torch.cuda.stream(s):
        engine.run()
    s.synchronize()
    with torch.cuda.graph(g, stream=s):
        engine.run()
    engine.set_stream(torch.cuda.current_stream())
    return g


def split_uneven(n: int, parts: int, seed: int = 0) -> List[int]:
    """Batch sizes that sum to n, skewed (a few large, many small)."""
    if parts < 1 or n < parts:
        raise ValueError("need 1 <= parts <= n")
    rng = np.random.default_rng(seed)
    w = rng.pareto(1.5, parts) + 0.05
    sizes = 1 + np.floor(w / w.sum() * (n - parts)).astype(np.int64)  # every batch non-empty
    sizes[np.argmax(w)] += n - sizes.sum()
    return [int(x) for x in sizes]
