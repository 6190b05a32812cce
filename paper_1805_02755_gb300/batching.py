"""Batched launches and CUDA-graph replay.

``BinomialBatch`` prices many option batches of uneven size in ONE persistent
launch (the "binomial_batch" program): a device table of
``ecl_binomial_instance`` entries (layout in include/ecl.h) maps every
work-group of the concatenated NDRange to its batch.  ``capture_graph``
records an engine's run into a CUDA graph (after one eager run has uploaded
the package plan, so the captured work is the kernel launch alone) for
replay without host launch overhead.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import Engine, Program

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

    def __init__(self, batches: Sequence[Dict], with_greeks: bool = True, device: int = 0,
                 scheduler=("hguided", (2.0, 1.0)), workers=(8, 0), stream=None):
        self.batches = list(batches)
        tab = np.zeros(len(self.batches), dtype=INSTANCE_DTYPE)
        first = 0
        for i, b in enumerate(self.batches):
            n = int(b["S"].numel())
            tab[i] = (_ptr(b["S"]), _ptr(b["K"]), _ptr(b["T"]), _ptr(b["sigma"]), _ptr(b["steps"]),
                      _ptr(b["price"]), _ptr(b.get("greeks")), first, n, float(b["r"]), 0)
            first += n
        self.total = first
        self.table = torch.from_numpy(tab.view(np.uint8).copy()).to(f"cuda:{device}")
        self.engine = Engine(device, stream)
        self.program = Program("binomial_batch").in_(self.table).args(self.table, len(self.batches), self.total,
                                                                      1 if with_greeks else 0)
        self.engine.work_items(self.total * 32, 32).scheduler(*scheduler).workers(*workers)
        self.engine.program(self.program)

    def run(self):
        self.engine.run()
        return self

    def close(self):
        self.engine.close()


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
