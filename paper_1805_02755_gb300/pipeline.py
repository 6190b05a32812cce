"""Copies overlapped with computation for several engines in sequence.

``Overlapped(stages).run()`` runs every stage's engine once, in order, on the
current CUDA stream, with the host-to-device copies of all stages' inputs
issued first on one copy stream and each stage's device-to-host copies issued
on a second copy stream as soon as that stage's run is done: the inputs of
later stages and the outputs of earlier ones move while other stages compute.
A stage's run waits (on the device) only for its own inputs.  ``run()``
returns with every output in host memory.

This is the asynchronous counterpart of an engine with host buffers, whose
``run()`` copies in, computes and copies out before it returns (the
synchronous run of Listing 1).  Host tensors should be pinned, or the copies
are not asynchronous.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch


class Stage:
    """One engine (anything with ``run()`` that launches on the current stream)
    with its input copies (device tensor, host tensor) and output copies
    (host tensor, device tensor)."""

    def __init__(self, engine, inputs: Sequence[Tuple[torch.Tensor, torch.Tensor]] = (),
                 outputs: Sequence[Tuple[torch.Tensor, torch.Tensor]] = ()):
        self.engine = engine
        self.inputs = list(inputs)
        self.outputs = list(outputs)


class Overlapped:
    def __init__(self, stages: List[Stage], device=None):
        self.stages = list(stages)
        self.h2d = torch.cuda.Stream(device=device)
        self.d2h = torch.cuda.Stream(device=device)
        self.bytes_in = sum(h.numel() * h.element_size() for s in self.stages for _, h in s.inputs)
        self.bytes_out = sum(h.numel() * h.element_size() for s in self.stages for h, _ in s.outputs)

    def run(self) -> "Overlapped":
        compute = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(compute)  # copies start after whatever the caller queued before
        ready = []
        with torch.cuda.stream(self.h2d):
            self.h2d.wait_event(start)
            for st in self.stages:
                for d, h in st.inputs:
                    d.copy_(h, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.h2d)
                ready.append(ev)
        self.d2h.wait_event(start)
        for st, ev in zip(self.stages, ready):
            compute.wait_event(ev)
            st.engine.run()
            done = torch.cuda.Event()
            done.record(compute)
            if st.outputs:
                with torch.cuda.stream(self.d2h):
                    self.d2h.wait_event(done)
                    for h, d in st.outputs:
                        h.copy_(d, non_blocking=True)
        self.d2h.synchronize()
        compute.synchronize()
        self.h2d.synchronize()
        return self
