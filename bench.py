#!/usr/bin/env python
"""Benchmark of the hot path: one step = one run of every configured program.

Configurations (seeded synthetic inputs, see workloads.py):
  mandelbrot  1024x1024, [-2,1]x[-1.5,1.5], 256 iterations, Static, one package
  gaussian    8192x8192 FP32, 31 taps sigma 5, clamp, Dynamic 256 row packages
  nbody       65536 bodies, eps^2 1e-3, HGuided: force, energy, adjoint, 256 FD samples
  binomial    2^20 options, depths U{256..2048}, price + delta + vega, HGuided
  gemm        8192^3, HGuided 128-row tiles: BF16 and split-BF16 three-product
Beside the step (own per-kernel entries, not in the step's value): the
six-product GEMM, the ray tracer (2048^2, 64 spheres) and Mandelbrot scaled
up to 8192^2 pixels and 1024 iterations.

With N GPUs (torchrun) every rank runs the whole step on its own GPU
(replicas); the step time is the slowest rank's and value counts all ranks.

Each program is one ecl_run() through the C ABI (one persistent launch).  The
JSON line reports:
  value        work-items per second over the whole step (device-timed, inputs
               resident in HBM, L2 flushed before every step)
  e2e          the same from pinned HOST memory through the C ABI (host
               buffers registered in the programs): every step copies its
               inputs in and its results out inside the timed region, the
               copies on two copy streams ordered around each launch by
               events (ecl_engine_copy_streams), runs returning at once;
               e2e_sync: the same with runs that copy in, compute and copy
               out before returning
  roofline     the dominant kernel against its bound, with the ncu-measured
               DRAM traffic of a launch
  kernels      per program: time, work-items/s, own-unit rate, roofline
               fraction, scheduler overhead against a monolithic launch
               (Sec. 7.3 overhead metric) and the load balance T_FD/T_LD
  cpu_baseline the CPU oracle on a bounded sample of the same step
--impl reference times the CPU oracle on this config (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

SMALL = False  # --small: reduced sizes for profiler captures (never a bench value)

# the six-product GEMM (FP32-accurate compensated mode) goes beyond config 5's
# three-product row: reported per kernel, not part of the step
EXTRA_PROGRAMS = {"gemm_split6"}

# programs run as a main kernel plus a pass beside it, timed also on their own
MAIN_KERNEL_TIMED = {"binomial": "k_binomial (banded lattice; the greeks pass after it excluded)"}
# ncu-measured DRAM bytes per launch of the dominant kernel (null once the kernel changes)
NCU_TRAFFIC = {
    "binomial": {"bytes_per_launch": 419.584e3 * 64,
                 "source": "profiles/binomial_greeks_16384_options.md (16384 options x 64; reads, the results "
                           "stay in L2 within the capture)"},
}
METRIC = ("work-items/s & % of roofline per kernel; sched overhead vs 1 launch; Δ vs plain")
L2_FLUSH_BYTES = 512 << 20
# the oracle's bounded sample: the same fraction of every program's work-items,
# so that the sample has the step's mix (a few seconds of oracle work on 16 cores)
CPU_SAMPLE = 1.0 / 1024
SMS_NOMINAL = 152
SM_MAX_MHZ = 2070.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), bf16_tflops=d.get("bf16_tflops", 1900.0),
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained", 1700.0),
                    sm_max_mhz=d.get("sm_max_mhz", SM_MAX_MHZ), src="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=SM_MAX_MHZ,
                src="fallback")


# ====================================================================== workloads
class Workload:
    name = ""
    sched = ()
    host_ok = True

    def __init__(self, E, torch, dev):
        self.E, self.torch, self.dev = E, torch, dev

    # builds self.eng (device buffers) and self.mono (monolithic launch)
    def setup(self):
        raise NotImplementedError

    def make_engine(self, sched, params, D=0, C=0, host=False):
        E = self.E
        eng = E.Engine()
        ins, outs = (self.h_in, self.h_out) if host else (self.d_in, self.d_out)
        eng.work_items(self.gws, self.lws).scheduler(sched, params).workers(D, C)
        eng.program(self.program(ins, outs))
        return eng

    def work_items(self):
        return self.gws

    in_step = True  # False: reported per kernel beside the step (not one of the five configurations)

    def tunable(self, name):
        """(fresh-program factory, gws, lws) of a program the autotuner may search, or None."""
        return None

    def host_halves(self):
        """Two host-buffer engines over the two halves of the work, or None."""
        return None

    def programs(self):
        """(name, engine, work-items) of every program the step runs."""
        if isinstance(self.eng, MultiEngine):
            return list(zip(self.eng.names, self.eng.engs, self.eng.wis))
        return [(self.name, self.eng, self.gws)]

    def alg(self, name):
        """Algorithmic work of one program: bound, flops and/or bytes, own unit."""
        return self.after()


class Mandelbrot(Workload):
    name = "mandelbrot"
    sched = ("static", (), 1, 0)  # one package, one device of every resident CTA

    def host_setup(self):
        self.r = W.mandelbrot_region(1024, 1024, 256)
        self.npx = self.r["width"] * self.r["height"]
        self.lws = 256
        self.gws = self.npx // 4
        self.config = dict(size="%dx%d" % (self.r["width"], self.r["height"]), max_iter=self.r["max_iter"],
                           scheduler="static, 1 package")

    def setup(self):
        torch = self.torch
        self.host_setup()
        self.d_in = []
        self.d_out = [torch.zeros(self.npx, dtype=torch.int32, device="cuda")]
        self.h_in = []
        self.h_out = [torch.zeros(self.npx, dtype=torch.int32).pin_memory()]

    def program(self, ins, outs):
        r = self.r
        out = outs[0]
        return self.E.Program("mandelbrot").out(out).args(out, r["width"], r["height"], r["x0"], r["y0"],
                                                          r["dx"], r["dy"], r["max_iter"])

    def after(self):
        # algorithmic work: 8 FP32 instructions per iteration (x^2, y^2, |z|^2, x^2-y^2, +cx, 2x, *y, +cy)
        its = int(self.d_out[0].to(self.torch.int64).sum().item())
        self.iterations = its
        return dict(bound="alu", inst=8.0 * its, flops=8.0 * its, unit_name="pixels/s", units=self.npx)

    def batched_report(self, timed):
        """The image as 16 horizontal strips of uneven height, each its own view
        (the same pixels): 16 plain launches (one grid each, as the step runs
        it) against one "mandelbrot_batch" launch and its CUDA-graph replay."""
        from paper_1805_02755_gb300.batching import MandelbrotBatch, capture_graph, split_uneven
        E, r = self.E, self.r
        out = self.d_out[0]
        Wd = r["width"]
        views, engines, row = [], [], 0
        for h in split_uneven(r["height"], 16, seed=12):
            o = out[row * Wd:(row + h) * Wd]
            y0 = float(np.float32(r["y0"]) + np.float32(row) * np.float32(r["dy"]))
            views.append(dict(out=o, W=Wd, H=h, x0=r["x0"], y0=y0, dx=r["dx"], dy=r["dy"], max_iter=r["max_iter"]))
            eng = E.Engine()
            eng.work_items(-(-(Wd * h) // 4 // 256) * 256, 256).scheduler("static", ()).workers(1, 0)
            eng.program(E.Program("mandelbrot").out(o).args(o, Wd, h, r["x0"], y0, r["dx"], r["dy"], r["max_iter"]))
            engines.append(eng)
            row += h

        def plain():
            for e in engines:
                e.run()
        ms_plain = timed(plain, 20)
        mb = MandelbrotBatch(views, scheduler=("hguided", (2.0, 1.0)), workers=(0, 0))
        ms_batched = timed(mb.run, 20)
        g = capture_graph(mb.engine)
        ms_graph = timed(g.replay, 20)
        for e in engines:
            e.close()
        mb.close()
        return dict(views=len(views), ms_16_launches=ms_plain, ms_one_batched_launch=ms_batched,
                    ms_batched_graph_replay=ms_graph, batched_over_plain=ms_batched / ms_plain,
                    scheduler="batched: hguided k=2, min 1, every resident CTA a device")

    def cpu_sample(self, O, threads, f):
        # k evenly spaced rows, each through the oracle as a one-row image
        r = self.r
        k = max(1, int(round(r["height"] * f)))
        rows = [int((i + 0.5) * r["height"] / k) for i in range(k)]
        t = time.perf_counter()
        for j in rows:
            cy = np.float32(np.float32(r["y0"]) + np.float32(j) * np.float32(r["dy"]))
            O.mandelbrot(r["width"], 1, np.float32(r["x0"]), cy, np.float32(r["dx"]), np.float32(r["dy"]),
                         r["max_iter"], threads=threads)
        return k / r["height"], time.perf_counter() - t, "%d evenly spaced of %d rows" % (k, r["height"])


class Gaussian(Workload):
    name = "gaussian"
    sched = ("dynamic", (256,), 8, 0)  # 256 row packages over 8 devices of CTAs

    def host_setup(self):
        self.H = self.Wd = 6144 if SMALL else 8192
        self.img = W.gaussian_image(self.H, self.Wd)
        self.w = W.gaussian_weights(31, 5.0)
        self.lws = 128
        self.gws = self.H * self.Wd
        self.config = dict(size="8192x8192", taps=31, sigma=5, scheduler="dynamic, 256 packages; devices autotuned")

    def setup(self):
        torch = self.torch
        self.host_setup()
        img = self.img
        self.d_in = [torch.from_numpy(img).cuda(), torch.from_numpy(self.w).cuda()]
        self.d_out = [torch.zeros(self.H * self.Wd, dtype=torch.float32, device="cuda")]
        self.h_in = [torch.from_numpy(img).pin_memory(), torch.from_numpy(self.w).pin_memory()]
        self.h_out = [torch.zeros(self.H * self.Wd, dtype=torch.float32).pin_memory()]

    def program(self, ins, outs):
        x, w = ins
        out = outs[0]
        return self.E.Program("gaussian").in_(x).in_(w).out(out).args(x, w, out, self.Wd, self.H, 31)

    def after(self):
        # algorithmic: 62 FMAs per pixel (31 vertical + 31 horizontal), 8 bytes of HBM per pixel
        npx = self.H * self.Wd
        return dict(bound="alu", inst=62.0 * npx, flops=2.0 * 62 * npx, bytes=8.0 * npx, unit_name="pixels/s",
                    units=npx)

    def batched_report(self, timed):
        """The 8192-column image cut into 16 images of uneven height (each its
        own image with clamped borders): 16 plain "gaussian" launches with the
        step's (tuned) configuration against one "gaussian_batch" launch with
        the same configuration, and its CUDA-graph replay."""
        from paper_1805_02755_gb300 import autotune as AT
        from paper_1805_02755_gb300.batching import GaussianBatch, capture_graph, split_uneven
        E = self.E
        x, w = self.d_in
        x = x.reshape(-1)
        out = self.d_out[0].reshape(-1)
        cfg = getattr(self, "tuned_config", None)
        images, engines, row = [], [], 0
        for h in split_uneven(self.H, 16, seed=13):
            xi, oi = x[row * self.Wd:(row + h) * self.Wd], out[row * self.Wd:(row + h) * self.Wd]
            images.append({"in": xi, "out": oi, "w": w, "W": self.Wd, "H": h})
            eng = E.Engine()
            s, p, D, C = self.sched
            eng.work_items(self.Wd * h, self.lws).scheduler(s, p).workers(D, C)
            if cfg is not None:
                AT.apply(eng, cfg)
            eng.program(E.Program("gaussian").in_(xi).in_(w).out(oi).args(xi, w, oi, self.Wd, h, 31))
            engines.append(eng)
            row += h

        def plain():
            for e in engines:
                e.run()
        ms_plain = timed(plain, 20)
        s, p, D, C = self.sched
        gb = GaussianBatch(images, scheduler=(s, p), workers=(D, C), config=cfg)
        ms_batched = timed(gb.run, 20)
        g = capture_graph(gb.engine)
        ms_graph = timed(g.replay, 20)
        for e in engines:
            e.close()
        gb.close()
        return dict(images=len(images), ms_16_launches=ms_plain, ms_one_batched_launch=ms_batched,
                    ms_batched_graph_replay=ms_graph, batched_over_plain=ms_batched / ms_plain,
                    config=cfg or dict(scheduler=s, params=list(p), devices=D, ctas=C))

    def cpu_sample(self, O, threads, f):
        k = max(1, int(round(self.H * f)))
        t = time.perf_counter()
        O.gaussian(self.img, self.w, rows=(0, k), threads=threads)
        return k / self.H, time.perf_counter() - t, "%d of %d rows" % (k, self.H)


def _single_program_tunable(self, name):
    return (lambda: self.program(self.d_in, self.d_out), self.gws, self.lws) if name == self.name else None


Gaussian.tunable = _single_program_tunable


class NBody(Workload):
    """Config 3: force (HGuided), potential energy (FP64 sums), its adjoint and
    the finite-difference check, four launches over the same 65536 bodies."""
    name = "nbody"
    sched = ("hguided", (2.0, 1.0), 8, 0)
    EPS2 = 1e-3
    NFD = 256

    def host_setup(self):
        self.sms = self.torch.cuda.get_device_properties(0).multi_processor_count if self.torch else 0
        self.n = 16384 if SMALL else 65536
        self.pos, _ = W.nbody_bodies(self.n)
        self.lws = 64
        self.gws = self.n
        rng = W.rng(W.SEED_BASE + 20)
        self.fd_body = rng.choice(self.n, self.NFD, replace=False).astype(np.int32)
        self.fd_comp = rng.integers(0, 3, self.NFD).astype(np.int32)
        self.config = dict(bodies=self.n, eps2=self.EPS2, lws=64,
                           scheduler="hguided (force: k, minimum package and devices autotuned; energy, adjoint: "
                                     "k=2 over 8 devices)",
                           programs="nbody_acc + nbody_energy + nbody_adjoint (HGuided) + nbody_fd (256 samples, "
                                    "h=1e-3, Static one package)")

    def setup(self):
        torch = self.torch
        self.host_setup()
        n = self.n
        pos = torch.from_numpy(self.pos)
        gE = torch.ones(1, dtype=torch.float32)
        fb, fc = torch.from_numpy(self.fd_body), torch.from_numpy(self.fd_comp)
        self.d_in = [pos.cuda(), gE.cuda(), fb.cuda(), fc.cuda()]
        self.d_out = [torch.zeros((n, 4), device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda"),
                      torch.zeros((n, 4), device="cuda"), torch.zeros(self.NFD, dtype=torch.float64, device="cuda")]
        self.h_in = [pos.pin_memory(), gE.pin_memory(), fb.pin_memory(), fc.pin_memory()]
        self.h_out = [torch.zeros((n, 4)).pin_memory(), torch.zeros(1, dtype=torch.float64).pin_memory(),
                      torch.zeros((n, 4)).pin_memory(), torch.zeros(self.NFD, dtype=torch.float64).pin_memory()]

    def make_engine(self, sched, params, D=0, C=0, host=False):
        E = self.E
        ins, outs = (self.h_in, self.h_out) if host else (self.d_in, self.d_out)
        pos, gE, fb, fc = ins
        acc, en, grad, fd = outs
        n = self.n
        progs = [
            (E.Program("nbody_acc").in_(pos).out(acc).args(pos, n, self.EPS2, acc), n, 64),
            (E.Program("nbody_energy").in_(pos).out(en).args(pos, n, self.EPS2, en), n, 64),
            (E.Program("nbody_adjoint").in_(pos).in_(gE).out(grad).args(pos, n, self.EPS2, gE, grad), n, 64),
            # the finite-difference check (256 samples of one work-group each) is one
            # Static package over one device: one grid, every sample resident at once
            (E.Program("nbody_fd").in_(pos).in_(fb).in_(fc).out(fd)
             .args(pos, n, self.EPS2, 1e-3, fb, fc, self.NFD, fd), self.NFD, 1, (1, 0), ("static", ())),
        ]
        return MultiEngine(E, progs, sched, params, D, C)

    def work_items(self):
        return 3 * self.n + self.NFD

    def tunable(self, name):
        if name != "nbody_acc":
            return None
        pos, acc = self.d_in[0], self.d_out[0]
        return (lambda: self.E.Program("nbody_acc").in_(pos).out(acc).args(pos, self.n, self.EPS2, acc), self.n, 64)

    def alg(self, name):
        n = self.n
        # FP32 pipe instructions per pair (flops with FMA = 2 in brackets): force 12 [18]
        # (3 sub, 3 FMA, 3 mul, 3 FMA) + 1 rsqrt; energy 7 [10] over i<j (3 sub, 3 FMA,
        # 1 FMA) + 1 rsqrt, which makes it bound by the 16/clk rsqrt unit; adjoint 13 [19];
        # finite differences: FP64-bound, 2 FP64 instructions per j for each sample
        # (the FP32 term difference converted, then added)
        if name == "nbody_acc":
            return dict(bound="alu", inst=12.0 * n * n, flops=18.0 * n * n, unit_name="interactions/s", units=n * n)
        if name == "nbody_energy":
            pairs = n * (n - 1) / 2
            return dict(bound="mufu", inst=pairs, flops=10.0 * pairs, unit_name="pairs/s", units=int(pairs))
        if name == "nbody_adjoint":
            return dict(bound="alu", inst=13.0 * n * n, flops=19.0 * n * n, unit_name="interactions/s", units=n * n)
        return dict(bound="fp64", inst=2.0 * n * self.NFD, flops=18.0 * n * self.NFD, unit_name="samples/s",
                    units=self.NFD)

    def cpu_sample(self, O, threads, f):
        n = self.n
        nb, nfd = max(1, int(round(n * f))), max(1, int(round(self.NFD * f)))
        m = max(1, int(round(n * f / 2)))  # energy rows 0..m-1: about f of the i<j pairs
        t = time.perf_counter()
        O.nbody_acc(self.pos, self.EPS2, bodies=(0, nb), threads=threads)
        O.nbody_energy_grad(self.pos, self.EPS2, bodies=(0, nb), threads=threads)
        O.nbody_potential(self.pos, self.EPS2, bodies=(0, nb), threads=threads)
        O.nbody_energy(self.pos, self.EPS2, threads=threads, rows=(0, m))
        O.nbody_fd_energy_grad(self.pos, self.EPS2, self.fd_body[:nfd], self.fd_comp[:nfd], 1e-3)
        secs = time.perf_counter() - t
        # work-items sampled: force and adjoint rows nb each; the energy's rows
        # [0, nb) hold their share of the n(n-1)/2 pair terms of its n work-items;
        # nfd of the finite-difference samples
        pairs = m * (n - 1) - m * (m - 1) // 2
        wi = 2 * nb + n * pairs / (n * (n - 1) / 2) + nfd
        return wi / self.work_items(), secs, (
            "rows 0..%d of %d of the force and adjoint, rows 0..%d of the energy (i<j), %d of %d "
            "finite-difference samples" % (nb - 1, n, m - 1, nfd, self.NFD))


class Binomial(Workload):
    """Config 4: 2^20 European options of depth U{256..2048}, price + delta + vega in one launch."""
    name = "binomial"
    sched = ("hguided", (2.0, 1.0), 8, 0)

    def host_setup(self):
        self.n = (1 << 14) if SMALL else (1 << 20)
        self.o = W.binomial_options(self.n)
        self.lws = 32
        self.gws = self.n * 32
        st = self.o["steps"].astype(np.int64)
        self.nodes = int((st * (st + 1) // 2).sum())
        self.nodes_price, self.greeks_terms = banded_node_updates(self.o)
        self.config = dict(options=self.n, steps="U{256..2048}", scheduler="hguided k=2 over 8 devices",
                           outputs="price + delta + vega", node_updates_full_lattice=self.nodes,
                           node_updates_nonzero_band=self.nodes_price, greeks_leaf_terms=self.greeks_terms)

    def setup(self):
        torch = self.torch
        self.host_setup()
        o = self.o
        ts = [torch.from_numpy(np.ascontiguousarray(o[k])) for k in ("S", "K", "T", "sigma", "steps")]
        self.d_in = [t.cuda() for t in ts]
        self.d_out = [torch.zeros(self.n, device="cuda"), torch.zeros((self.n, 2), device="cuda")]
        self.h_in = [t.pin_memory() for t in ts]
        self.h_out = [torch.zeros(self.n).pin_memory(), torch.zeros((self.n, 2)).pin_memory()]

    def program(self, ins, outs, greeks=True):
        S, K, T, sig, st = ins
        price, gr = outs
        p = self.E.Program("binomial")
        for t in ins:
            p.in_(t)
        p.out(price)
        if greeks:
            p.out(gr)
        return p.args(S, K, T, sig, st, self.o["r"], self.n, price, gr if greeks else None)

    def plain_engine(self):
        E = self.E
        eng = E.Engine()
        s, prm, D, C = self.sched
        eng.work_items(self.gws, self.lws).scheduler(s, prm).workers(D, C)
        eng.program(self.program(self.d_in, self.d_out, greeks=False))
        return eng

    def host_halves(self):
        """Host-buffer engines over options [0, n/2) and [n/2, n) (views of the
        pinned buffers), so that another stage's copies can run during each."""
        E = self.E
        s, prm, D, C = self.sched
        engs = []
        for lo, hi in ((0, self.n // 2), (self.n // 2, self.n)):
            ins = [t[lo:hi] for t in self.h_in]
            price, gr = self.h_out[0][lo:hi], self.h_out[1][lo:hi]
            p = E.Program("binomial")
            for t in ins:
                p.in_(t)
            p.out(price).out(gr)
            p.args(*ins, self.o["r"], hi - lo, price, gr)
            eng = E.Engine()
            eng.work_items((hi - lo) * 32, 32).scheduler(s, prm).workers(D, C).program(p)
            engs.append(eng)
        return engs

    def batched_report(self, timed):
        """The same options as 64 batches of uneven size: 64 launches (plain)
        against one batched launch, and that launch replayed from a CUDA graph."""
        from paper_1805_02755_gb300.batching import BinomialBatch, capture_graph, split_uneven
        E = self.E
        S, K, T, sig, st = self.d_in
        price, gr = self.d_out
        sizes = split_uneven(self.n, 64, seed=11)
        batches, engines = [], []
        o = 0
        sch, prm, D, C = self.sched
        for n in sizes:
            sl = slice(o, o + n)
            b = dict(S=S[sl], K=K[sl], T=T[sl], sigma=sig[sl], steps=st[sl], r=self.o["r"], price=price[sl],
                      greeks=gr[sl])
            batches.append(b)
            eng = E.Engine()
            p = E.Program("binomial")
            for t in (b["S"], b["K"], b["T"], b["sigma"], b["steps"]):
                p.in_(t)
            p.out(b["price"]).out(b["greeks"])
            p.args(b["S"], b["K"], b["T"], b["sigma"], b["steps"], self.o["r"], n, b["price"], b["greeks"])
            eng.work_items(n * 32, 32).scheduler(sch, prm).workers(D, C).program(p)
            engines.append(eng)
            o += n

        def plain():
            for e in engines:
                e.run()
        ms_plain = timed(plain, 2)
        bb = BinomialBatch(batches, with_greeks=True, scheduler=(sch, prm), workers=(D, C))
        ms_batched = timed(bb.run, 2)
        g = capture_graph(bb.engine)
        ms_graph = timed(g.replay, 2)
        for e in engines:
            e.close()
        bb.close()
        return dict(batches=len(sizes), largest=max(sizes), smallest=min(sizes), ms_64_launches=ms_plain,
                    ms_one_batched_launch=ms_batched, ms_batched_graph_replay=ms_graph,
                    batched_over_plain=ms_batched / ms_plain)

    def after(self):
        # FP32 instructions per node update of the backward induction: 2 (add,
        # FMA; flops with FMA = 2: 3), over the nodes that can be nonzero
        # (its band).  Delta and the vega leaf part are sums over the nonzero
        # leaves with closed-form adjoint weights, O(b) per option, not counted
        # (conservative).  The full lattice's node count is reported beside it.
        nb = self.nodes_price
        return dict(bound="alu", inst=2.0 * nb, flops=3.0 * nb, unit_name="options/s",
                    units=self.n, extra={"node_updates_per_s": nb,
                                         "full_lattice_node_updates_per_s": self.nodes,
                                         "greeks_leaf_terms_per_s": self.greeks_terms})

    def cpu_sample(self, O, threads, f):
        t = time.perf_counter()
        k = max(1, int(round(self.n * f)))
        o = self.o
        O.binomial(o["S"][:k], o["K"][:k], o["T"][:k], o["sigma"][:k], o["steps"][:k], o["r"], threads=threads)
        return k / self.n, time.perf_counter() - t, "%d of %d options (price, delta, vega)" % (k, self.n)


def banded_node_updates(o):
    """Node updates of the binomial kernel's backward induction over its
    nonzero band, and the leaf terms of its closed-form greeks.

    The out-of-the-money side is priced; its nonzero leaves form a run of b
    leaves (FP64 estimate of the FP32 payoff test).  The backward induction
    updates min(t + 1, b) nodes to produce level t (t = N-1 .. 0); delta and
    vega sum b weighted leaf terms.
    """
    S, K, T, sig = (o[k].astype(np.float64) for k in ("S", "K", "T", "sigma"))
    N = o["steps"].astype(np.int64)
    a = sig * np.sqrt(T / N)
    x = (N + np.log(K / S) / a) / 2.0           # leaf j is in the money for 2j - N vs ln(K/S)/a
    put = S > K
    b_put = np.clip(np.ceil(x), 0, N + 1)       # j < x
    b_call = np.clip(N - np.floor(x), 0, N + 1)  # j > x
    b = np.maximum(np.where(put, b_put, b_call), 1).astype(np.int64)
    bb = np.minimum(b, N)
    p0 = bb * (bb + 1) // 2 + (N - bb) * bb
    return int(p0.sum()), int(np.minimum(b, N + 1).sum())


class Gemm(Workload):
    """Config 5: M = N = K = 8192, HGuided packages of 128-row tiles over 4
    devices; the plain BF16 product and the compensated split-BF16 modes
    (three products; six products with FP32 promotion)."""
    name = "gemm"
    sched = ("hguided", (2.0, 1.0), 4, 0)
    M = N = K = 8192

    def host_setup(self):
        if SMALL:
            self.M = self.N = self.K = 4096
        self.A, self.Bt = W.gemm_matrices(self.M, self.N, self.K)
        self.lws = 128 * 256
        self.tiles = (self.M // 128) * (self.N // 256)
        self.gws = self.tiles * self.lws
        self.lws6 = 128 * 128
        self.gws6 = (self.M // 128) * (self.N // 128) * self.lws6
        self.config = dict(M=self.M, N=self.N, K=self.K, tile="128x256x64 work-groups, computed in vertical pairs",
                           scheduler="hguided, packages of 128-row tiles (pairs of tile rows); k, minimum package and "
                                     "devices autotuned for gemm_bf16 and gemm_split3 (k=2 over 4 devices otherwise)",
                           programs="gemm_bf16 (bf16 inputs) + gemm_split3 (fp32 inputs, 3 products) + "
                                    "gemm_split6 (fp32 inputs, 6 products, FP32 promotion every 64 of K, 128x128 tiles)")

    def setup(self):
        torch = self.torch
        E = self.E
        self.host_setup()
        A, Bt = torch.from_numpy(self.A), torch.from_numpy(self.Bt)
        dA, dB = A.cuda(), Bt.cuda()
        ab = torch.empty(self.A.shape, dtype=torch.bfloat16, device="cuda")
        bb = torch.empty(self.Bt.shape, dtype=torch.bfloat16, device="cuda")
        for src, dst in ((dA, ab), (dB, bb)):  # the input cast, in the library's kernel
            ce = E.Engine()
            pr = E.Program("cast_bf16").in_(src).out(dst).args(src, dst, src.numel())
            ce.work_items(src.numel(), 256).scheduler("dynamic", (256,)).program(pr).run().synchronize()
            ce.close()
        self.d_in = [ab, bb, dA, dB]
        self.d_out = [torch.zeros(self.M * self.N, device="cuda") for _ in range(3)]
        self.h_in = [ab.cpu().pin_memory(), bb.cpu().pin_memory(), A.pin_memory(), Bt.pin_memory()]
        self.h_out = [torch.zeros(self.M * self.N).pin_memory() for _ in range(2)]  # the step's programs
        del dA, dB

    def make_engine(self, sched, params, D=0, C=0, host=False):
        E = self.E
        ins, outs = (self.h_in, self.h_out) if host else (self.d_in, self.d_out)
        ab, bb, af, bf = ins
        c1, c2 = outs[:2]
        progs = [
            (E.Program("gemm_bf16").in_(ab).in_(bb).out(c1).args(ab, bb, c1, self.M, self.N, self.K),
             self.gws, self.lws),
            (E.Program("gemm_split3").in_(af).in_(bf).out(c2).args(af, bf, c2, self.M, self.N, self.K),
             self.gws, self.lws),
        ]
        if not host:  # the six-product mode is reported beside the step, not timed end to end
            c3 = outs[2]
            progs.append((E.Program("gemm_split6").in_(af).in_(bf).out(c3).args(af, bf, c3, self.M, self.N, self.K, 1),
                          self.gws6, self.lws6))
        return MultiEngine(E, progs, sched, params, D, C)

    def work_items(self):
        return 2 * self.M * self.N

    def tunable(self, name):
        # the step's two products: HGuided's devices, k and minimum package are searched
        if name not in ("gemm_bf16", "gemm_split3"):
            return None
        ab, bb, af, bf = self.d_in
        c = self.d_out[0] if name == "gemm_bf16" else self.d_out[1]
        a, b = (ab, bb) if name == "gemm_bf16" else (af, bf)
        return (lambda: self.E.Program(name).in_(a).in_(b).out(c).args(a, b, c, self.M, self.N, self.K),
                self.gws, self.lws)

    def alg(self, name):
        f = 2.0 * self.M * self.N * self.K
        if name == "gemm_bf16":
            return dict(bound="tensor", flops=f, unit_name="TFLOP/s", units=f / 1e12)
        # three (six) products on the tensor cores (+ the split pass); "effective" counts the plain product
        nprod = 6.0 if name == "gemm_split6" else 3.0
        return dict(bound="tensor", flops=nprod * f, unit_name="effective TFLOP/s", units=f / 1e12)

    def cpu_sample(self, O, threads, f):
        rng = W.rng(5)
        ne = max(1, int(round(self.M * self.N * f)))
        ii = rng.integers(0, self.M, ne)
        jj = rng.integers(0, self.N, ne)
        t = time.perf_counter()
        for mode in (0, 2):  # the step's plain and three-product values
            O.gemm_entries(self.A, self.Bt, mode, ii, jj, threads=threads)
        return ne / (self.M * self.N), time.perf_counter() - t, "%d of %d entries, both modes" % (
            ne, self.M * self.N)


class MultiEngine:
    """Several programs of one configuration, each on its own engine, run in order."""

    def __init__(self, E, progs, sched, params, D, C):
        self.engs = []
        self.names = [pr[0].kernel for pr in progs]
        self.wis = [pr[1] for pr in progs]
        for pr in progs:
            prog, gws, lws = pr[:3]
            d, c = pr[3] if len(pr) > 3 else (D, C)  # a program may name its own workers
            s, p = pr[4] if len(pr) > 4 and sched != "monolithic" else (sched, params)  # ... and scheduler
            e = E.Engine()
            e.work_items(gws, lws).scheduler(s, p).workers(d, c)
            e.program(prog)
            self.engs.append(e)

    def run(self):
        for e in self.engs:
            e.run()
        return self

    def stats(self):
        return self.engs[0].stats()

    def worker_stats(self):
        return self.engs[0].worker_stats()

    def plan_info(self):
        return self.engs[0].plan_info()

    def close(self):
        for e in self.engs:
            e.close()

    @property
    def launches(self):
        return len(self.engs)


class Ray(Workload):
    """The paper's fifth benchmark (Sec. 7 "Ray"), not one of the five measured
    configurations: a Whitted tracer over a seeded 64-sphere, 3-light scene at
    2048 x 2048, HGuided over one device of one-warp CTAs; reported beside the step."""
    name = "ray"
    sched = ("hguided", (2.0, 1.0), 1, 0)
    in_step = False

    def host_setup(self):
        self.sc = W.ray_scene()
        self.Wd = self.Hd = 1024 if SMALL else 2048
        self.lws = 128
        self.gws = self.Wd * self.Hd
        self.config = dict(size="%dx%d" % (self.Wd, self.Hd), spheres=self.sc["nspheres"], lights=self.sc["nlights"],
                           max_depth=self.sc["max_depth"], scheduler="hguided k=2, one device")

    def setup(self):
        torch = self.torch
        self.host_setup()
        s = torch.from_numpy(self.sc["scene"])
        self.d_in = [s.cuda()]
        self.d_out = [torch.zeros((self.gws, 4), device="cuda")]
        self.h_in = [s.pin_memory()]
        self.h_out = [torch.zeros((self.gws, 4)).pin_memory()]

    def program(self, ins, outs):
        sc = self.sc
        return self.E.Program("ray").in_(ins[0]).out(outs[0]).args(
            ins[0], sc["nspheres"], sc["nlights"], self.Wd, self.Hd, sc["ka"], *sc["bg"], sc["max_depth"], outs[0])

    def after(self):
        # every ray (camera, reflected, shadow) is tested against every sphere:
        # 16 FP32 instructions per test (3 sub, 5 for o.d, 5 for |o|^2, 1 sub, 2 for the discriminant)
        rays = float(self.d_out[0][:, 3].double().sum().item())
        tests = rays * self.sc["nspheres"]
        return dict(bound="alu", inst=16.0 * tests, flops=16.0 * tests, unit_name="pixels/s", units=self.gws,
                    extra={"rays_per_s": rays, "ray_sphere_tests_per_s": tests})

    def cpu_sample(self, O, threads, f):
        sc = self.sc
        rows = max(2, 2 * int(round(self.Hd * f / 2)))
        t = time.perf_counter()
        O.ray(sc["scene"], sc["nspheres"], sc["nlights"], self.Wd, self.Hd, sc["ka"], sc["bg"], sc["max_depth"],
              rows=(self.Hd // 2 - rows // 2, self.Hd // 2 + rows // 2), threads=threads)
        return rows / self.Hd, time.perf_counter() - t, "%d of %d rows" % (rows, self.Hd)


Ray.tunable = _single_program_tunable


class MandelbrotLarge(Mandelbrot):
    """Config 1 scaled up, a secondary labelled row beside the step: 8192 x 8192
    pixels over the same view, up to 1024 iterations, Static one package (the
    1024 x 1024 case is too small to fill the GPU)."""
    name = "mandelbrot_8192"
    in_step = False

    def host_setup(self):
        n = 2048 if SMALL else 8192
        self.r = W.mandelbrot_region(n, n, 1024)
        self.npx = self.r["width"] * self.r["height"]
        self.lws = 256
        self.gws = self.npx // 4
        self.config = dict(size="%dx%d" % (n, n), max_iter=1024, scheduler="static, 1 package")


WORKLOADS = [Mandelbrot, Gaussian, NBody, Binomial, Gemm, Ray, MandelbrotLarge]


# ====================================================================== helpers
class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


def balance_of(stats):
    """Sec. 7.3 balance T_FD / T_LD over devices (time from the first package start)."""
    if len(stats) == 0:
        return None
    t0 = int(stats["t0_ns"].min())
    fin = {}
    for d, t1 in zip(stats["device"], stats["t1_ns"]):
        fin[int(d)] = max(fin.get(int(d), 0), int(t1) - t0)
    f = list(fin.values())
    return (min(f) / max(f)) if len(f) > 1 and max(f) > 0 else 1.0


def worker_efficiency(ws, info):
    """Mean over max busy time of the persistent CTAs; None for Static over one
    device, which runs as a grid of one-chunk CTAs (no persistent workers)."""
    if info["devices"] == 1 and info["ctas_per_device"] == info["ctas"] and len(ws) and (ws["chunks"] == 1).all():
        return None
    busy = ws["busy_ns"].astype(np.float64)
    return float(busy.mean() / busy.max()) if len(busy) and busy.max() > 0 else None


# ====================================================================== arms
def run_ours(args):
    import torch

    import paper_1805_02755_gb300 as E
    from paper_1805_02755_gb300 import build as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count

    names = args.only.split(",") if args.only else None
    wls = [cls(E, torch, local) for cls in WORKLOADS if names is None or cls.name in names]
    if not any(w.in_step for w in wls):  # only workloads from beside the step were asked for: time them as one
        for w in wls:
            w.in_step = True
    tuned = {}
    for w in wls:
        w.setup()
        s, p, D, C = w.sched
        w.eng = w.make_engine(s, p, D, C)
        w.mono = w.make_engine("monolithic", ())
        w.host = w.make_engine(s, p, D, C, host=True)
        if not args.no_autotune:
            # the autotuner's pick (searched once per problem shape, then cached)
            # drives the timed runs of every tunable program
            for name, eng, _ in w.programs():
                if w.tunable(name) is not None:
                    tuned[name] = autotune_report(w, name)
                    apply_tuned(w, name, tuned[name]["best"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    allprogs = [(w, name, eng, wi) for w in wls for (name, eng, wi) in w.programs()]
    # programs beyond the configurations' hot path (precision variants) are timed on
    # their own and reported per kernel, outside the step and its work-item count
    progs = [pr for pr in allprogs if pr[1] not in EXTRA_PROGRAMS and pr[0].in_step]

    # programs whose main kernel has a pass beside it inside one run (the
    # binomial's greeks pass): the main kernel is also timed on its own, by
    # events the library records around it on the engine's stream
    main_timed = [i for i, (_, name, eng, _) in enumerate(progs) if name in MAIN_KERNEL_TIMED
                  and hasattr(eng, "kernel_events")]

    def step(record):
        flush.fill_(1.0)  # evict L2 (outside the timed events)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(progs) + 1)]
        kev = {i: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for i in main_timed}
        for i, (b0, b1) in kev.items():
            # recorded here first so that torch reads them; the library's records around
            # the main kernel come later on the same stream and replace these
            b0.record(stream)
            b1.record(stream)
            progs[i][2].kernel_events(b0, b1)
        ev[0].record(stream)
        for i, (_, _, eng, _) in enumerate(progs):
            eng.run()
            ev[i + 1].record(stream)
        record.append((ev, kev))

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    recs = []
    for _ in range(args.steps):
        step(recs)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per = {name: [] for _, name, _, _ in progs}
    per_main = {progs[i][1]: [] for i in main_timed}
    tot = []
    for ev, kev in recs:
        tot.append(ev[0].elapsed_time(ev[-1]))
        for i, (_, name, _, _) in enumerate(progs):
            per[name].append(ev[i].elapsed_time(ev[i + 1]))
        for i, (b0, b1) in kev.items():
            per_main[progs[i][1]].append(b0.elapsed_time(b1))
    for i in main_timed:
        progs[i][2].kernel_events(None, None)
    step_ms = max_over_ranks(sum(tot) / len(tot), world)
    launches = sum(2 if name in ("gemm_split3", "gemm_split6", "binomial") else 1 for _, name, _, _ in progs)  # split + main; lattice + greeks

    def quantiles(ts):
        q = sorted(ts)
        at = lambda f: q[min(len(q) - 1, int(round(f * (len(q) - 1))))]  # noqa: E731
        return dict(p10=at(0.1), median=statistics.median(q), p90=at(0.9), n=len(q))

    # scheduler overhead against the monolithic launch (same kernel body, no queue)
    def timed(fn, n, samples=None):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(n):
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        if samples is not None:
            samples.extend(ts)
        return statistics.median(ts)

    kern = {}
    dominant = None
    monos = {}
    for w in wls:
        for name, eng, _ in (zip(w.mono.names, w.mono.engs, w.mono.wis) if isinstance(w.mono, MultiEngine)
                             else [(w.name, w.mono, 0)]):
            monos[name] = eng
    for w, name, eng, wi in allprogs:
        extra = name in EXTRA_PROGRAMS or not w.in_step
        mono_ts, sched_ts = [], []
        ms_mono = timed(monos[name].run, max(5, min(args.steps, 10)), mono_ts)
        ms_sched = timed(eng.run, max(5, min(args.steps, 10)), sched_ts)
        sets = None
        if max(ms_mono, ms_sched) < 5.0:
            # short kernels: two sets of 50 runs per form, alternating forms
            sets = []
            for _ in range(2):
                m_ts, s_ts = [], []
                timed(monos[name].run, 50, m_ts)
                timed(eng.run, 50, s_ts)
                sets.append(dict(ms_monolithic=statistics.median(m_ts), ms_scheduled=statistics.median(s_ts)))
                mono_ts += m_ts
                sched_ts += s_ts
            ms_mono = statistics.median(mono_ts)
            ms_sched = statistics.median(sched_ts)
        ms = ms_sched if extra else statistics.median(per[name])
        alg = w.alg(name)
        st = eng.stats()
        wst = eng.worker_stats()
        info = eng.plan_info()
        d = dict(ms=ms, work_items=wi, work_items_per_s=wi / (ms * 1e-3),
                 overhead_vs_monolithic_pct=100.0 * (ms_sched - ms_mono) / ms_mono,
                 ms_monolithic=ms_mono, ms_scheduled_isolated=ms_sched, plan=info,
                 balance_T_FD_over_T_LD=balance_of(st), cta_busy_efficiency=worker_efficiency(wst, info),
                 packages=len(st), ms_quantiles=quantiles(sched_ts if extra else per[name]),
                 ms_monolithic_quantiles=quantiles(mono_ts), overhead_sets=sets)
        d[alg["unit_name"]] = alg["units"] / (ms * 1e-3)
        for k2, v2 in alg.get("extra", {}).items():
            d[k2] = v2 / (ms * 1e-3)
        if hasattr(w, "batched_report") and not args.no_batched:
            d["batched"] = w.batched_report(timed)
        if name in tuned:
            d["autotuned"] = dict(tuned[name], applied_to_the_timed_runs=True)
        if hasattr(w, "plain_engine"):  # the plain form beside the adjoint form
            pe = w.plain_engine()
            ms_plain = timed(pe.run, max(3, min(args.steps, 5)))
            d["plain_ms"] = ms_plain
            d["adjoint_over_plain"] = ms / ms_plain
            pe.close()
        if name in per_main:
            # the main kernel alone (same step, same launch), the algorithmic work being
            # the main kernel's: the roofline of the dominant kernel uses this duration
            ms_main = statistics.median(per_main[name])
            d["ms_main_kernel"] = ms_main
            d["ms_main_kernel_quantiles"] = quantiles(per_main[name])
            if alg["bound"] in ("alu", "mufu", "fp64"):
                lanes = {"alu": 128, "mufu": 16, "fp64": 2}[alg["bound"]]
                peak = sms * lanes * peaks["sm_max_mhz"] * 1e6 / 1e12
                ach = alg["inst"] / (ms_main * 1e-3) / 1e12
                unit = {"alu": "T FP32-inst/s", "mufu": "T rsqrt/s", "fp64": "T FP64-inst/s"}[alg["bound"]]
                d["roofline_main_kernel"] = dict(bound=alg["bound"], achieved=ach, peak=peak, unit=unit,
                                                 frac=ach / peak, kernel=MAIN_KERNEL_TIMED[name])
        if alg["bound"] in ("alu", "mufu", "fp64"):
            # FP32 pipe: 128 lanes per SM; rsqrt unit: 16 per SM; FP64: 2 instructions per SM
            # (the nominal 1.25 TFLOP/s of FMA); per clock at the max SM clock
            lanes = {"alu": 128, "mufu": 16, "fp64": 2}[alg["bound"]]
            peak = sms * lanes * peaks["sm_max_mhz"] * 1e6 / 1e12
            ach = alg["inst"] / (ms * 1e-3) / 1e12
            unit = {"alu": "T FP32-inst/s", "mufu": "T rsqrt/s", "fp64": "T FP64-inst/s"}[alg["bound"]]
            d["roofline"] = dict(bound=alg["bound"], achieved=ach, peak=peak, unit=unit, frac=ach / peak)
            d["fp32_tflops"] = alg["flops"] / (ms * 1e-3) / 1e12
            if "bytes" in alg:
                gbs = alg["bytes"] / (ms * 1e-3) / 1e9
                d["hbm"] = dict(achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s", frac=gbs / peaks["hbm_gbs"])
        elif alg["bound"] == "hbm":
            ach = alg["bytes"] / (ms * 1e-3) / 1e9
            d["roofline"] = dict(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                                 frac=ach / peaks["hbm_gbs"])
        else:
            ach = alg["flops"] / (ms * 1e-3) / 1e12
            pk = peaks["bf16_tflops"]
            d["roofline"] = dict(bound="tensor", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk)
        d["in_step"] = not extra
        kern[name] = d
        if not extra and (dominant is None or ms > kern[dominant]["ms"]):
            dominant = name
    if "gemm_bf16" in kern and "gemm_split3" in kern:
        kern["gemm_split3"]["compensated_over_plain"] = kern["gemm_split3"]["ms"] / kern["gemm_bf16"]["ms"]
    if "gemm_bf16" in kern and "gemm_split6" in kern:
        kern["gemm_split6"]["compensated_over_plain"] = kern["gemm_split6"]["ms"] / kern["gemm_bf16"]["ms"]

    # End to end from pinned host memory, every step: the inputs copied in, the
    # programs run, the results copied out, all through the C ABI with host
    # buffers registered in the programs.  Measured two ways: (1) "e2e": every
    # engine's copies on two copy streams (ecl_engine_copy_streams), ordered
    # around its launch by events, each run returning at once; the copies of
    # one configuration overlap another's computation and the step ends when
    # every result is in host memory; (2) "e2e_sync": each run copies in,
    # computes and copies out before it returns (the synchronous run of
    # Listing 1).
    swls = [w for w in wls if w.in_step]
    h2d = sum(t.numel() * t.element_size() for w in swls for t in w.h_in)
    d2h = sum(t.numel() * t.element_size() for w in swls for t in w.h_out)
    # stage order: the longest computation first (the other stages' inputs move
    # while it runs), then by output size, largest first (their results move
    # while the shorter stages compute)
    def dev_ms(w):
        return sum(kern[n]["ms"] for n, _, _ in w.programs() if n in kern)

    def out_bytes(w):
        return sum(t.numel() * t.element_size() for t in w.h_out)

    def engines_of(x):
        return x.engs if isinstance(x, MultiEngine) else [x]

    first = max(swls, key=dev_ms)
    rest = sorted((w for w in swls if w is not first), key=out_bytes, reverse=True)
    order = [first] + rest
    # the asynchronous pass: the longest stage's batch as two halves when it can
    # be split, the stages with large results between them, so that those
    # results move to the host while the second half computes (one copy stream
    # each way is first-in first-out: a result queued behind the longest
    # stage's would wait for it)
    halves = first.host_halves()
    big_out = [w for w in rest if out_bytes(w) >= (64 << 20)]
    if halves is not None:
        stages = ([("%s[0:n/2]" % first.name, [halves[0]])] + [(w.name, engines_of(w.host)) for w in big_out] +
                  [("%s[n/2:n]" % first.name, [halves[1]])] +
                  [(w.name, engines_of(w.host)) for w in rest if w not in big_out])
    else:
        stages = [(w.name, engines_of(w.host)) for w in order]
    for _ in range(max(1, args.warmup)):
        for w in swls:
            w.host.run()
    torch.cuda.synchronize()
    # the host link as the synchronous pass finds it: one pinned copy of the
    # largest input, device-timed
    big = max((t for w in swls for t in w.h_in), key=lambda t: t.numel() * t.element_size(), default=None)
    link_gbs = None
    if big is not None and big.numel() * big.element_size() >= (1 << 20):
        dbig = torch.empty_like(big, device="cuda")
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        dbig.copy_(big, non_blocking=True)
        eb.record(stream)
        eb.synchronize()
        link_gbs = big.numel() * big.element_size() / (ea.elapsed_time(eb) * 1e6)
        del dbig
    t0 = time.perf_counter()
    per_cfg = {w.name: 0.0 for w in swls}
    per_cfg_dev = {w.name: 0.0 for w in swls}
    for _ in range(args.steps):
        for w in swls:
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tw = time.perf_counter()
            ea.record(stream)
            w.host.run()  # synchronous: returns with the outputs in host memory
            eb.record(stream)
            per_cfg[w.name] += time.perf_counter() - tw
            eb.synchronize()
            per_cfg_dev[w.name] += ea.elapsed_time(eb) * 1e-3
    e2e_sync_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)

    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    for _, es in stages:
        for e in es:
            e.copy_streams(copy_in, copy_out, asynchronous=True)

    def e2e_step():
        for _, es in stages:
            for e in es:
                e.run()  # enqueues copies in, the launch and copies out; returns at once
        for _, es in stages:
            for e in es:
                e.synchronize()  # this step's results are in host memory

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)

    total_wi = sum(wi for _, _, _, wi in progs)
    value = job_rate(total_wi, world, step_ms * 1e-3)
    if "roofline_main_kernel" in kern[dominant]:
        # the dominant kernel's own launches, timed by events around it inside the timed
        # steps; its program's run (with the pass beside it) is kern[dominant]["roofline"]
        rf = dict(kern[dominant]["roofline_main_kernel"])
        rf["ms_per_launch"] = kern[dominant]["ms_main_kernel"]
        rf["timed"] = ("CUDA events recorded by the library right before and after the kernel on the "
                       "engine's stream in every timed step (ecl_engine_kernel_events)")
        rf["program"] = dominant
    else:
        rf = dict(kern[dominant]["roofline"])
        rf["kernel"] = dominant
    # DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
    # committed ncu summary of the current kernel; small-case captures are scaled to a
    # full launch by the units processed (the traffic is per option)
    t = NCU_TRAFFIC.get(dominant)
    rf["traffic"] = None if (t is None or SMALL) else t["bytes_per_launch"]
    if t is not None and not SMALL:
        rf["traffic_source"] = t["source"]
    probe = fp32_probe(E, torch, sms, clk.get("sm_mhz") or peaks["sm_max_mhz"])
    rf["peak_source"] = peaks["src"] if rf["bound"] not in ("alu", "mufu") else \
        "derived: %d SMs x %d lanes x %.0f MHz (max SM clock); the fp32_probe program measured %.1f FFMA/clk/SM " \
        "at %.0f MHz in this run" % (sms, 128 if rf["bound"] == "alu" else 16, peaks["sm_max_mhz"],
                                     probe["ffma_per_clk_per_sm"], probe["at_sm_mhz"])
    out = {
        "metric": METRIC, "value": value, "unit": "work-items/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "ms_per_step_quantiles": quantiles(tot),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, shaped like the paper's workloads)",
        "config": step_config(wls),
        "e2e": {"value": job_rate(total_wi, world, e2e_s), "unit": "work-items/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                "how": "C ABI, host buffers: ecl_engine_copy_streams (copies on two copy streams, "
                       "event-ordered around each launch, asynchronous runs); the longest stage's batch as two "
                       "halves with the large-result stages between them; one synchronize per engine ends "
                       "each step", "stage_order": [n for n, _ in stages]},
        "e2e_sync": {"value": job_rate(total_wi, world, e2e_sync_s), "unit": "work-items/s",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_sync_s * 1e3,
                     "how": "C ABI, host buffers: each run copies in, computes, copies out, then returns",
                     "ms_per_config": {k: v * 1e3 / args.steps for k, v in per_cfg.items()},
                     "device_ms_per_config": {k: v * 1e3 / args.steps for k, v in per_cfg_dev.items()},
                     "h2d_gbs_largest_input": link_gbs},
        "gpu_launches": launches * args.steps,
        "fp32_probe": probe,
        "roofline": rf,
        "clocks": clk,
        "kernels": kern,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(swls, total_wi, args)
    if rank == 0:
        print(json.dumps(out))
    for w in wls:
        w.eng.close()
        w.mono.close()
        w.host.close()
    for e in halves or []:
        e.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def apply_tuned(w, name, config):
    """Applies a tuned configuration to the step's device and host engines of one program."""
    from paper_1805_02755_gb300 import autotune as AT
    for eng in (w.eng, w.host):
        if isinstance(eng, MultiEngine):
            AT.apply(eng.engs[eng.names.index(name)], config)
        else:
            AT.apply(eng, config)
    w.tuned_config = config


def autotune_report(w, name):
    """The autotuner's search over devices, CTAs, HGuided k / minimum package and
    Dynamic package counts for one program, next to the bench's own configuration
    timed the same way (CUDA events, median of 3 after one warm-up run)."""
    from paper_1805_02755_gb300 import autotune as AT
    make, gws, lws = w.tunable(name)
    s, p, D, C = w.sched
    default = dict(scheduler=s, params=list(p), devices=D, ctas=C)
    # the configuration fixes the scheduler (and Dynamic's package count):
    # the search varies what it leaves free (devices, CTAs per device, and
    # HGuided's k and minimum package)
    space = [c for c in AT.default_space(name, gws // lws) if c["scheduler"] == s and
             (s != "dynamic" or list(c["params"]) == list(p))]
    if default not in space:
        space.append(default)
    res = AT.autotune(name, make, gws, lws, space=space, reps=3, warmup=1)
    ms_default = next(ms for cfg, ms in res["table"] if cfg == default)
    return dict(best=res["config"], ms_best=res["ms"], bench_config=default, ms_bench_config=ms_default,
                candidates=len(res["table"]))


def fp32_probe(E, torch, sms, sm_mhz, reps=10):
    """FFMA throughput of the FP32 pipe, measured with the library's fp32_probe
    program (independent FFMA chains, four waves of every CTA slot) through the
    monolithic launch: the measured side of the FP32 rooflines."""
    lws, iters = 256, 512
    G = sms * 8 * 4
    out = torch.empty(G * lws, device="cuda")
    eng = E.Engine()
    eng.work_items(G * lws, lws).scheduler("monolithic", ())
    eng.program(E.Program("fp32_probe").out(out).args(out, iters, 0.999, 0.001))
    s = torch.cuda.current_stream()
    for _ in range(2):
        eng.run()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        eng.run()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    eng.close()
    ms = statistics.median(ts)
    rate = 128.0 * iters * G * lws / (ms * 1e-3)
    return dict(ffma_per_s=rate, ms=ms, at_sm_mhz=sm_mhz, ffma_per_clk_per_sm=rate / (sms * sm_mhz * 1e6),
                launch="%d CTAs x 256 threads, 8 chains x %d FFMA each" % (G, 16 * iters))


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks (the slowest rank's time); every rank gets it."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def step_config(wls):
    """The workload's description, the same for both arms."""
    swls = [w for w in wls if w.in_step]
    return {"workload": "+".join(w.name for w in swls), "programs": {w.name: w.config for w in swls},
            "beside_the_step": {w.name: w.config for w in wls if not w.in_step},
            "l2": "flushed (512 MiB write) before every step", "parallelism": "replicas"}


def cpu_baseline(wls, total_wi, args):
    """Oracle on the host cores: a bounded sample of each program, scaled to the full step."""
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    full_s = 0.0
    samples = []
    for w in wls:
        frac, secs, what = w.cpu_sample(oracle, threads, CPU_SAMPLE)
        full_s += secs / frac
        samples.append("%s: %s in %.2fs" % (w.name, what, secs))
    return dict(value=total_wi / full_s, unit="work-items/s", cores=threads, kind="oracle",
                sample="; ".join(samples) + " (the full step's time projected from these samples)")


def run_reference(args):
    """The reference arm: the CPU oracle timed on this configuration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.default_threads()

    names = args.only.split(",") if args.only else None
    allw = []
    for cls in WORKLOADS:
        if names is None or cls.name in names:
            w = cls(None, None, 0)
            w.host_setup()
            allw.append(w)
    if names is not None and not any(w.in_step for w in allw):
        for w in allw:
            w.in_step = True
    wls = [w for w in allw if w.in_step]  # sampled; the rest only describe the configuration
    total_wi = sum(w.work_items() for w in wls)
    # a step is one bounded sample of every program of the workload: its time
    # is the measured time of that sample, its work the sampled work-items
    times, wis = [], []
    what, frac = {}, {}
    for i in range(args.warmup + args.steps):
        secs_step, wi_step = 0.0, 0.0
        for w in wls:
            f, secs, desc = w.cpu_sample(oracle, threads, CPU_SAMPLE)
            what[w.name], frac[w.name] = desc, f
            secs_step += secs
            wi_step += f * w.work_items()
        if i >= args.warmup:
            times.append(secs_step)
            wis.append(wi_step)
    step_s = statistics.median(times)
    val = statistics.median(wi / t for wi, t in zip(wis, times))
    samples = "; ".join("%s: %s" % kv for kv in what.items())
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "work-items/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, shaped like the "
        "paper's workloads)",
        "config": step_config(allw),
        "step": "one bounded sample of every program per step (ms_per_step is its measured time); the full "
                "step of %d work-items would take %.0f s at this rate" % (total_wi, total_wi / val),
        "sampled_fraction": frac,
        "cpu_baseline": {"value": val, "unit": "work-items/s", "cores": threads, "kind": "oracle",
                         "sample": samples},
        "e2e": {"value": val, "unit": "work-items/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--only", default="")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="reduced sizes for profiler captures")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-launch comparison")
    ap.add_argument("--no-autotune", action="store_true", help="skip the autotuner's search for the tunable programs")
    args = ap.parse_args()
    global SMALL
    SMALL = args.small
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
