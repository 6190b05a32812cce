"""torch.autograd wrappers whose backward passes are the library's adjoint kernels.

* ``nbody_energy(pos4, eps2)``: E = -sum_{i<j} m_i m_j / sqrt(|r_ij|^2 + eps2)
  (the "nbody_energy" program, FP32 pair terms, FP64 sums).  Backward runs the
  "nbody_adjoint" program: dL/dpos4 = dL/dE * (dE/dr_i, dE/dm_i).
* ``binomial_price(S, K, T, sigma, steps, r)``: CRR call prices (the
  "binomial" program).  When S or sigma requires a gradient the forward launch
  also computes delta and vega (the lattice's adjoint weights in closed form,
  binomial probabilities: delta and the leaf part of vega are sums of those
  weights times the leaf derivatives over the nonzero leaves), and
  backward returns dL/dS = dL/dV * delta, dL/dsigma = dL/dV * vega.  K, T and
  r get no gradient.

Both run through the C ABI on the caller's current CUDA stream; engines are
cached per (program, device).
"""
from __future__ import annotations

import threading

import torch

from . import Engine, Program

_engines = {}
_lock = threading.Lock()


def _engine(kernel: str, device: int) -> Engine:
    key = (kernel, device)
    with _lock:
        eng = _engines.get(key)
        if eng is None:
            eng = Engine(device)
            _engines[key] = eng
    eng.set_stream(torch.cuda.current_stream(device))
    return eng


def _check_cuda(*ts):
    for t in ts:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("inputs must be contiguous CUDA tensors")


class NBodyEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos4: torch.Tensor, eps2: float, lws: int = 64):
        _check_cuda(pos4)
        if pos4.dtype != torch.float32 or pos4.dim() != 2 or pos4.shape[1] != 4:
            raise ValueError("pos4 must be float32 of shape (n, 4)")
        n = pos4.shape[0]
        dev = pos4.device.index if pos4.device.index is not None else torch.cuda.current_device()
        out = torch.empty(1, dtype=torch.float64, device=pos4.device)
        eng = _engine("nbody_energy", dev)
        p = Program("nbody_energy").in_(pos4).out(out).args(pos4, n, eps2, out)
        eng.work_items(-(-n // lws) * lws, lws).scheduler("hguided", (2.0, 1.0)).program(p).run()
        ctx.save_for_backward(pos4)
        ctx.eps2 = eps2
        ctx.lws = lws
        return out[0]

    @staticmethod
    def backward(ctx, grad_e: torch.Tensor):
        (pos4,) = ctx.saved_tensors
        n = pos4.shape[0]
        dev = pos4.device.index if pos4.device.index is not None else torch.cuda.current_device()
        g = grad_e.reshape(1).to(device=pos4.device, dtype=torch.float32).contiguous()
        grad = torch.empty_like(pos4)
        eng = _engine("nbody_adjoint", dev)
        p = Program("nbody_adjoint").in_(pos4).in_(g).out(grad).args(pos4, n, ctx.eps2, g, grad)
        eng.work_items(-(-n // ctx.lws) * ctx.lws, ctx.lws).scheduler("hguided", (2.0, 1.0)).program(p).run()
        return grad, None, None


class BinomialPrice(torch.autograd.Function):
    @staticmethod
    def forward(ctx, S, K, T, sigma, steps, r: float):
        _check_cuda(S, K, T, sigma, steps)
        n = S.shape[0]
        dev = S.device.index if S.device.index is not None else torch.cuda.current_device()
        price = torch.empty(n, dtype=torch.float32, device=S.device)
        need = ctx.needs_input_grad[0] or ctx.needs_input_grad[3]
        greeks = torch.empty((n, 2), dtype=torch.float32, device=S.device) if need else None
        eng = _engine("binomial", dev)
        p = Program("binomial")
        for t in (S, K, T, sigma, steps):
            p.in_(t)
        p.out(price)
        if greeks is not None:
            p.out(greeks)
        p.args(S, K, T, sigma, steps, r, n, price, greeks)
        eng.work_items(n * 32, 32).scheduler("hguided", (2.0, 1.0)).program(p).run()
        if greeks is not None:
            ctx.save_for_backward(greeks)
        ctx.has_greeks = greeks is not None
        return price

    @staticmethod
    def backward(ctx, grad_price):
        if not ctx.has_greeks:
            return None, None, None, None, None, None
        (greeks,) = ctx.saved_tensors
        g = grad_price.to(torch.float32)
        dS = g * greeks[:, 0] if ctx.needs_input_grad[0] else None
        dsig = g * greeks[:, 1] if ctx.needs_input_grad[3] else None
        return dS, None, None, dsig, None, None


def nbody_energy(pos4: torch.Tensor, eps2: float, lws: int = 64) -> torch.Tensor:
    return NBodyEnergy.apply(pos4, eps2, lws)


def binomial_price(S, K, T, sigma, steps, r: float) -> torch.Tensor:
    return BinomialPrice.apply(S, K, T, sigma, steps, r)
