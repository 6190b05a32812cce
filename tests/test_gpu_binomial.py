"""Binomial (CRR European call) through the C ABI vs the FP64 oracle.

Tolerance from the FP32 error analysis of the lattice: each backward level adds
at most eps times the probability-weighted node values, whose sum is the price
itself, so the error is ~sqrt(N) eps V (N eps V worst case); 1e-5 relative is
applied to max(V64, 1e-4 S) so that prices far out of the money, which carry
the rounding of S-sized leaves, are measured on the scale of S.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available()
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def run_bino(E, o, greeks=True, sched="hguided", params=(2.0, 1.0), D=8, C=0, coverage=False, kernel="binomial"):
    import torch
    n = len(o["S"])
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    price = torch.full((n,), -1.0, device="cuda")
    gr = torch.full((n, 2), -1.0, device="cuda") if greeks else None
    eng = E.Engine(0)
    cov = torch.zeros(n, dtype=torch.int32, device="cuda") if coverage else None
    p = E.Program(kernel)
    for k in ("S", "K", "T", "sigma", "steps"):
        p.in_(t[k])
    p.out(price)
    if gr is not None:
        p.out(gr)
    p.args(t["S"], t["K"], t["T"], t["sigma"], t["steps"], o["r"], n, price, gr)
    eng.work_items(n * 32, 32).scheduler(sched, params).workers(D, C).program(p)
    eng.set_coverage(cov)
    eng.run().synchronize()
    out = (price.cpu().numpy(), gr.cpu().numpy() if gr is not None else None, cov)
    eng.close()
    return out


def check(o, price, gr, oracle_mod, idx=None):
    idx = np.arange(len(o["S"])) if idx is None else idx
    sub = {k: o[k][idx] for k in ("S", "K", "T", "sigma", "steps")}
    rp, rd, rv = oracle_mod.binomial(sub["S"], sub["K"], sub["T"], sub["sigma"], sub["steps"], o["r"])
    S = sub["S"].astype(np.float64)
    ep = np.abs(price[idx] - rp) / np.maximum(rp, 1e-4 * S)
    assert ep.max() <= RTOL, (ep.max(), idx[ep.argmax()])
    if gr is not None:
        ed = np.abs(gr[idx, 0] - rd) / np.maximum(np.abs(rd), 1e-4)
        ev = np.abs(gr[idx, 1] - rv) / np.maximum(np.abs(rv), 1e-4 * S)
        assert ed.max() <= RTOL, (ed.max(), idx[ed.argmax()])
        assert ev.max() <= RTOL, (ev.max(), idx[ev.argmax()])
    return ep.max()


@pytest.mark.parametrize("lo,hi", [(1, 40), (1, 300), (256, 700), (1000, 2048)])
def test_depth_ranges(E, oracle_mod, lo, hi):
    o = W.binomial_options(300 if hi < 1000 else 60, seed=400 + lo, min_steps=lo, max_steps=hi)
    price, gr, _ = run_bino(E, o)
    check(o, price, gr, oracle_mod)


def test_every_depth_boundary(E, oracle_mod):
    # depths at every lane-width switch (32 x {1, 2, ..., 56, 64}) and the extremes
    widths = [1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64]  # both width lists
    steps = sorted({v for w in widths for v in (32 * w - 1, 32 * w, 32 * w + 1) if 1 <= v <= 2048} | {1, 2, 3})
    steps = np.array(steps, dtype=np.int32)
    o = W.binomial_options(len(steps), seed=41)
    o["steps"] = steps
    price, gr, _ = run_bino(E, o)
    check(o, price, gr, oracle_mod)


def test_price_only_equals_price_with_greeks(E):
    o = W.binomial_options(500, seed=42)
    p1, _, _ = run_bino(E, o, greeks=False)
    p2, _, _ = run_bino(E, o, greeks=True)
    assert np.array_equal(p1, p2)


@pytest.mark.parametrize("sched,params,D,C", [("static", (), 1, 0), ("dynamic", (64,), 0, 0),
                                              ("hguided", (2.0, 1.0), 0, 0), ("monolithic", (), 0, 0)])
def test_schedulers(E, oracle_mod, sched, params, D, C):
    o = W.binomial_options(400, seed=43, min_steps=1, max_steps=600)
    price, gr, cov = run_bino(E, o, True, sched, params, D, C, coverage=(sched != "monolithic"))
    check(o, price, gr, oracle_mod)
    if cov is not None:
        assert (cov.cpu().numpy() == 1).all()


def test_config4_full_batch_sampled(E, oracle_mod):
    o = W.binomial_options(1 << 20)
    price, gr, _ = run_bino(E, o, True, "hguided", (2.0, 1.0), 8, 0)
    assert np.isfinite(price).all() and np.isfinite(gr).all()
    idx = np.sort(np.random.default_rng(7).choice(1 << 20, 384, replace=False))
    check(o, price, gr, oracle_mod, idx)
    # price within no-arbitrage bounds everywhere: max(S - K e^{-rT}, 0) <= C <= S
    S, K, T = o["S"], o["K"], o["T"]
    lb = np.maximum(S - K * np.exp(-o["r"] * T), 0)
    assert (price >= lb - 1e-4 * S).all() and (price <= S * (1 + 1e-6)).all()
    assert (gr[:, 0] >= -1e-6).all() and (gr[:, 0] <= 1 + 1e-5).all() and (gr[:, 1] >= -1e-4).all()


def test_banded_lattice_matches_the_full_lattice(E):
    # The banded program skips nodes that are exactly zero, stores the call
    # lattice reflected and takes its greeks from closed-form adjoint
    # weights; the full program computes every node in node order and runs
    # the adjoint lattice.  Prices agree bit for bit; the two greeks
    # evaluations (each within ~1e-6 of the exact values) agree to 5e-6.
    # Every width boundary, the extremes, then a random batch.
    widths = [1, 2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64]
    steps = sorted({v for w in widths for v in (32 * w - 1, 32 * w, 32 * w + 1) if 1 <= v <= 2048} | {1, 2, 3})
    o = W.binomial_options(len(steps), seed=44)
    o["steps"] = np.array(steps, dtype=np.int32)
    for opts in (o, W.binomial_options(4096, seed=45)):
        for greeks in (True, False):
            pb, gb, _ = run_bino(E, opts, greeks, kernel="binomial")
            pf, gf, _ = run_bino(E, opts, greeks, kernel="binomial_full")
            assert np.array_equal(pb.view(np.uint32), pf.view(np.uint32))
            if greeks:
                scale = np.maximum(np.abs(gf), np.stack([np.full(len(gf), 1e-4), 1e-4 * opts["S"]], 1))
                assert (np.abs(gb - gf) <= 5e-6 * scale).all(), (np.abs(gb - gf) / scale).max()


def test_deep_out_of_the_money_band_of_one_leaf(E, oracle_mod):
    # strikes far from the spot: no leaf or a single leaf in the money
    o = W.binomial_options(64, seed=46, min_steps=1, max_steps=2048)
    o["K"] = (o["S"] * np.where(np.arange(64) % 2 == 0, 40.0, 0.02)).astype(np.float32)
    price, gr, _ = run_bino(E, o)
    pf, gf, _ = run_bino(E, o, kernel="binomial_full")
    assert np.array_equal(price.view(np.uint32), pf.view(np.uint32))
    check(o, price, gr, oracle_mod)


def test_kernel_events_time_the_lattice_kernel_alone(E):
    # ecl_engine_kernel_events: the events bracket the lattice kernel, not the
    # greeks pass after it, so they span less than the whole run; the results
    # are those of a run without events
    import torch
    o = W.binomial_options(4096, seed=47)
    n = len(o["S"])
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    outs = []
    for with_events in (False, True):
        price = torch.full((n,), -1.0, device="cuda")
        gr = torch.full((n, 2), -1.0, device="cuda")
        eng = E.Engine(0)
        p = E.Program("binomial")
        for k in ("S", "K", "T", "sigma", "steps"):
            p.in_(t[k])
        p.out(price).out(gr)
        p.args(t["S"], t["K"], t["T"], t["sigma"], t["steps"], o["r"], n, price, gr)
        eng.work_items(n * 32, 32).scheduler("hguided", (2.0, 1.0)).workers(8, 0).program(p)
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if with_events:
            k0.record(stream)
            k1.record(stream)
            eng.kernel_events(k0, k1)
        a.record(stream)
        eng.run()
        b.record(stream)
        torch.cuda.synchronize()
        if with_events:
            whole, main = a.elapsed_time(b), k0.elapsed_time(k1)
            assert 0 < main < whole, (main, whole)
            assert a.elapsed_time(k0) >= 0 and k1.elapsed_time(b) > 0
            eng.kernel_events(None, None)
        outs.append((price.cpu().numpy(), gr.cpu().numpy()))
        eng.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
