"""Failure path without a GPU fault: a fetcher that never publishes its package
(ECL_DEBUG_WITHHOLD) makes the other CTAs of its device wait out a short spin
limit; the run ends with ECL_ERR_TIMEOUT at the next synchronising call, and
the same engine then runs correctly again.  Every wait involved is bounded."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available()
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def expect_timeout_then_recover(E, eng, check):
    eng.debug(E.ECL_DEBUG_SPIN_LIMIT, 5000).debug(E.ECL_DEBUG_WITHHOLD, 1)
    with pytest.raises(E.EclError) as ei:
        eng.run()
        eng.synchronize()
    assert ei.value.status == E.ECL_ERR_TIMEOUT
    assert "void" in eng.last_error()
    eng.debug(E.ECL_DEBUG_WITHHOLD, 0).debug(E.ECL_DEBUG_SPIN_LIMIT, 0)
    eng.run().synchronize()
    check()


@pytest.mark.parametrize("sched,params", [("dynamic", (16,)), ("hguided", (2.0, 1.0))])
def test_mandelbrot_withheld_package_times_out(E, oracle_mod, sched, params):
    import torch
    Wd, H, it = 128, 96, 64
    out = torch.zeros(Wd * H, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    p = E.Program("mandelbrot").out(out).args(out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, it)
    eng.work_items(Wd * H // 4, 256).scheduler(sched, params).workers(2, 0).program(p)

    def check():
        ref = oracle_mod.mandelbrot(Wd, H, -2.0, -1.5, np.float32(3.0 / Wd), np.float32(3.0 / H), it)
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(H, Wd), ref)
    expect_timeout_then_recover(E, eng, check)
    eng.close()


def test_binomial_withheld_package_times_out(E, oracle_mod):
    import torch
    o = W.binomial_options(256, min_steps=1, max_steps=200)
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    price = torch.zeros(256, device="cuda")
    p = E.Program("binomial")
    for k in ("S", "K", "T", "sigma", "steps"):
        p.in_(t[k])
    p.out(price).args(t["S"], t["K"], t["T"], t["sigma"], t["steps"], o["r"], 256, price, None)
    eng = E.Engine(0)
    eng.work_items(256 * 32, 32).scheduler("dynamic", (8,)).workers(2, 0).program(p)

    def check():
        P, _, _ = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
        assert np.all(np.abs(price.cpu().numpy() - P) <= 1e-5 * np.maximum(P, 1e-4 * o["S"]))
    expect_timeout_then_recover(E, eng, check)
    eng.close()


def test_gemm_withheld_package_times_out(E, oracle_mod):
    import torch
    M, N, K = 512, 512, 128
    A, Bt = W.gemm_matrices(M, N, K, seed=5)
    a, b = torch.from_numpy(A).cuda(), torch.from_numpy(Bt).cuda()
    c = torch.zeros(M * N, device="cuda")
    eng = E.Engine(0)
    p = E.Program("gemm_split3").in_(a).in_(b).out(c).args(a, b, c, M, N, K)
    eng.work_items((M // 128) * (N // 256) * 32768, 32768).scheduler("dynamic", (4,)).workers(2, 0).program(p)

    def check():
        ref = oracle_mod.gemm(A, Bt, 2)
        aa = np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T
        assert np.all(np.abs(c.cpu().numpy().reshape(M, N) - ref) <= 1e-4 * aa)
    expect_timeout_then_recover(E, eng, check)
    eng.close()


def test_debug_rejects_bad_knobs(E):
    eng = E.Engine(0)
    with pytest.raises(E.EclError):
        eng.debug(99, 1)
    with pytest.raises(E.EclError):
        eng.debug(E.ECL_DEBUG_SPIN_LIMIT, -1)
    eng.close()


def test_trace_env_writes_chrome_traces(E, tmp_path, monkeypatch):
    import json
    import torch
    monkeypatch.setenv("ECL_TRACE", str(tmp_path))
    Wd, H = 128, 64
    out = torch.zeros(Wd * H, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    p = E.Program("mandelbrot").out(out).args(out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, 32)
    eng.work_items(Wd * H // 4, 256).scheduler("dynamic", (4,)).workers(2, 0).program(p)
    eng.run()
    files = sorted(tmp_path.glob("ecl_mandelbrot_*.json"))
    assert len(files) == 1
    ev = json.load(open(files[0]))["traceEvents"]
    assert len(ev) == 4 and sum(e["args"]["len_wg"] for e in ev) == Wd * H // 4 // 256
    eng.close()
