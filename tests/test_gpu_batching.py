"""Batched launches (many uneven option batches, one persistent launch), CUDA
graph replay of engine runs, and the autotuner."""
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


def make_batches(torch, sizes, seed, greeks=True):
    out = []
    for i, n in enumerate(sizes):
        o = W.binomial_options(n, seed=seed + i, min_steps=1, max_steps=700)
        b = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
        b["r"] = o["r"]
        b["price"] = torch.full((n,), -1.0, device="cuda")
        b["greeks"] = torch.full((n, 2), -1.0, device="cuda") if greeks else None
        b["host"] = o
        out.append(b)
    return out


def check_batches(batches, oracle_mod):
    for b in batches:
        o = b["host"]
        rp, rd, rv = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
        S = o["S"].astype(np.float64)
        p = b["price"].cpu().numpy()
        assert (np.abs(p - rp) <= 1e-5 * np.maximum(rp, 1e-4 * S)).all()
        if b["greeks"] is not None:
            g = b["greeks"].cpu().numpy()
            assert (np.abs(g[:, 0] - rd) <= 1e-5 * np.maximum(np.abs(rd), 1e-4)).all()
            assert (np.abs(g[:, 1] - rv) <= 1e-5 * np.maximum(np.abs(rv), 1e-4 * S)).all()


def test_uneven_batches_one_launch(E, oracle_mod):
    import torch
    from paper_1805_02755_gb300.batching import BinomialBatch
    sizes = [1, 37, 250, 3, 1000, 64, 2]
    batches = make_batches(torch, sizes, 800)
    bb = BinomialBatch(batches, with_greeks=True)
    bb.run()
    torch.cuda.synchronize()
    assert bb.engine.plan_info()["G"] == sum(sizes)
    check_batches(batches, oracle_mod)
    bb.close()
    # without greeks (and one batch without a greeks buffer) the prices are the same
    nb = make_batches(torch, sizes, 800, greeks=False)
    bb = BinomialBatch(nb, with_greeks=False)
    bb.run()
    torch.cuda.synchronize()
    for a, b in zip(batches, nb):
        assert torch.equal(a["price"], b["price"])
    bb.close()


def test_graph_replay_equals_eager(E, oracle_mod):
    import torch
    from paper_1805_02755_gb300.batching import BinomialBatch, capture_graph
    batches = make_batches(torch, [200, 5, 700, 31], 900)
    bb = BinomialBatch(batches)
    g = capture_graph(bb.engine)
    for _ in range(2):
        for b in batches:
            b["price"].fill_(-1.0)
            b["greeks"].fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        check_batches(batches, oracle_mod)
    bb.close()
    # a Gaussian engine captured and replayed
    img = W.gaussian_image(300, 517, seed=3)
    w = W.gaussian_weights(31, 5.0)
    x, wt = torch.from_numpy(img).cuda(), torch.from_numpy(w).cuda()
    out = torch.zeros(300 * 517, device="cuda")
    eng = E.Engine(0)
    p = E.Program("gaussian").in_(x).in_(wt).out(out).args(x, wt, out, 517, 300, 31)
    eng.work_items(-(-300 * 517 // 128) * 128, 128).scheduler("dynamic", (16,)).workers(4, 0).program(p)
    g2 = capture_graph(eng)
    out.zero_()
    g2.replay()
    torch.cuda.synchronize()
    ref = oracle_mod.gaussian(img, w)
    assert (np.abs(out.cpu().numpy().reshape(300, 517) - ref) <= 1e-5 * np.abs(ref)).all()
    eng.close()


def test_autotune_picks_and_caches(E, tmp_path):
    import torch
    from paper_1805_02755_gb300 import autotune
    Wd = H = 512
    out = torch.zeros(Wd * H, dtype=torch.int32, device="cuda")

    def prog():
        return E.Program("mandelbrot").out(out).args(out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, 128)
    space = [dict(scheduler="hguided", params=[2.0, 1.0], devices=8, ctas=0),
             dict(scheduler="dynamic", params=[64], devices=1, ctas=0),
             dict(scheduler="static", params=[], devices=4, ctas=0)]
    cache = str(tmp_path / "tune.json")
    res = autotune.autotune("mandelbrot", prog, Wd * H // 4, 256, space=space, reps=2, cache_path=cache)
    assert res["config"] in space and len(res["table"]) == 3 and res["ms"] > 0
    again = autotune.autotune("mandelbrot", prog, Wd * H // 4, 256, space=[], cache_path=cache)
    assert again["config"] == res["config"]
