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


def _single_launch(E, torch, t, r):
    n = t["S"].numel()
    price = torch.full((n,), -2.0, device="cuda")
    gr = torch.full((n, 2), -2.0, device="cuda")
    eng = E.Engine(0)
    prog = E.Program("binomial")
    for k in ("S", "K", "T", "sigma", "steps"):
        prog.in_(t[k])
    prog.out(price).out(gr)
    prog.args(t["S"], t["K"], t["T"], t["sigma"], t["steps"], r, n, price, gr)
    eng.work_items(n * 32, 32).scheduler("hguided", (2.0, 1.0)).workers(8, 0).program(prog)
    eng.run().synchronize()
    eng.close()
    return price, gr


def test_greeks_pass_bit_exact_across_options_per_warp_and_batching(E):
    # The greeks pass sets up several options per warp (one per lane: 32 at
    # 200003 options, 1 at 1037) and sums each option's leaves in turn.  An
    # option's results must not depend on that grouping, nor on the batched
    # launch's instance lookup: prices and greeks agree bit for bit,
    # including options of one step and of the deepest lattice.
    import torch
    from paper_1805_02755_gb300.batching import BinomialBatch
    n, m = 200003, 1037
    b = make_batches(torch, [n], 830)[0]
    b["steps"][:3] = 1
    b["steps"][3:6] = 2048  # the deepest lattice
    keys = ("S", "K", "T", "sigma", "steps")
    price, gr = _single_launch(E, torch, {k: b[k] for k in keys}, b["r"])
    p1, g1 = _single_launch(E, torch, {k: b[k][:m].clone() for k in keys}, b["r"])
    assert torch.equal(p1, price[:m])
    assert torch.equal(g1, gr[:m])
    # the same options as uneven instances of one batched launch
    sizes, lo, batches = [37, 1, 90000, 2, 109963], 0, []
    assert sum(sizes) == n
    for z in sizes:
        d = {k: b[k][lo:lo + z] for k in keys}
        d["r"] = b["r"]
        d["price"] = torch.full((z,), -1.0, device="cuda")
        d["greeks"] = torch.full((z, 2), -1.0, device="cuda")
        batches.append(d)
        lo += z
    bb = BinomialBatch(batches, with_greeks=True)
    bb.run()
    torch.cuda.synchronize()
    bb.close()
    assert torch.equal(torch.cat([d["price"] for d in batches]), price)
    assert torch.equal(torch.cat([d["greeks"] for d in batches]), gr)


def test_batches_with_and_without_greeks_arrays_in_one_launch(E, oracle_mod):
    # The greeks of a batch come from a pass after the lattice kernel, which
    # reads what the lattice left in each instance's greeks array: instances
    # without an array get prices only, the others their oracle greeks.
    import torch
    from paper_1805_02755_gb300.batching import BinomialBatch
    sizes = [5, 300, 1, 64, 129]
    batches = make_batches(torch, sizes, 810)
    for i in (1, 3):
        batches[i]["greeks"] = None
    bb = BinomialBatch(batches, with_greeks=True)
    bb.run()
    torch.cuda.synchronize()
    check_batches(batches, oracle_mod)
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


# ---------------------------------------------------------------- many views / images
VIEWS = [  # (W, H, x0, y0, dx, dy, max_iter): uneven sizes, ragged work-groups, zooms
    (1024, 768, -2.0, -1.5, 3.0 / 1024, 3.0 / 768, 256),
    (37, 5, -0.75, 0.05, 0.003, 0.002, 100),
    (1, 1, -0.5, 0.0, 0.01, 0.01, 64),
    (333, 129, -0.7453, 0.1127, 6.5e-5, 6.5e-5, 500),
    (64, 64, -1.8, -0.1, 0.003, 0.003, 1),
    (2000, 3, -2.0, -0.01, 0.0015, 0.01, 300),
]


def make_views(torch):
    out = []
    for (Wd, H, x0, y0, dx, dy, it) in VIEWS:
        out.append(dict(out=torch.full((Wd * H,), -1, dtype=torch.int32, device="cuda"), W=Wd, H=H,
                        x0=np.float32(x0), y0=np.float32(y0), dx=np.float32(dx), dy=np.float32(dy), max_iter=it))
    return out


def check_views(views, oracle_mod):
    for v in views:
        ref = oracle_mod.mandelbrot(v["W"], v["H"], v["x0"], v["y0"], v["dx"], v["dy"], v["max_iter"])
        got = v["out"].cpu().numpy().view(np.uint32).reshape(v["H"], v["W"])
        assert np.array_equal(got, ref), (v["W"], v["H"])


@pytest.mark.parametrize("sched,params,D,C", [("hguided", (2.0, 1.0), 0, 0), ("dynamic", (16,), 8, 0),
                                              ("static", (), 1, 0), ("hguided", (1.0, 4.0), 4, 3)])
def test_mandelbrot_views_one_launch_bit_exact(E, oracle_mod, sched, params, D, C):
    import torch
    from paper_1805_02755_gb300.batching import MandelbrotBatch
    views = make_views(torch)
    mb = MandelbrotBatch(views, scheduler=(sched, params), workers=(D, C))
    cov = torch.zeros(mb.total, dtype=torch.int32, device="cuda")
    mb.engine.set_coverage(cov)
    mb.run().engine.synchronize()
    assert mb.engine.plan_info()["G"] == sum(MandelbrotBatch.workgroups(v[0], v[1]) for v in VIEWS)
    assert (cov.cpu().numpy() == 1).all()  # every work-group of every view exactly once
    check_views(views, oracle_mod)
    mb.close()


IMAGES = [(96, 160, 5.0), (33, 300, 2.0), (512, 17, 8.0), (1, 1, 5.0), (250, 700, 3.5), (40, 225, 5.0)]  # H, W, sigma


def make_images(torch):
    out = []
    for i, (H, Wd, sg) in enumerate(IMAGES):
        img = W.gaussian_image(H, Wd, seed=900 + i)
        w = W.gaussian_weights(31, sg)
        out.append(dict(host=img, hw=w, **{"in": torch.from_numpy(img).cuda()},
                        out=torch.full((H * Wd,), -1.0, device="cuda"), w=torch.from_numpy(w).cuda(), W=Wd, H=H))
    return out


def check_images(images, oracle_mod):
    for im in images:
        ref = oracle_mod.gaussian(im["host"], im["hw"])
        got = im["out"].cpu().numpy().reshape(im["H"], im["W"])
        assert (np.abs(got - ref) <= 1e-5 * np.abs(ref)).all(), (im["H"], im["W"])


@pytest.mark.parametrize("sched,params,D,C", [("hguided", (2.0, 1.0), 0, 0), ("dynamic", (7,), 0, 0),
                                              ("static", (0.3, 0.3), 3, 0)])
def test_gaussian_images_one_launch(E, oracle_mod, sched, params, D, C):
    import torch
    from paper_1805_02755_gb300.batching import GaussianBatch
    images = make_images(torch)
    gb = GaussianBatch(images, scheduler=(sched, params), workers=(D, C))
    cov = torch.zeros(gb.total, dtype=torch.int32, device="cuda")
    gb.engine.set_coverage(cov)
    gb.run().engine.synchronize()
    assert gb.total == sum(GaussianBatch.tiles(w, h) for (h, w, _) in IMAGES)
    assert (cov.cpu().numpy() == 1).all()
    check_images(images, oracle_mod)
    gb.close()


def test_mixed_batches_replayed_from_one_graph_with_a_tuned_config(E, oracle_mod):
    # a Mandelbrot batch and a Gaussian batch, each one persistent launch,
    # captured together into one CUDA graph and replayed; the scheduler
    # parameters come from the autotuner's result format
    import torch
    from paper_1805_02755_gb300.batching import GaussianBatch, MandelbrotBatch
    views, images = make_views(torch), make_images(torch)
    cfg = dict(scheduler="hguided", params=[1.0, 2.0], devices=16, ctas=0)
    mb = MandelbrotBatch(views, config=cfg)
    gb = GaussianBatch(images, config=cfg)
    s = torch.cuda.Stream()
    for b in (mb, gb):
        b.engine.set_stream(s)
    with torch.cuda.stream(s):
        mb.run()
        gb.run()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mb.run()
        gb.run()
    for v in views:
        v["out"].fill_(-1)
    for im in images:
        im["out"].fill_(-1.0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert mb.engine.plan_info()["devices"] == 16 and gb.engine.plan_info()["devices"] == 16
    check_views(views, oracle_mod)
    check_images(images, oracle_mod)
    mb.close()
    gb.close()


def test_batch_tables_reject_bad_instances(E):
    import torch
    from paper_1805_02755_gb300.batching import GaussianBatch, MandelbrotBatch
    ok = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        MandelbrotBatch([dict(out=ok, W=8, H=9, x0=0, y0=0, dx=1, dy=1, max_iter=1)])  # 72 > 64 pixels
    with pytest.raises(ValueError):
        MandelbrotBatch([dict(out=ok[1:], W=4, H=4, x0=0, y0=0, dx=1, dy=1, max_iter=1)])  # misaligned
    f = torch.zeros(64, device="cuda")
    w = torch.zeros(30, device="cuda")
    with pytest.raises(ValueError):
        GaussianBatch([{"in": f, "out": f, "w": w, "W": 8, "H": 8}])  # 30 weights
