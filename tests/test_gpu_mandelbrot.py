"""Mandelbrot through the C ABI on the GPU, bit-exact against the oracle, under
every scheduler, plus the package-queue invariants (coverage, package
sequence, self-resetting queue) and the host-buffer path."""
import numpy as np
import pytest

import workloads as W
from oracle import schedule as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def mandel_program(E, out, Wd, H, x0, y0, dx, dy, it):
    p = E.Program("mandelbrot")
    p.out(out)
    p.args(out, Wd, H, x0, y0, dx, dy, it)
    return p


def gws_for(npx, lws):
    wi = -(-npx // 4)
    return -(-wi // lws) * lws


def run(E, torch, Wd, H, it, sched, params=(), D=0, C=0, lws=256, coverage=False, region=None):
    r = region or dict(x0=-2.0, y0=-1.5, dx=3.0 / Wd, dy=3.0 / H)
    out = torch.full((Wd * H + 4,), -1, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    gws = gws_for(Wd * H, lws)
    G = gws // lws
    cov = torch.zeros(G, dtype=torch.int32, device="cuda") if coverage else None
    eng.work_items(gws, lws).scheduler(sched, params).workers(D, C)
    eng.program(mandel_program(E, out, Wd, H, r["x0"], r["y0"], r["dx"], r["dy"], it))
    if cov is not None:
        eng.set_coverage(cov)
    eng.run()
    eng.synchronize()
    res = out[: Wd * H].cpu().numpy().view(np.uint32).reshape(H, Wd)
    assert int(out[Wd * H]) == -1, "wrote past the image"
    return eng, res, cov, G, r


def oracle_img(O, Wd, H, it, r):
    return O.mandelbrot(Wd, H, np.float32(r["x0"]), np.float32(r["y0"]), np.float32(r["dx"]),
                        np.float32(r["dy"]), it)


def test_config1_full_static_one_package(E, torch, oracle_mod):
    reg = W.mandelbrot_region(1024, 1024, 256)
    r = dict(x0=reg["x0"], y0=reg["y0"], dx=reg["dx"], dy=reg["dy"])
    eng, img, _, G, _ = run(E, torch, 1024, 1024, 256, "static", (), D=1, region=r)
    assert G == 1024
    ref = oracle_img(oracle_mod, 1024, 1024, 256, r)
    assert np.array_equal(img, ref)
    st = eng.stats()
    assert len(st) == 1 and st[0]["off_wg"] == 0 and st[0]["len_wg"] == 1024
    ws = eng.worker_stats()
    assert ws["chunks"].sum() == 1024
    eng.close()


def test_static_one_device_runs_as_one_grid(E, torch, oracle_mod):
    """Static over one device has a single package [0, G) and nothing left to
    decide at run time: it runs as one grid, CTA b = chunk b, keeping the
    package record and one worker record per CTA.  Alternating with queue
    runs on the same engine keeps every run exact and covered once."""
    Wd, H, it = 1000, 37, 200
    r = dict(x0=-2.0, y0=-1.5, dx=3.0 / Wd, dy=3.0 / H)
    ref = oracle_img(oracle_mod, Wd, H, it, r)
    lws = 64
    gws = gws_for(Wd * H, lws)
    G = gws // lws
    out = torch.zeros(Wd * H + 4, dtype=torch.int32, device="cuda")
    cov = torch.zeros(G, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    eng.program(mandel_program(E, out, Wd, H, r["x0"], r["y0"], r["dx"], r["dy"], it)).set_coverage(cov)
    for sched, params, D, C in (("static", (), 1, 0), ("dynamic", (7,), 3, 1), ("static", (), 1, 0),
                                ("static_rev", (), 1, 5), ("hguided", (2.0, 1.0), 2, 3), ("static", (), 1, 0)):
        out.zero_()
        cov.zero_()
        eng.work_items(gws, lws).scheduler(sched, params).workers(D, C)
        eng.run()
        eng.synchronize()
        assert np.array_equal(out[: Wd * H].cpu().numpy().view(np.uint32).reshape(H, Wd), ref), sched
        assert (cov.cpu().numpy() == 1).all(), sched
        st, ws, info = eng.stats(), eng.worker_stats(), eng.plan_info()
        if sched.startswith("static"):
            assert info["devices"] == 1 and info["ctas"] == G and info["ctas_per_device"] == G
            assert len(st) == 1 and int(st[0]["off_wg"]) == 0 and int(st[0]["len_wg"]) == G
            assert len(ws) == G and (ws["chunks"] == 1).all() and (ws["device"] == 0).all()
            assert sorted(ws["cta"].tolist()) == list(range(G))
            assert (ws["t_last_ns"] >= ws["t_first_ns"]).all()
            assert int(st[0]["t1_ns"]) == int(ws["t_last_ns"].max())
            assert int(st[0]["t0_ns"]) == int(ws[ws["cta"] == 0]["t_first_ns"][0])
        else:
            assert int(ws["chunks"].sum()) >= len(st) >= 1
    eng.close()


def test_scale_up_8192_sampled_rows_and_symmetry(E, torch, oracle_mod):
    """The 8192^2, 1024-iteration scale-up (a row of the bench beside the step),
    Static one package: sampled rows bit-exact against the oracle (each as a
    one-row image at that row's c_y, formed in float32 as the kernel forms it),
    and the whole image symmetric about y = 0: dy = 3 * 2^-13, so rows j and
    8192 - j have c_y of opposite sign exactly, and the iteration commutes with
    conjugation in IEEE arithmetic (negation is exact, rounding symmetric)."""
    n, it = 8192, 1024
    reg = W.mandelbrot_region(n, n, it)
    r = dict(x0=reg["x0"], y0=reg["y0"], dx=reg["dx"], dy=reg["dy"])
    eng, img, _, G, _ = run(E, torch, n, n, it, "static", (), D=1, region=r)
    eng.close()
    assert G == n * n // 4 // 256
    assert np.array_equal(img[1:n // 2], img[n - 1:n // 2:-1])
    rows = [0, 1, 2047, n // 2 - 1, n // 2, 5000, n - 1] + \
        np.random.default_rng(1805).integers(0, n, 9).tolist()
    for j in rows:
        cy = np.float32(r["y0"]) + np.float32(j) * np.float32(r["dy"])
        ref = oracle_mod.mandelbrot(n, 1, np.float32(r["x0"]), cy, np.float32(r["dx"]), np.float32(r["dy"]), it)
        assert np.array_equal(img[j], ref[0]), j
    assert int(img.max()) == it and int(img[0, 0]) == 1


SCHEDS = [
    ("static", (), 1, 0), ("static", (), 5, 1), ("static", (0.1, 0.2, 0.3), 4, 3),
    ("static_rev", (0.1, 0.2, 0.3), 4, 2), ("dynamic", (7,), 3, 1), ("dynamic", (50,), 2, 8),
    ("dynamic", (150,), 0, 0), ("hguided", (2.0, 1.0), 8, 1), ("hguided", (1.0, 2.0), 3, 5),
    ("hguided", (2.0, 1.0, 1.0, 2.0, 4.0), 3, 1), ("hguided", (0.5, 1.0, 3.0, 1.0), 2, 4),
    ("monolithic", (), 0, 0),
]


@pytest.mark.parametrize("sched,params,D,C", SCHEDS)
def test_every_scheduler_bit_exact_and_covers_once(E, torch, oracle_mod, sched, params, D, C):
    Wd, H, it = 1000, 37, 200  # ragged: 37000 pixels, last work-group partial
    eng, img, cov, G, r = run(E, torch, Wd, H, it, sched, params, D, C, lws=64, coverage=True)
    assert np.array_equal(img, oracle_img(oracle_mod, Wd, H, it, r))
    if sched == "monolithic":
        eng.close()
        return
    assert (cov.cpu().numpy() == 1).all()
    st = eng.stats()
    info = eng.plan_info()
    Dn = info["devices"]
    if sched in ("static", "static_rev"):
        want = OS.static(G, Dn, list(params) or None, reverse=(sched == "static_rev"))
        got = [(0, 0)] * Dn
        for rec in st:
            assert rec["device"] == rec["pkg"]
            got[rec["pkg"]] = (int(rec["off_wg"]), int(rec["len_wg"]))
        assert got == want
    elif sched == "dynamic":
        want = OS.dynamic(G, int(params[0]))
        got = [(int(a), int(b)) for a, b in zip(st["off_wg"], st["len_wg"])]
        assert sorted(st["pkg"].tolist()) == list(range(len(want)))
        assert got == want
    else:
        k, mb = params[0], int(params[1])
        powers = list(params[2:]) or None
        by_off = st[np.argsort(st["off_wg"])]
        order = by_off["device"].tolist()
        want = OS.hguided(G, Dn, k=k, min_base=mb, powers=powers, request_order=order)
        assert [(d, o, l) for d, o, l in want] == \
            [(int(d), int(o), int(l)) for d, o, l in zip(by_off["device"], by_off["off_wg"], by_off["len_wg"])]
    assert (st["t1_ns"] >= st["t0_ns"]).all()
    eng.close()


@pytest.mark.parametrize("sched,params,D,C,Wd,H", [
    ("static", (), 300, 1, 1000, 37),          # more devices than work-groups: empty packages
    ("static_rev", (), 64, 2, 1000, 37),
    ("hguided", (1000.0, 1.0), 16, 3, 1000, 37),  # every package at the minimum size
    ("dynamic", (4,), 32, 4, 64, 4),           # one work-group in all (64 x 4 px, lws 64)
    ("hguided", (2.0, 1.0), 8, 8, 64, 4),
])
def test_degenerate_schedules_cover_once(E, torch, oracle_mod, sched, params, D, C, Wd, H):
    it = 150
    eng, img, cov, G, r = run(E, torch, Wd, H, it, sched, params, D, C, lws=64, coverage=True)
    assert np.array_equal(img, oracle_img(oracle_mod, Wd, H, it, r))
    assert (cov.cpu().numpy() == 1).all()
    st = eng.stats()
    assert int(st["len_wg"].sum()) == G
    eng.close()


def test_repeated_runs_reset_the_queue(E, torch, oracle_mod):
    Wd, H, it = 512, 512, 64
    out = torch.zeros(Wd * H, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    eng.work_items(gws_for(Wd * H, 256), 256).scheduler("dynamic", (33,)).workers(16, 4)
    eng.program(mandel_program(E, out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, it))
    ref = oracle_mod.mandelbrot(Wd, H, -2.0, -1.5, np.float32(3.0 / Wd), np.float32(3.0 / H), it)
    for _ in range(5):
        out.zero_()
        eng.run()
        eng.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(H, Wd), ref)
        # Dynamic: ceil(256 / 33) = 8 work-groups per package -> 32 packages
        assert len(eng.stats()) == len(OS.dynamic(Wd * H // 1024, 33)) == 32
    # switching scheduler on the same engine re-plans
    eng.scheduler("hguided", (2.0, 1.0)).workers(0, 0)
    out.zero_()
    eng.run()
    eng.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(H, Wd), ref)
    eng.close()


def test_host_buffers_are_copied_in_and_out(E, oracle_mod):
    Wd, H, it = 300, 200, 128
    out = np.zeros(Wd * H, dtype=np.uint32)
    eng = E.Engine(0)
    eng.work_items(gws_for(Wd * H, 256), 256).scheduler("hguided", (2.0, 2.0))
    eng.program(mandel_program(E, out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, it))
    eng.run()  # synchronous with host buffers: results are in `out` on return
    ref = oracle_mod.mandelbrot(Wd, H, -2.0, -1.5, np.float32(3.0 / Wd), np.float32(3.0 / H), it)
    assert np.array_equal(out.reshape(H, Wd), ref)
    eng.close()


def test_errors_are_latched_not_thrown(E, torch):
    out = torch.zeros(64 * 64, dtype=torch.int32, device="cuda")
    eng = E.Engine(0)
    with pytest.raises(E.EclError) as ei:
        eng.run()
    assert ei.value.status == E.ECL_ERR_STATE
    with pytest.raises(E.EclError) as ei:
        eng.work_items(1000, 256)
    assert ei.value.status == E.ECL_ERR_SIZE
    eng.work_items(256, 256)  # covers 1024 pixels of 4096
    eng.program(mandel_program(E, out, 64, 64, -2.0, -1.5, 3 / 64, 3 / 64, 10))
    with pytest.raises(E.EclError) as ei:
        eng.run()
    assert ei.value.status == E.ECL_ERR_SIZE
    assert eng.has_errors() and "does not cover" in eng.last_error()
    eng.clear_errors()
    # a buffer argument that was never registered
    other = torch.zeros(64 * 64, dtype=torch.int32, device="cuda")
    p = E.Program("mandelbrot")
    p.out(out)
    p.args(other, 64, 64, -2.0, -1.5, 3 / 64, 3 / 64, 10)
    eng.program(p).work_items(1024, 256)
    with pytest.raises(E.EclError) as ei:
        eng.run()
    assert ei.value.status == E.ECL_ERR_BUFFER
    # a registered buffer that is too small
    small = torch.zeros(100, dtype=torch.int32, device="cuda")
    p = E.Program("mandelbrot")
    p.out(small)
    p.args(small, 64, 64, -2.0, -1.5, 3 / 64, 3 / 64, 10)
    eng.program(p)
    with pytest.raises(E.EclError) as ei:
        eng.run()
    assert ei.value.status == E.ECL_ERR_BUFFER
    # scheduler parameters checked against D at run time
    p = E.Program("mandelbrot")
    p.out(out)
    p.args(out, 64, 64, -2.0, -1.5, 3 / 64, 3 / 64, 10)
    eng.program(p).scheduler("static", (0.5, 0.5, 0.5)).workers(2, 1)
    with pytest.raises(E.EclError) as ei:
        eng.run()
    assert ei.value.status == E.ECL_ERR_SCHED
    eng.close()
