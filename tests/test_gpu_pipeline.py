"""pipeline.Overlapped: engines run in order with their host copies on two copy
streams; every result lands in pinned host memory equal to the oracle's, run
after run (the device inputs are rewritten from the host each time)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def test_overlapped_stages_match_the_oracle(E, oracle_mod):
    import torch
    from paper_1805_02755_gb300 import pipeline as PL
    # stage 1: Mandelbrot, output only
    Wd, H, it = 512, 256, 200
    m_out = torch.zeros(Wd * H, dtype=torch.int32, device="cuda")
    m_host = torch.zeros(Wd * H, dtype=torch.int32).pin_memory()
    e1 = E.Engine(0)
    e1.work_items(Wd * H // 4, 256).scheduler("static", ()).workers(1, 0)
    e1.program(E.Program("mandelbrot").out(m_out).args(m_out, Wd, H, -2.0, -1.5, 3.0 / Wd, 3.0 / H, it))
    # stage 2: Gaussian, input and output
    img = W.gaussian_image(192, 320)
    w = W.gaussian_weights()
    g_in_h = torch.from_numpy(img).pin_memory()
    g_w_h = torch.from_numpy(w).pin_memory()
    g_in = torch.zeros_like(g_in_h, device="cuda")
    g_w = torch.zeros_like(g_w_h, device="cuda")
    g_out = torch.zeros_like(g_in)
    g_host = torch.zeros_like(g_in_h).pin_memory()
    e2 = E.Engine(0)
    e2.work_items(192 * 320, 128).scheduler("dynamic", (16,)).workers(4, 0)
    e2.program(E.Program("gaussian").in_(g_in).in_(g_w).out(g_out).args(g_in, g_w, g_out, 320, 192, 31))
    ov = PL.Overlapped([PL.Stage(e1, outputs=[(m_host, m_out)]),
                        PL.Stage(e2, inputs=[(g_in, g_in_h), (g_w, g_w_h)], outputs=[(g_host, g_out)])])
    assert ov.bytes_in == img.nbytes + w.nbytes and ov.bytes_out == m_host.numel() * 4 + g_host.numel() * 4
    m_ref = oracle_mod.mandelbrot(Wd, H, -2.0, -1.5, np.float32(3.0 / Wd), np.float32(3.0 / H), it)
    g_ref = oracle_mod.gaussian(img, w)
    for _ in range(3):
        g_in.zero_()  # the next run must copy the input in again
        m_host.zero_()
        g_host.zero_()
        ov.run()
        assert np.array_equal(m_host.numpy().view(np.uint32).reshape(H, Wd), m_ref)
        g = g_host.numpy().reshape(192, 320)
        assert np.all(np.abs(g - g_ref) <= 1e-5 * np.abs(g_ref))
    e1.close()
    e2.close()


def test_c_abi_copy_streams_asynchronous_runs(E, oracle_mod):
    # Two engines with host (pinned) buffers, copies on two copy streams,
    # asynchronous runs: the Gaussian input changes between runs, so a copy
    # in that overtook the previous run's kernel, or a kernel that overtook
    # the previous run's copy out, would show in the results.
    import torch
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    Wd, H = 320, 192
    w = torch.from_numpy(W.gaussian_weights()).pin_memory()
    imgs = [W.gaussian_image(H, Wd, seed=1200 + i) for i in range(4)]
    g_in = torch.zeros(H * Wd).pin_memory()
    g_out = torch.zeros(H * Wd).pin_memory()
    eg = E.Engine(0)
    eg.work_items(H * Wd, 128).scheduler("dynamic", (16,)).workers(8, 0)
    eg.program(E.Program("gaussian").in_(g_in).in_(w).out(g_out).args(g_in, w, g_out, Wd, H, 31))
    eg.copy_streams(copy_in, copy_out, asynchronous=True)
    mw, mh, it = 512, 128, 300
    m_out = torch.zeros(mw * mh, dtype=torch.int32).pin_memory()
    em = E.Engine(0)
    em.work_items(mw * mh // 4, 256).scheduler("hguided", (2.0, 1.0)).workers(8, 0)
    em.program(E.Program("mandelbrot").out(m_out).args(m_out, mw, mh, -2.0, -1.0, 3.0 / mw, 2.0 / mh, it))
    em.copy_streams(copy_in, copy_out, asynchronous=True)
    mref = oracle_mod.mandelbrot(mw, mh, -2.0, -1.0, np.float32(3.0 / mw), np.float32(2.0 / mh), it)
    for img in imgs:
        g_in.copy_(torch.from_numpy(img.reshape(-1)))
        eg.run()
        em.run()
        eg.synchronize()
        em.synchronize()
        ref = oracle_mod.gaussian(img, W.gaussian_weights())
        got = g_out.numpy().reshape(H, Wd)
        assert (np.abs(got - ref) <= 1e-5 * np.abs(ref)).all()
        assert np.array_equal(m_out.numpy().view(np.uint32).reshape(mh, mw), mref)
        g_out.zero_()
        m_out.zero_()
    # back to synchronous runs with the copies on the copy streams
    eg.copy_streams(copy_in, copy_out, asynchronous=False)
    g_in.copy_(torch.from_numpy(imgs[0].reshape(-1)))
    eg.run()
    ref = oracle_mod.gaussian(imgs[0], W.gaussian_weights())
    assert (np.abs(g_out.numpy().reshape(H, Wd) - ref) <= 1e-5 * np.abs(ref)).all()
    eg.close()
    em.close()
