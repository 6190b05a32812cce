"""The FP32 pipe probe (the measured side of the FP32 rooflines) through the C
ABI: every work-item writes the sum of its eight FFMA chains, checked against
the same chains run in float64 on the host (the chains contract toward
c / (1 - m), so FP32 rounding stays below 1e-6 relative)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def test_probe_values_and_rate(E):
    import torch
    lws, iters, G = 256, 3, 37
    m, c = np.float32(0.999), np.float32(0.001)
    out = torch.full((G * lws + 1,), -1.0, device="cuda")
    eng = E.Engine(0)
    eng.work_items(G * lws, lws).scheduler("monolithic", ())
    eng.program(E.Program("fp32_probe").out(out).args(out, iters, float(m), float(c)))
    eng.run()
    eng.synchronize()
    got = out.cpu().numpy()
    assert got[-1] == -1.0, "wrote past gws"
    wi = np.arange(G * lws)
    x = np.stack([(np.float32(1.0) + (wi & 255).astype(np.float32) * np.float32(1e-3)
                   + np.float32(k) * np.float32(1e-4)).astype(np.float64) for k in range(8)])
    for _ in range(16 * iters):
        x = x * float(m) + float(c)
    want = x.sum(0)
    assert np.all(np.abs(got[:-1] - want) <= 1e-6 * np.abs(want))
    eng.close()


def test_probe_rejects_other_lws(E):
    import torch
    out = torch.zeros(128 * 4, device="cuda")
    eng = E.Engine(0)
    eng.work_items(128 * 4, 128).scheduler("monolithic", ())
    eng.program(E.Program("fp32_probe").out(out).args(out, 1, 0.999, 0.001))
    with pytest.raises(E.EclError):
        eng.run()
    eng.close()
