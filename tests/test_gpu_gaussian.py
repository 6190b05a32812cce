"""Separable Gaussian through the C ABI vs the FP64 oracle (1e-5 relative per pixel)."""
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


def run_gauss(E, img, w, lws=128, sched="dynamic", params=(256,), D=0, C=0, coverage=False, eng=None):
    import torch
    H, Wd = img.shape
    x = torch.from_numpy(img).cuda()
    wt = torch.from_numpy(w).cuda()
    out = torch.full((H * Wd + 8,), -7.0, dtype=torch.float32, device="cuda")
    own = eng is None
    eng = eng or E.Engine(0)
    gws = -(-H * Wd // lws) * lws
    cov = torch.zeros(gws // lws, dtype=torch.int32, device="cuda") if coverage else None
    p = E.Program("gaussian").in_(x).in_(wt).out(out).args(x, wt, out, Wd, H, len(w))
    eng.work_items(gws, lws).scheduler(sched, params).workers(D, C).program(p)
    eng.set_coverage(cov)
    eng.run().synchronize()
    res = out[: H * Wd].cpu().numpy().reshape(H, Wd)
    assert (out[H * Wd:].cpu().numpy() == -7.0).all(), "wrote past the image"
    if own:
        eng.close()
    return res, cov


def check(got, ref):
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
    assert np.isfinite(got).all()
    assert rel.max() <= RTOL, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))


@pytest.mark.parametrize("shape", [(64, 256), (37, 1000), (300, 515), (5, 3), (1, 1), (33, 257), (96, 4096)])
@pytest.mark.parametrize("taps", [31, 1, 7, 63])
def test_shapes_and_taps(E, oracle_mod, shape, taps):
    img = W.gaussian_image(*shape, seed=100 + shape[0])
    w = W.gaussian_weights(taps, max(taps / 6.0, 0.5))
    got, _ = run_gauss(E, img, w, sched="hguided", params=(2.0, 1.0))
    check(got, oracle_mod.gaussian(img, w))


SCHEDS = [("static", (), 1, 0), ("static", (0.2, 0.3), 3, 2), ("static_rev", (0.2, 0.3), 3, 1),
          ("dynamic", (256,), 0, 0), ("dynamic", (13,), 8, 4), ("hguided", (2.0, 1.0), 0, 0),
          ("hguided", (1.0, 4.0, 1.0, 2.0), 2, 3), ("monolithic", (), 0, 0)]


@pytest.mark.parametrize("sched,params,D,C", SCHEDS)
def test_schedulers_partial_rows(E, oracle_mod, sched, params, D, C):
    # lws 100 does not divide the width: packages start and end mid-row
    img = W.gaussian_image(150, 777, seed=7)
    w = W.gaussian_weights(31, 5.0)
    got, cov = run_gauss(E, img, w, lws=100, sched=sched, params=params, D=D, C=C,
                         coverage=(sched != "monolithic"))
    check(got, oracle_mod.gaussian(img, w))
    if cov is not None:
        assert (cov.cpu().numpy() == 1).all()


def test_config2_full_size_sampled_rows(E, oracle_mod):
    # 8192 x 8192, 31 taps sigma 5, Dynamic with 256 row packages (32 rows each)
    img = W.gaussian_image(8192, 8192)
    w = W.gaussian_weights(31, 5.0)
    got, _ = run_gauss(E, img, w, lws=128, sched="dynamic", params=(256,))
    rows = [0, 1, 14, 15, 16, 31, 32, 33, 4095, 4096, 5000, 8160, 8176, 8190, 8191]
    for r in rows:
        ref = oracle_mod.gaussian(img, w, rows=(r, r + 1))[r]
        check(got[r][None, :], ref[None, :])
    # a constant image stays constant at full size (edges included)
    const = np.full((8192, 8192), 0.625, dtype=np.float32)
    got, _ = run_gauss(E, const, w)
    s = float(w.astype(np.float64).sum()) ** 2
    assert np.abs(got - 0.625 * s).max() <= RTOL * 0.625
