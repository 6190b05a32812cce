"""NBody force / step / energy / adjoint / finite differences through the C ABI
against the FP64 oracle.

Tolerance (1e-5 relative for FP32 kernels) is applied condition-aware: the
error of a_i is divided by sum_j m_j |d_ij| / (|d_ij|^2+eps2)^(3/2), the size of
the terms that cancel in it; a plain normwise error is checked as well.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-5
EPS2 = 1e-3


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available()
    from paper_1805_02755_gb300 import build as B
    B.build()
    import paper_1805_02755_gb300 as E
    return E


def cond(pos, idx, eps2=EPS2):
    """sum_j m_j |d_ij| (|d_ij|^2 + eps2)^(-3/2) for the bodies idx (FP64)."""
    p = pos.astype(np.float64)
    out = np.zeros(len(idx))
    for t, i in enumerate(idx):
        d = p[:, :3] - p[i, :3]
        r2 = (d * d).sum(1)
        out[t] = (p[:, 3] * np.sqrt(r2) / (r2 + eps2) ** 1.5).sum()
    return out


def gws_of(n, lws):
    return -(-n // lws) * lws


def run_acc(E, pos, lws=64, sched="hguided", params=(2.0, 1.0), D=0, C=0, coverage=False):
    import torch
    n = pos.shape[0]
    x = torch.from_numpy(pos).cuda()
    acc = torch.full((n, 4), 7.0, device="cuda")
    eng = E.Engine(0)
    gws = gws_of(n, lws)
    cov = torch.zeros(gws // lws, dtype=torch.int32, device="cuda") if coverage else None
    p = E.Program("nbody_acc").in_(x).out(acc).args(x, n, EPS2, acc)
    eng.work_items(gws, lws).scheduler(sched, params).workers(D, C).program(p)
    eng.set_coverage(cov)
    eng.run().synchronize()
    a = acc.cpu().numpy()
    eng.close()
    return a, cov


def check_acc(got, ref, pos, idx):
    err = np.abs(got[idx, :3] - ref[idx]).max(1)
    c = cond(pos, idx)
    assert (err[c == 0] == 0).all()  # a lone body feels no force
    k = c > 0
    assert (err[k] / c[k]).max(initial=0.0) <= RTOL, (err[k] / c[k]).max()
    assert np.linalg.norm(got[idx, :3] - ref[idx]) <= RTOL * np.linalg.norm(ref[idx])


@pytest.mark.parametrize("n", [1, 2, 3, 100, 257, 1000, 4096])
@pytest.mark.parametrize("lws", [32, 64, 256])
def test_acc_sizes(E, oracle_mod, n, lws):
    pos, _ = W.nbody_bodies(n, seed=200 + n)
    got, _ = run_acc(E, pos, lws=lws)
    ref = oracle_mod.nbody_acc(pos, EPS2)
    check_acc(got, ref, pos, np.arange(n))
    assert (got[:, 3] == 0).all()


SCHEDS = [("static", (), 1, 0), ("static_rev", (0.3, 0.3), 3, 1), ("dynamic", (50,), 4, 2),
          ("dynamic", (150,), 0, 0), ("hguided", (2.0, 2.0), 8, 1), ("hguided", (2.0, 1.0, 1.0, 3.0), 2, 5),
          ("monolithic", (), 0, 0)]


@pytest.mark.parametrize("sched,params,D,C", SCHEDS)
def test_acc_schedulers(E, oracle_mod, sched, params, D, C):
    pos, _ = W.nbody_bodies(3000, seed=5)
    got, cov = run_acc(E, pos, 64, sched, params, D, C, coverage=(sched != "monolithic"))
    ref = oracle_mod.nbody_acc(pos, EPS2)
    check_acc(got, ref, pos, np.arange(3000))
    if cov is not None:
        assert (cov.cpu().numpy() == 1).all()


def test_config3_full_size_sampled(E, oracle_mod):
    pos, _ = W.nbody_bodies(65536)
    got, _ = run_acc(E, pos, 64, "hguided", (2.0, 1.0), 8, 0)
    idx = np.random.default_rng(1).choice(65536, 256, replace=False)
    idx.sort()
    ref = np.zeros((65536, 3))
    for i in idx:
        ref[i] = oracle_mod.nbody_acc(pos, EPS2, bodies=(int(i), int(i) + 1))[i]
    check_acc(got, ref, pos, idx)
    # momentum: sum_i m_i a_i ~ 0 relative to sum |m_i a_i|
    f = pos[:, 3:4].astype(np.float64) * got[:, :3].astype(np.float64)
    assert np.abs(f.sum(0)).max() <= 1e-5 * np.abs(f).sum(0).max()


def test_step_matches_oracle(E, oracle_mod):
    import torch
    n = 777
    pos, vel = W.nbody_bodies(n, seed=9)
    vel[:, :3] = np.random.default_rng(2).uniform(-1, 1, (n, 3)).astype(np.float32)
    dt = 0.005
    xp, xv = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    op, ov = torch.zeros_like(xp), torch.zeros_like(xv)
    eng = E.Engine(0)
    p = E.Program("nbody").in_(xp).in_(xv).out(op).out(ov).args(xp, xv, n, dt, EPS2, op, ov)
    eng.work_items(gws_of(n, 64), 64).scheduler("dynamic", (10,)).program(p).run().synchronize()
    rp, rv = oracle_mod.nbody_step(pos, vel, dt, EPS2)
    c = cond(pos, np.arange(n))[:, None]
    gp, gv = op.cpu().numpy().astype(np.float64), ov.cpu().numpy().astype(np.float64)
    assert (np.abs(gv[:, :3] - rv[:, :3]) <= RTOL * (np.abs(vel[:, :3]) + c * dt) + 1e-7).all()
    assert (np.abs(gp[:, :3] - rp[:, :3]) <= RTOL * (np.abs(pos[:, :3]) + np.abs(vel[:, :3]) * dt + c * dt * dt)
            + 1e-7).all()
    assert np.array_equal(gp[:, 3], pos[:, 3]) and np.array_equal(gv[:, 3], vel[:, 3])
    eng.close()


def run_energy(E, pos, sched="hguided", params=(2.0, 1.0), D=0, C=0, lws=64):
    import torch
    n = pos.shape[0]
    x = torch.from_numpy(pos).cuda()
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    eng = E.Engine(0)
    p = E.Program("nbody_energy").in_(x).out(e).args(x, n, EPS2, e)
    eng.work_items(gws_of(n, lws), lws).scheduler(sched, params).workers(D, C).program(p)
    eng.run().synchronize()
    v1 = float(e.item())
    eng.run().synchronize()  # the workspace counter must have reset itself
    v2 = float(e.item())
    eng.close()
    assert v1 == v2
    return v1


@pytest.mark.parametrize("n", [2, 3, 65, 1000, 4096])
def test_energy_small(E, oracle_mod, n):
    pos, _ = W.nbody_bodies(n, seed=300 + n)
    ref = oracle_mod.nbody_energy(pos, EPS2)
    got = run_energy(E, pos)
    assert math.isclose(got, ref, rel_tol=RTOL)


def test_energy_schedule_independent_and_full_size(E, oracle_mod):
    pos, _ = W.nbody_bodies(65536)
    ref = oracle_mod.nbody_energy(pos, EPS2)
    a = run_energy(E, pos, "hguided", (2.0, 1.0), 8, 0)
    b = run_energy(E, pos, "dynamic", (37,), 0, 0)
    c = run_energy(E, pos, "monolithic", ())
    assert a == b == c  # fixed-order FP64 sums: bit-identical under any schedule
    assert math.isclose(a, ref, rel_tol=RTOL), (a, ref)


def test_adjoint_matches_oracle_gradient(E, oracle_mod):
    import torch
    n = 2000
    pos, _ = W.nbody_bodies(n, seed=17)
    x = torch.from_numpy(pos).cuda()
    g = torch.tensor([0.75], device="cuda")
    out = torch.zeros((n, 4), device="cuda")
    eng = E.Engine(0)
    p = E.Program("nbody_adjoint").in_(x).in_(g).out(out).args(x, n, EPS2, g, out)
    eng.work_items(gws_of(n, 64), 64).scheduler("hguided", (2.0, 1.0)).program(p).run().synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = 0.75 * oracle_mod.nbody_energy_grad(pos, EPS2)
    m = pos[:, 3].astype(np.float64)
    c = 0.75 * m * cond(pos, np.arange(n))
    assert (np.abs(got[:, :3] - ref).max(1) / c).max() <= RTOL
    phi = oracle_mod.nbody_potential(pos, EPS2)
    assert np.allclose(got[:, 3], -0.75 * phi, rtol=RTOL, atol=0)
    eng.close()


def test_fd_kernel_matches_oracle_and_adjoint(E, oracle_mod):
    import torch
    n = 4096
    pos, _ = W.nbody_bodies(n, seed=19)
    rng = np.random.default_rng(4)
    body = rng.choice(n, 64, replace=False).astype(np.int32)
    comp = rng.integers(0, 3, 64).astype(np.int32)
    h = 1e-3
    x = torch.from_numpy(pos).cuda()
    tb, tc = torch.from_numpy(body).cuda(), torch.from_numpy(comp).cuda()
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    eng = E.Engine(0)
    p = E.Program("nbody_fd").in_(x).in_(tb).in_(tc).out(out).args(x, n, EPS2, h, tb, tc, 64, out)
    eng.work_items(64, 1).scheduler("dynamic", (16,)).program(p).run().synchronize()
    got = out.cpu().numpy()
    ref = oracle_mod.nbody_fd_energy_grad(pos, EPS2, body, comp, h)
    # FP32 pair terms t_j = m_j / sqrt(|q - r_j|^2 + eps2) in FP64 sums: each
    # term carries a few units of 2^-24 of relative rounding (differences,
    # squares, the approximate rsqrt, the product), independent from term to
    # term, so the two rows' difference errs like a random walk of scale
    # 2^-23 sqrt(sum_j t+_j^2 + t-_j^2).  Bound: 16 of those units, times m_i,
    # over the FP32 distance x+ - x- (an FP32 emulation with a 2-ulp rsqrt
    # peaks at 7.5 units over 192 samples); no relative term.
    p64 = pos.astype(np.float64)
    tol = np.empty(64)
    for t, (b, c) in enumerate(zip(body, comp)):
        xp = float(np.float32(pos[b, c] + np.float32(h)))
        xm = float(np.float32(pos[b, c] - np.float32(h)))
        ss = 0.0
        for x in (xp, xm):
            q = p64[b, :3].copy()
            q[c] = x
            d = p64[:, :3] - q
            tt = p64[:, 3] / np.sqrt((d * d).sum(1) + np.float32(EPS2))
            tt[b] = 0.0
            ss += (tt * tt).sum()
        tol[t] = 16 * 2.0 ** -23 * p64[b, 3] * np.sqrt(ss) / (xp - xm)
    err = np.abs(got - ref)
    assert (err <= tol).all(), (err / tol).max()
    # against the analytic gradient (FD truncation O(h^2) dominates near close pairs)
    grad = oracle_mod.nbody_energy_grad(pos, EPS2)
    gi = np.array([grad[b, c] for b, c in zip(body, comp)])
    near = np.array([np.sort(np.linalg.norm(p64[:, :3] - p64[b, :3], axis=1))[1] for b in body])
    far = near > 10 * h
    assert far.sum() > 32
    assert (np.abs(got[far] - gi[far]) <= 1e-2 * np.abs(gi[far]) + 1e-3 * n).all()
    eng.close()
