"""autograd wrappers: backward passes are the adjoint kernels; checked against
the oracle gradient and against finite differences."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
EPS2 = 1e-3


@pytest.fixture(scope="module")
def A():
    import torch
    assert torch.cuda.is_available()
    from paper_1805_02755_gb300 import build as B
    B.build()
    from paper_1805_02755_gb300 import autograd as A
    return A


def cond(pos, eps2=EPS2):
    p = pos.astype(np.float64)
    out = np.zeros(len(p))
    for i in range(len(p)):
        d = p[:, :3] - p[i, :3]
        r2 = (d * d).sum(1)
        out[i] = (p[:, 3] * np.sqrt(r2) / (r2 + eps2) ** 1.5).sum()
    return out


def test_nbody_energy_backward_matches_oracle_and_fd(A, oracle_mod):
    import torch
    n = 3000
    pos, _ = W.nbody_bodies(n, seed=700)
    x = torch.from_numpy(pos).cuda().requires_grad_(True)
    E = A.nbody_energy(x, EPS2)
    assert abs(E.item() - oracle_mod.nbody_energy(pos, EPS2)) <= 1e-5 * abs(E.item())
    (2.5 * E).backward()
    g = x.grad.cpu().numpy().astype(np.float64)
    ref = 2.5 * oracle_mod.nbody_energy_grad(pos, EPS2)
    m = pos[:, 3].astype(np.float64)
    assert (np.abs(g[:, :3] - ref).max(1) / (2.5 * m * cond(pos))).max() <= 1e-5
    assert np.allclose(g[:, 3], -2.5 * oracle_mod.nbody_potential(pos, EPS2), rtol=1e-5, atol=0)
    # central finite differences of the oracle energy (FP64), h = 1e-3
    rng = np.random.default_rng(7)
    idx = rng.choice(n, 24, replace=False)
    comp = rng.integers(0, 3, 24)
    fd = 2.5 * oracle_mod.nbody_fd_energy_grad(pos, EPS2, idx, comp, 1e-3)
    got = np.array([g[i, c] for i, c in zip(idx, comp)])
    p64 = pos.astype(np.float64)
    near = np.array([np.sort(np.linalg.norm(p64[:, :3] - p64[i, :3], axis=1))[1] for i in idx])
    far = near > 1e-2
    assert far.sum() >= 12
    assert (np.abs(got[far] - fd[far]) <= 1e-2 * np.abs(fd[far]) + 1e-3 * n).all()


def test_binomial_backward_matches_oracle_and_fd(A, oracle_mod):
    import torch
    o = W.binomial_options(256, seed=701, min_steps=64, max_steps=1024)
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    S = t["S"].clone().requires_grad_(True)
    sig = t["sigma"].clone().requires_grad_(True)
    w = torch.linspace(0.5, 1.5, 256, device="cuda")
    price = A.binomial_price(S, t["K"], t["T"], sig, t["steps"], o["r"])
    (w * price).sum().backward()
    rp, rd, rv = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    wn = w.cpu().numpy().astype(np.float64)
    Sn = o["S"].astype(np.float64)
    assert (np.abs(price.detach().cpu().numpy() - rp) <= 1e-5 * np.maximum(rp, 1e-4 * Sn)).all()
    assert (np.abs(S.grad.cpu().numpy() - wn * rd) <= 1e-5 * wn * np.maximum(np.abs(rd), 1e-4)).all()
    assert (np.abs(sig.grad.cpu().numpy() - wn * rv) <= 1e-5 * wn * np.maximum(np.abs(rv), 1e-4 * Sn)).all()
    # central differences of the GPU price (FP32) with a bump of 1% of S, against
    # the oracle's central differences (FP64) at the same bumped spots: each
    # price is within 1e-5 max(V, 1e-4 S), so the quotients agree to
    # 2e-5 max(V, 1e-4 S) / (2h) = 1e-3 max(V/S, 1e-4)
    with torch.no_grad():
        h = 0.01 * t["S"]
        sp, sm = t["S"] + h, t["S"] - h
        up = A.binomial_price(sp, t["K"], t["T"], t["sigma"], t["steps"], o["r"])
        dn = A.binomial_price(sm, t["K"], t["T"], t["sigma"], t["steps"], o["r"])
        fd = ((up - dn) / (sp - sm)).cpu().numpy()
    spn, smn = sp.cpu().numpy(), sm.cpu().numpy()
    rup = oracle_mod.binomial(spn, o["K"], o["T"], o["sigma"], o["steps"], o["r"])[0]
    rdn = oracle_mod.binomial(smn, o["K"], o["T"], o["sigma"], o["steps"], o["r"])[0]
    fd_ref = (rup - rdn) / (spn.astype(np.float64) - smn.astype(np.float64))
    assert (np.abs(fd - fd_ref) <= 1e-3 * np.maximum(rp / Sn, 1e-4) + 1e-6).all()
    # the lattice price is piecewise linear in S: the quotient is delta averaged over
    # [S - h, S + h], within gamma * h of delta at S
    assert np.median(np.abs(fd - rd)) < 1e-2


def test_no_grad_path_skips_greeks(A):
    import torch
    o = W.binomial_options(64, seed=702)
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    p = A.binomial_price(t["S"], t["K"], t["T"], t["sigma"], t["steps"], o["r"])
    assert not p.requires_grad and p.shape == (64,)
