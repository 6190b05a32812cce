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
    # Central differences of the GPU prices against the oracle's at the same
    # FP32 bumps, and against the GPU's own delta and vega, option by option.
    K, T, N = (o[k].astype(np.float64) for k in ("K", "T", "steps"))
    sg = o["sigma"].astype(np.float64)

    def gpu_price(Sv, sigv):
        with torch.no_grad():
            return A.binomial_price(torch.from_numpy(Sv).cuda(), t["K"], t["T"], torch.from_numpy(sigv).cuda(),
                                    t["steps"], o["r"]).cpu().numpy().astype(np.float64)

    def kinks(Slo, Shi, siglo, sighi):
        # options with a leaf whose payoff S u^j d^(N-j) - K changes sign
        # between the two bumped inputs (the lattice price has a kink there)
        out = np.zeros(len(K), bool)
        for i in range(len(K)):
            m = 2.0 * np.arange(N[i] + 1) - N[i]
            sdt = np.sqrt(T[i] / N[i])
            a = Slo[i] * np.exp(siglo[i] * sdt * m) - K[i]
            b = Shi[i] * np.exp(sighi[i] * sdt * m) - K[i]
            out[i] = ((a * b <= 0) | (np.minimum(np.abs(a), np.abs(b)) <= 1e-6 * K[i])).any()
        return out

    def fd_pair(Sp, Sm, sigp, sigm, x_p, x_m):
        up, dn = gpu_price(Sp, sigp), gpu_price(Sm, sigm)
        rup = oracle_mod.binomial(Sp, o["K"], o["T"], sigp, o["steps"], o["r"])[0]
        rdn = oracle_mod.binomial(Sm, o["K"], o["T"], sigm, o["steps"], o["r"])[0]
        dx = x_p.astype(np.float64) - x_m.astype(np.float64)
        # each GPU price is within 1e-5 max(V, 1e-4 S) of the oracle's
        noise = 1e-5 * (np.maximum(rup, 1e-4 * Sp) + np.maximum(rdn, 1e-4 * Sm)) / dx
        return (up - dn) / dx, (rup - rdn) / dx, noise

    Sf = o["S"]
    # delta: S bumped by 0.1%.  Without a kink in [S-, S+] the lattice price is
    # linear in S, so the oracle quotient equals the oracle delta; with one,
    # the quotient is delta averaged over the bump and the oracle measures
    # the gap.
    Sp = (Sf + np.float32(1e-3) * Sf).astype(np.float32)
    Sm = (Sf - np.float32(1e-3) * Sf).astype(np.float32)
    fd, fd_ref, noise = fd_pair(Sp, Sm, o["sigma"], o["sigma"], Sp, Sm)
    assert (np.abs(fd - fd_ref) <= noise).all(), (np.abs(fd - fd_ref) / noise).max()
    kd = kinks(Sm.astype(np.float64), Sp.astype(np.float64), sg, sg)
    assert (~kd).sum() >= 64
    assert np.allclose(fd_ref[~kd], rd[~kd], rtol=1e-9, atol=1e-12)
    dg = S.grad.cpu().numpy().astype(np.float64) / wn
    gap = np.where(kd, np.abs(rd - fd_ref), 0.0)
    assert (np.abs(dg - fd) <= gap + noise + 1e-5 * np.maximum(np.abs(rd), 1e-4)).all()
    # vega: sigma bumped by 1e-3 (FP32-representable bumps); the price is
    # smooth in sigma between kinks, and the oracle's own quotient gives the
    # truncation gap |vega - quotient| of this lattice at these bumps
    sp = (o["sigma"] + np.float32(1e-3)).astype(np.float32)
    sm = (o["sigma"] - np.float32(1e-3)).astype(np.float32)
    fdv, fdv_ref, noisev = fd_pair(o["S"], o["S"], sp, sm, sp, sm)
    assert (np.abs(fdv - fdv_ref) <= noisev).all(), (np.abs(fdv - fdv_ref) / noisev).max()
    vg = sig.grad.cpu().numpy().astype(np.float64) / wn
    gapv = np.abs(rv - fdv_ref)
    assert (np.abs(vg - fdv) <= gapv + noisev + 1e-5 * np.maximum(np.abs(rv), 1e-4 * Sn)).all()
    kv = kinks(Sn, Sn, sm.astype(np.float64), sp.astype(np.float64))
    # away from kinks the central quotient's truncation is O(h^2): small
    assert (~kv).sum() >= 64 and (gapv[~kv] <= 1e-3 * np.maximum(np.abs(rv[~kv]), 1e-4 * Sn[~kv])).all()


def test_no_grad_path_skips_greeks(A):
    import torch
    o = W.binomial_options(64, seed=702)
    t = {k: torch.from_numpy(np.ascontiguousarray(o[k])).cuda() for k in ("S", "K", "T", "sigma", "steps")}
    p = A.binomial_price(t["S"], t["K"], t["T"], t["sigma"], t["steps"], o["r"])
    assert not p.requires_grad and p.shape == (64,)
