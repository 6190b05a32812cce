"""Pins of the CPU oracle's kernels against facts fixed outside the oracle.

Each case names what pins it: a hand-derived orbit, a closed form, an
identity of the mathematics, a library routine for a special case, or a
brute-force evaluation of a different formula.  A dropped term, a wrong
sign, a transposed operand or a swapped index in oracle.c fails at least one.
"""
import math

import numpy as np
import pytest

import workloads as W


# ================================================================ Mandelbrot
def _point(O, cx, cy, it=256):
    return int(O.mandelbrot(1, 1, cx, cy, 1.0, 1.0, it)[0, 0])


def test_mandelbrot_hand_orbits(oracle_mod):
    O = oracle_mod
    # c = 0.5: z = 0.5, 0.75, 1.0625, 1.62890625, 3.1533... (all exact in FP32);
    # the fifth value has |z|^2 > 4, so the count is 5.
    assert _point(O, 0.5, 0.0) == 5
    # c = 1: z = 1, 2 (|z|^2 = 4 is not > 4), 5 -> count 3
    assert _point(O, 1.0, 0.0) == 3
    # c = -2: z = -2, 2, 2, ... |z|^2 = 4 forever -> never escapes
    assert _point(O, -2.0, 0.0) == 256
    # c = i: 0, i, -1+i, -i, -1+i, ... periodic -> never escapes
    assert _point(O, 0.0, 1.0) == 256
    # corner of the configuration's view: |c|^2 = 6.25 > 4 after one step
    assert _point(O, -2.0, -1.5) == 1
    # max_iter 0 -> 0 for every pixel
    assert _point(O, 0.0, 0.0, it=0) == 0


def test_mandelbrot_config_view_structure(oracle_mod):
    r = W.mandelbrot_region()
    img = oracle_mod.mandelbrot(r["width"], r["height"], r["x0"], r["y0"], r["dx"], r["dy"], r["max_iter"])
    H, Wd = img.shape
    j = np.arange(H)[:, None]
    i = np.arange(Wd)[None, :]
    cx = -2.0 + i * 3.0 / 1024
    cy = -1.5 + j * 3.0 / 1024
    # interior of the main cardioid and the period-2 bulb, away from their boundary
    q = (cx - 0.25) ** 2 + cy ** 2
    card = q * (q + (cx - 0.25)) < 0.2 * cy ** 2
    bulb = (cx + 1.0) ** 2 + cy ** 2 < (1.0 / 16) * 0.8
    assert card.sum() > 10000 and bulb.sum() > 1000
    assert (img[card] == 256).all() and (img[bulb] == 256).all()
    # outside the radius-2 disc a pixel escapes after exactly one step
    far = cx ** 2 + cy ** 2 > 4.0 + 1e-9
    assert (img[far] == 1).all()
    # conjugate symmetry: row j and row 1024 - j are mirror images (cy exact in FP32)
    assert (img[1:513] == img[1023:511:-1]).all()
    # row 512 is the real axis: inside for c in [-2, 0.25], out beyond 0.25
    row = img[512]
    assert (row[cx[0] <= 0.25][:-1] == 256).all()
    assert (row[cx[0] > 0.26] < 256).all()


# ================================================================ Gaussian
def test_gaussian_weights_symmetric_normalised():
    w = W.gaussian_weights(31, 5.0).astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-6
    assert np.array_equal(w, w[::-1])
    assert np.argmax(w) == 15


def test_gaussian_constant_image_is_fixed(oracle_mod):
    w = W.gaussian_weights(31, 5.0)
    img = np.full((40, 50), 0.375, dtype=np.float32)
    out = oracle_mod.gaussian(img, w)
    assert np.allclose(out, 0.375 * w.astype(np.float64).sum() ** 2, rtol=0, atol=1e-15)


def test_gaussian_impulse_gives_outer_product(oracle_mod):
    w = W.gaussian_weights(31, 5.0)
    img = np.zeros((64, 64), dtype=np.float32)
    img[32, 40] = 1.0
    out = oracle_mod.gaussian(img, w)
    wd = w.astype(np.float64)
    want = np.zeros((64, 64))
    want[17:48, 25:56] = np.outer(wd[::-1], wd[::-1])
    assert np.allclose(out, want, rtol=0, atol=1e-17)


def test_gaussian_separable_equals_direct_2d(oracle_mod):
    rng = np.random.default_rng(5)
    for taps, (H, Wd) in [(31, (37, 53)), (5, (9, 7)), (1, (3, 4)), (63, (70, 20))]:
        w = rng.random(taps).astype(np.float32)
        img = rng.random((H, Wd), dtype=np.float32)
        assert np.allclose(oracle_mod.gaussian(img, w), oracle_mod.gaussian_direct(img, w), rtol=1e-13,
                           atol=0)


def test_gaussian_border_clamp_matches_padded_convolution(oracle_mod):
    # independent route: pad with edge replication, then a full 2-D correlation
    rng = np.random.default_rng(7)
    w = W.gaussian_weights(7, 1.5)
    img = rng.random((12, 10), dtype=np.float32)
    pad = np.pad(img.astype(np.float64), 3, mode="edge")
    k2 = np.outer(w.astype(np.float64), w.astype(np.float64))
    want = np.zeros(img.shape)
    for y in range(12):
        for x in range(10):
            want[y, x] = (pad[y:y + 7, x:x + 7] * k2).sum()
    assert np.allclose(oracle_mod.gaussian(img, w), want, rtol=1e-13, atol=0)


def test_gaussian_row_range(oracle_mod):
    rng = np.random.default_rng(9)
    w = W.gaussian_weights(31, 5.0)
    img = rng.random((50, 33), dtype=np.float32)
    full = oracle_mod.gaussian(img, w)
    part = oracle_mod.gaussian(img, w, rows=(10, 21))
    assert np.array_equal(part[10:21], full[10:21])
    assert not part[:10].any() and not part[21:].any()


# ================================================================ NBody
def _bodies(rows):
    return np.array(rows, dtype=np.float32)


def test_nbody_two_body_closed_form(oracle_mod):
    # m1 at the origin, m2 at (d,0,0): a_1 = m2 d / (d^2+eps2)^(3/2) along +x, a_2 opposite
    d, m1, m2, eps2 = 0.5, 1.25, 0.75, 1e-3
    pos = _bodies([[0, 0, 0, m1], [d, 0, 0, m2]])
    acc = oracle_mod.nbody_acc(pos, eps2)
    s = (d * d + eps2) ** 1.5
    assert np.allclose(acc[0], [m2 * d / s, 0, 0], rtol=1e-12)
    assert np.allclose(acc[1], [-m1 * d / s, 0, 0], rtol=1e-12)
    assert math.isclose(oracle_mod.nbody_energy(pos, eps2), -m1 * m2 / math.sqrt(d * d + eps2), rel_tol=1e-12)


def test_nbody_equilateral_triangle(oracle_mod):
    # three unit masses on a triangle of side L: each is pulled to the centroid with
    # magnitude 2 * L cos(30deg) / (L^2 + eps2)^(3/2) = sqrt(3) L / (L^2+eps2)^(3/2)
    L, eps2 = 1.0, 0.01
    h = math.sqrt(3) / 2
    pos = _bodies([[0, 0, 0, 1], [L, 0, 0, 1], [L / 2, h, 0, 1]])
    acc = oracle_mod.nbody_acc(pos, eps2)
    c = pos[:, :3].astype(np.float64).mean(0)
    mag = math.sqrt(3) * L / (L * L + eps2) ** 1.5
    for i in range(3):
        u = (c - pos[i, :3]) / np.linalg.norm(c - pos[i, :3])
        assert np.allclose(acc[i], mag * u, rtol=1e-6, atol=1e-12)
    assert math.isclose(oracle_mod.nbody_energy(pos, eps2), -3 / math.sqrt(L * L + eps2), rel_tol=1e-6)


def test_nbody_momentum_and_gradient_identity(oracle_mod):
    pos, _ = W.nbody_bodies(300, seed=11)
    eps2 = 1e-3
    acc = oracle_mod.nbody_acc(pos, eps2)
    m = pos[:, 3].astype(np.float64)
    f = m[:, None] * acc
    # Newton's third law: the total force vanishes
    assert np.abs(f.sum(0)).max() < 1e-12 * np.abs(f).sum()
    # the energy gradient, differentiated term by term, equals -m_i a_i
    g = oracle_mod.nbody_energy_grad(pos, eps2)
    assert np.allclose(g, -f, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_nbody_energy_brute_force_pair_matrix(oracle_mod):
    pos, _ = W.nbody_bodies(64, seed=12)
    p = pos.astype(np.float64)
    eps2 = 1e-3
    d2 = ((p[:, None, :3] - p[None, :, :3]) ** 2).sum(-1) + eps2
    mm = p[:, 3][:, None] * p[:, 3][None, :]
    iu = np.triu_indices(64, 1)
    want = -(mm[iu] / np.sqrt(d2[iu])).sum()
    assert math.isclose(oracle_mod.nbody_energy(pos, eps2), want, rel_tol=1e-13)


def test_nbody_energy_gradient_finite_difference(oracle_mod):
    pos, _ = W.nbody_bodies(200, seed=13)
    eps2 = 1e-3
    g = oracle_mod.nbody_energy_grad(pos, eps2)
    idx = [3, 50, 199, 7]
    comp = [0, 1, 2, 1]
    fd = oracle_mod.nbody_fd_energy_grad(pos, eps2, idx, comp, 1e-3)
    ref = np.array([g[i, c] for i, c in zip(idx, comp)])
    assert np.allclose(fd, ref, rtol=2e-3, atol=1e-3 * np.abs(g).max())


def test_nbody_potential_pins(oracle_mod):
    pos, _ = W.nbody_bodies(120, seed=15)
    eps2 = 1e-3
    phi = oracle_mod.nbody_potential(pos, eps2)
    m = pos[:, 3].astype(np.float64)
    E = oracle_mod.nbody_energy(pos, eps2)
    # every pair appears twice in sum_i m_i phi_i
    assert math.isclose((m * phi).sum(), -2.0 * E, rel_tol=1e-12)
    # dE/dm_i = -phi_i: E is linear in m_i, so a finite difference in the mass is exact
    i = 17
    q = pos.copy()
    q[i, 3] = np.float32(pos[i, 3] + np.float32(0.25))
    dm = float(q[i, 3]) - float(pos[i, 3])
    assert math.isclose((oracle_mod.nbody_energy(q, eps2) - E) / dm, -phi[i], rel_tol=1e-9)


def test_nbody_step_kinematics(oracle_mod):
    pos, vel = W.nbody_bodies(50, seed=14)
    vel[:, :3] = 0.1
    acc = oracle_mod.nbody_acc(pos, 1e-3)
    po, vo = oracle_mod.nbody_step(pos, vel, 0.005, 1e-3)
    dt = 0.005
    assert np.allclose(vo[:, :3], vel[:, :3] + acc * dt, rtol=1e-14)
    assert np.allclose(po[:, :3], pos[:, :3].astype(np.float64) + 0.1 * dt + 0.5 * acc * dt * dt, rtol=1e-14)
    assert np.array_equal(po[:, 3], pos[:, 3].astype(np.float64))


# ================================================================ Binomial
def _crr_sum(S, K, T, sig, N, r, put=False):
    """Closed form of the lattice: disc^N sum_j C(N,j) p^j (1-p)^(N-j) payoff_j."""
    dt = T / N
    u = math.exp(sig * math.sqrt(dt))
    d = 1 / u
    p = (math.exp(r * dt) - d) / (u - d)
    tot = 0.0
    for j in range(N + 1):
        ST = S * u ** j * d ** (N - j)
        pay = max(K - ST, 0.0) if put else max(ST - K, 0.0)
        tot += math.comb(N, j) * p ** j * (1 - p) ** (N - j) * pay
    return math.exp(-r * T) * tot


def _bs(S, K, T, sig, r):
    d1 = (math.log(S / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    Nf = lambda x: 0.5 * math.erfc(-x / math.sqrt(2))  # noqa: E731
    call = S * Nf(d1) - K * math.exp(-r * T) * Nf(d2)
    delta = Nf(d1)
    vega = S * math.exp(-0.5 * d1 * d1) / math.sqrt(2 * math.pi) * math.sqrt(T)
    return call, delta, vega


def test_binomial_matches_closed_form_sum(oracle_mod):
    cases = [(50.0, 55.0, 1.0, 0.3, 1), (50.0, 45.0, 0.5, 0.2, 2), (80.0, 80.0, 2.0, 0.5, 17),
             (12.0, 14.0, 0.25, 0.1, 64), (99.0, 80.0, 1.5, 0.45, 40)]
    S, K, T, sig, N = [np.array(c) for c in zip(*cases)]
    for put in (False, True):
        price, _, _ = oracle_mod.binomial(S, K, T, sig, N, 0.02, put=put)
        for t, c in enumerate(cases):
            want = _crr_sum(float(np.float32(c[0])), float(np.float32(c[1])), float(np.float32(c[2])),
                            float(np.float32(c[3])), c[4], 0.02, put)
            assert math.isclose(price[t], want, rel_tol=1e-11, abs_tol=1e-12), (c, put)


def test_binomial_put_call_parity(oracle_mod):
    # On the CRR lattice C - P = S - K e^{-rT} exactly (p u + (1-p) d = e^{r dt}).
    o = W.binomial_options(50, seed=21, min_steps=1, max_steps=400)
    c, _, _ = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    p, _, _ = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"], put=True)
    S = o["S"].astype(np.float64)
    K = o["K"].astype(np.float64)
    T = o["T"].astype(np.float64)
    assert np.allclose(c - p, S - K * np.exp(-o["r"] * T), rtol=0, atol=1e-10 * S.max())


def test_binomial_black_scholes_limit(oracle_mod):
    # |V_N - BS| = O(1/N): at N = 2048 the lattice is within a few 1e-3 S of Black-Scholes,
    # and the error shrinks roughly 4x from N=512 to N=2048 (averaged over odd/even N).
    S, K, T, sig, r = 50.0, 52.0, 1.0, 0.3, 0.02
    bs, bdelta, bvega = _bs(S, K, T, sig, r)
    errs = {}
    for N in (512, 513, 2048, 2049):
        pr, de, ve = oracle_mod.binomial(np.array([S]), np.array([K]), np.array([T]), np.array([sig]),
                                         np.array([N]), r)
        errs[N] = abs(pr[0] - bs)
        assert errs[N] < 2.0 * S / N
        assert abs(de[0] - bdelta) < 20.0 / N
        assert abs(ve[0] - bvega) < 0.02 * bvega
    assert (errs[2048] + errs[2049]) < 0.6 * (errs[512] + errs[513])


def test_binomial_tangents_match_finite_differences(oracle_mod):
    o = W.binomial_options(6, seed=22, min_steps=16, max_steps=300)
    S = o["S"].astype(np.float64)
    sig = o["sigma"].astype(np.float64)
    _, delta, vega = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    # the oracle reads FP32 inputs, so finite differences use FP32-representable bumps
    for t in range(6):
        one = lambda **kw: {k: np.array([v[t]]) for k, v in o.items() if k != "r"} | kw  # noqa: E731
        hS = np.float32(2.0 ** math.floor(math.log2(S[t] * 1e-3)))
        up = oracle_mod.binomial(**one(S=np.array([np.float32(S[t] + hS)])), r=o["r"])[0][0]
        dn = oracle_mod.binomial(**one(S=np.array([np.float32(S[t] - hS)])), r=o["r"])[0][0]
        # the price is piecewise linear in S between payoff kinks: central FD is exact
        # unless a leaf crosses the strike inside the bump
        assert math.isclose((up - dn) / (2 * hS), delta[t], rel_tol=2e-3, abs_tol=1e-6)
        hv = np.float32(2.0 ** -12)
        up = oracle_mod.binomial(**one(sigma=np.array([np.float32(sig[t] + hv)])), r=o["r"])[0][0]
        dn = oracle_mod.binomial(**one(sigma=np.array([np.float32(sig[t] - hv)])), r=o["r"])[0][0]
        assert math.isclose((up - dn) / (2 * hv), vega[t], rel_tol=2e-3, abs_tol=1e-4)


# ================================================================ GEMM
def test_bf16_rounding_definition(oracle_mod):
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -2.5, 0.0, -0.0,
                  3.0e38, 1e-40, np.inf, -np.inf], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5, 0.0, -0.0, 2.9937e38, 1e-40, np.inf,
                     -np.inf], dtype=np.float32)
    got = oracle_mod.bf16_round(x)
    assert got[0] == 1.0 and got[1] == 1.0  # tie to even
    assert got[2] == np.float32(1.0 + 2 ** -6)  # tie, odd neighbour below -> up
    assert got[3] == np.float32(1.0 + 2 ** -7)  # above the tie -> up
    assert got[4] == -2.5 and got[5] == 0.0 and np.signbit(got[6])
    assert np.isinf(got[9]) and np.isinf(got[10])
    assert np.isnan(oracle_mod.bf16_round(np.array([np.nan], dtype=np.float32)))[0]
    del want


def test_bf16_rounding_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32),
                        (rng.standard_normal(1000) * 1e30).astype(np.float32),
                        (rng.standard_normal(1000) * 1e-30).astype(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle_mod.bf16_round(x), ref)


def test_gemm_modes_brute_force(oracle_mod):
    A, Bt = W.gemm_matrices(24, 20, 40, seed=31)
    Ab = oracle_mod.bf16_round(A).astype(np.float64)
    Bb = oracle_mod.bf16_round(Bt).astype(np.float64)
    assert np.allclose(oracle_mod.gemm(A, Bt, 0), Ab @ Bb.T, rtol=1e-14, atol=1e-13)
    assert np.allclose(oracle_mod.gemm(A, Bt, 1), A.astype(np.float64) @ Bt.astype(np.float64).T,
                       rtol=1e-14, atol=1e-13)
    Al = oracle_mod.bf16_round((A - Ab.astype(np.float32)).astype(np.float32)).astype(np.float64)
    Bl = oracle_mod.bf16_round((Bt - Bb.astype(np.float32)).astype(np.float32)).astype(np.float64)
    assert np.allclose(oracle_mod.gemm(A, Bt, 2), Ab @ Bb.T + Ab @ Bl.T + Al @ Bb.T, rtol=1e-14, atol=1e-13)


def test_gemm_identity_and_permutation(oracle_mod):
    A, _ = W.gemm_matrices(16, 16, 16, seed=32)
    eye = np.eye(16, dtype=np.float32)
    assert np.array_equal(oracle_mod.gemm(A, eye, 0), oracle_mod.bf16_round(A).astype(np.float64))
    perm = np.eye(16, dtype=np.float32)[np.random.default_rng(1).permutation(16)]
    # C = A P^T with P stored as "Bt": columns of A permuted
    got = oracle_mod.gemm(A, perm, 1)
    assert np.array_equal(got, (A.astype(np.float64) @ perm.astype(np.float64).T))


def test_gemm_split3_error_model(oracle_mod):
    # the three-product split misses lo*lo and the residuals beyond two bf16 terms:
    # a relative error near 2^-16 normwise, far below plain BF16 (~2^-9).
    A, Bt = W.gemm_matrices(32, 32, 256, seed=33)
    exact = oracle_mod.gemm(A, Bt, 1)
    e0 = np.linalg.norm(oracle_mod.gemm(A, Bt, 0) - exact) / np.linalg.norm(exact)
    e2 = np.linalg.norm(oracle_mod.gemm(A, Bt, 2) - exact) / np.linalg.norm(exact)
    assert 1e-4 < e0 < 1e-2
    assert e2 < 2e-5


def test_gemm_split6_worked_value(oracle_mod):
    # x = 1 + 2^-10 + 2^-20 splits into h = 1, m = 2^-10, l = 2^-20 (each a bf16);
    # the six products give x^2 minus exactly the dropped 2ml + l^2 = 2^-29 + 2^-40
    x = np.array([[1.0 + 2 ** -10 + 2 ** -20]], dtype=np.float32)
    assert float(x[0, 0]) == 1.0 + 2 ** -10 + 2 ** -20
    c6 = oracle_mod.gemm(x, x, 3)[0, 0]
    c1 = oracle_mod.gemm(x, x, 1)[0, 0]
    assert c1 - c6 == 2.0 ** -29 + 2.0 ** -40
    assert c6 == 1.0 + 2.0 ** -9 + 2.0 ** -19 + 2.0 ** -20


def test_gemm_split6_split_is_exact(oracle_mod):
    # with Bt = [[1]] the six products reduce to h + m + l, which must equal x
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(4000), rng.standard_normal(1000) * 1e20,
                        rng.standard_normal(1000) * 1e-20]).astype(np.float32).reshape(-1, 1)
    one = np.ones((1, 1), dtype=np.float32)
    got = oracle_mod.gemm(x, one, 3)[:, 0]
    assert np.array_equal(got, x[:, 0].astype(np.float64))


def test_gemm_split6_bf16_inputs_are_exact(oracle_mod):
    # inputs that are already bf16 have m = l = 0: all modes give the same exact product
    A, Bt = W.gemm_matrices(12, 10, 24, seed=34)
    A = oracle_mod.bf16_round(A)
    Bt = oracle_mod.bf16_round(Bt)
    c1 = oracle_mod.gemm(A, Bt, 1)
    assert np.array_equal(oracle_mod.gemm(A, Bt, 3), c1)
    assert np.array_equal(oracle_mod.gemm(A, Bt, 0), c1)


def test_gemm_split6_error_bound(oracle_mod):
    # |m| <= 2^-8 |x| and |l| <= 2^-16 |x| (round to nearest twice), so the dropped
    # ml + lm + ll are at most 2^-23 |a||b| per term; far below the split-3 error
    A, Bt = W.gemm_matrices(32, 32, 256, seed=35)
    exact = oracle_mod.gemm(A, Bt, 1)
    c6 = oracle_mod.gemm(A, Bt, 3)
    absprod = np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T
    assert np.all(np.abs(c6 - exact) <= 2.0 ** -23 * absprod)
    e6 = np.linalg.norm(c6 - exact) / np.linalg.norm(exact)
    e2 = np.linalg.norm(oracle_mod.gemm(A, Bt, 2) - exact) / np.linalg.norm(exact)
    assert e6 < 1e-7 and e6 < e2 / 100
