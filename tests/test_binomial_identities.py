"""The identities the binomial kernel's greeks rest on, in FP64 on the CPU,
against the oracle's forward-mode (dual-number) greeks.

On the CRR lattice scaled by 2 per level, B' = (B_up + B) + 2q (B_up - B):
* delta and the leaf part of vega are the same recursion applied to the leaf
  derivatives, so one reverse pass suffices: weights A of the nodes of level
  N - 1 in the root, A = 1 at the root and A'_j = (A_j + A_{j-1}) +
  2q (A_{j-1} - A_j) outwards, dotted with the leaf derivatives pushed back
  one level;
* the q-dependence of every level adds up to N 2q' (B_1 - B_0) (the level
  operator and the difference operator commute), q' = dq/dsigma.
The test restates that arithmetic in numpy (plain loops, no kernel code) and
compares price, delta and vega with the oracle."""
import math

import numpy as np
import pytest

import workloads as W


def lattice_and_adjoint(S, K, T, sigma, N, r):
    S, K, T, sigma = float(S), float(K), float(T), float(sigma)
    dt = T / N
    sdt = math.sqrt(dt)
    a = sigma * sdt
    q = (math.expm1(r * dt) - 2.0 * math.sinh(0.5 * a) ** 2) / (2.0 * math.sinh(a))
    q2 = 2.0 * q
    m = 2.0 * np.arange(N + 1) - N
    g = np.exp(a * m)
    ST = S * g
    itm = ST > K
    x = np.where(itm, ST - K, 0.0)
    dl = np.where(itm, g, 0.0)          # dS_T/dS
    vg = np.where(itm, ST * m * sdt, 0.0)  # dS_T/dsigma

    def level(v):
        return (v[1:] + v[:-1]) + q2 * (v[1:] - v[:-1])

    B = x
    for _ in range(N - 1):
        B = level(B)               # down to level 1 (two nodes)
    d1 = B[1] - B[0]
    root = level(B)[0]
    A = np.array([1.0])
    for _ in range(N - 1):         # root outwards to level N - 1
        A2 = np.zeros(A.size + 1)
        A2[:-1] += (1.0 - q2) * A
        A2[1:] += (1.0 + q2) * A
        A = A2
    scale = math.exp(-r * T) * 2.0 ** (-N)
    q2p = 2.0 * sdt * (-0.5 - q * math.cosh(a) / math.sinh(a))  # 2 dq/dsigma
    price = root * scale
    delta = float(A @ level(dl)) * scale
    vega_leaf = float(A @ level(vg)) * scale
    vega_q = N * q2p * d1 * scale
    return price, delta, vega_leaf, vega_q


@pytest.mark.parametrize("lo,hi", [(1, 8), (20, 64), (150, 200)])
def test_adjoint_greeks_match_forward_mode(oracle_mod, lo, hi):
    o = W.binomial_options(24, seed=77 + lo, min_steps=lo, max_steps=hi)
    P, D, V = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    for i in range(24):
        p, d, vl, vq = lattice_and_adjoint(o["S"][i], o["K"][i], o["T"][i], o["sigma"][i], int(o["steps"][i]),
                                           o["r"])
        v = vl + vq
        s = float(o["S"][i])
        assert abs(p - P[i]) <= 1e-10 * max(abs(P[i]), 1e-4 * s)
        assert abs(d - D[i]) <= 1e-10 * max(abs(D[i]), 1e-4)
        assert abs(v - V[i]) <= 1e-9 * max(abs(V[i]), 1e-4 * s)


def test_the_q_term_is_needed(oracle_mod):
    """Without N 2q' (B_1 - B_0) the leaf part alone misses vega by far more
    than any tolerance: the term carries a large share of it."""
    o = W.binomial_options(16, seed=5, min_steps=40, max_steps=60)
    P, D, V = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    misses = []
    for i in range(16):
        _, _, vl, vq = lattice_and_adjoint(o["S"][i], o["K"][i], o["T"][i], o["sigma"][i], int(o["steps"][i]),
                                           o["r"])
        assert abs(vl + vq - V[i]) <= 1e-9 * max(abs(V[i]), 1e-4 * float(o["S"][i]))
        misses.append(abs(vl - V[i]) / max(abs(V[i]), 1e-4 * float(o["S"][i])))
    assert min(misses) > 1e-3


def test_closed_form_leaf_weights_give_the_oracle_delta_and_vega(oracle_mod):
    # The adjoint of N levels of B' = 2p shift(B) + 2(1-p) B is, at the leaves,
    # 2^N times the binomial probabilities C(N,j) p^j (1-p)^(N-j) (the paths
    # from leaf j to the root), so delta and the vega leaf part are
    # probability-weighted sums of the leaf derivatives.  Restated in numpy
    # in log space from math.lgamma, against the oracle's dual numbers; a
    # weight taken from the wrong end of the lattice (pmf(N - j)) fails.
    o = W.binomial_options(48, seed=77, min_steps=1, max_steps=2048)
    rp, rd, rv = oracle_mod.binomial(o["S"], o["K"], o["T"], o["sigma"], o["steps"], o["r"])
    r = o["r"]
    for k in range(48):
        S, K, T, sg = (float(o[x][k]) for x in ("S", "K", "T", "sigma"))
        N = int(o["steps"][k])
        dt = T / N
        sdt = math.sqrt(dt)
        a = sg * sdt
        q = (math.expm1(r * dt) - 2.0 * math.sinh(0.5 * a) ** 2) / (2.0 * math.sinh(a))
        p = 0.5 + q
        j = np.arange(N + 1)
        m = 2.0 * j - N
        g = np.exp(a * m)
        ST = S * g
        lpmf = np.array([math.lgamma(N + 1) - math.lgamma(i + 1) - math.lgamma(N - i + 1) for i in j])
        pmf = np.exp(lpmf + j * math.log(p) + (N - j) * math.log1p(-p))
        disc = math.exp(-r * T)
        put = S > K
        itm = (ST < K) if put else (ST > K)
        sgn = -1.0 if put else 1.0
        delta = disc * (pmf * np.where(itm, sgn * g, 0.0)).sum() + (1.0 if put else 0.0)
        # vega = leaf part + the q term (the lattice's dependence on sigma through p)
        qp = sdt * (-0.5 - q * math.cosh(a) / math.sinh(a))  # dq/dsigma
        dpmf = pmf * (j / p - (N - j) / (1.0 - p)) * qp
        pay = np.where(itm, sgn * (ST - K), 0.0)
        vega = disc * ((pmf * np.where(itm, sgn * ST * m * sdt, 0.0)).sum() + (dpmf * pay).sum())
        assert abs(delta - rd[k]) <= 1e-9 * max(abs(rd[k]), 1e-4), (k, delta, rd[k])
        assert abs(vega - rv[k]) <= 1e-9 * max(abs(rv[k]), 1e-4 * S), (k, vega, rv[k])
        wrong = disc * (pmf[::-1] * np.where(itm, sgn * g, 0.0)).sum() + (1.0 if put else 0.0)
        if abs(2 * q) > 1e-3:
            assert abs(wrong - rd[k]) > 1e-6 * max(abs(rd[k]), 1e-4)
