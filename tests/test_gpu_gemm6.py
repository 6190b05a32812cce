"""Six-product split-BF16 GEMM ("gemm_split6") through the C ABI vs the FP64 oracle.

Against the exact value of the six-product expansion (oracle mode 3) the only
error is accumulation: FP32 round-to-nearest additions of the per-chunk hh
sums plus the tensor core's accumulation inside a chunk.  Against the FP64
product of the FP32 inputs (mode 1) the dropped products add at most 2^-23 of
(|A||B|)_ij; the stated target is 1e-6 normwise.
"""
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


def tiles(M, N):
    return -(-M // 128) * -(-N // 128)


def run_gemm6(E, A, Bt, chunk_k=0, sched="hguided", params=(2.0, 1.0), D=0, C=0, coverage=False):
    import torch
    M, K = A.shape
    N = Bt.shape[0]
    a = torch.from_numpy(A).cuda()
    b = torch.from_numpy(Bt).cuda()
    c = torch.full((M * N + 64,), -3.0, device="cuda")
    eng = E.Engine(0)
    G = tiles(M, N)
    cov = torch.zeros(G, dtype=torch.int32, device="cuda") if coverage else None
    p = E.Program("gemm_split6").in_(a).in_(b).out(c).args(a, b, c, M, N, K, chunk_k)
    eng.work_items(G * 16384, 16384).scheduler(sched, params).workers(D, C).program(p)
    eng.set_coverage(cov)
    eng.run().synchronize()
    out = c.cpu().numpy()
    assert (out[M * N:] == -3.0).all(), "wrote past C"
    eng.close()
    return out[: M * N].reshape(M, N), cov


def absab(A, Bt):
    return np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T


# (300, 2000, 1000): 16 tile columns in column groups of 12 and 4 with 152 CTAs
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 300, 136), (1, 1, 8), (129, 257, 1000), (256, 384, 2048),
                                   (300, 2000, 1000)])
def test_split6_shapes(E, oracle_mod, M, N, K):
    A, Bt = W.gemm_matrices(M, N, K, seed=900 + M + N + K)
    got, _ = run_gemm6(E, A, Bt)
    exact6 = oracle_mod.gemm(A, Bt, 3)
    full = oracle_mod.gemm(A, Bt, 1)
    aa = absab(A, Bt)
    assert (np.abs(got - exact6) <= 2e-7 * aa + 1e-30).all(), np.max(np.abs(got - exact6) / aa)
    assert np.linalg.norm(got - full) <= 1e-6 * np.linalg.norm(full)


@pytest.mark.parametrize("chunk_k", [1, 2, 4])
def test_split6_chunk_lengths(E, oracle_mod, chunk_k):
    A, Bt = W.gemm_matrices(256, 256, 1536, seed=950)
    got, _ = run_gemm6(E, A, Bt, chunk_k=chunk_k)
    exact6 = oracle_mod.gemm(A, Bt, 3)
    aa = absab(A, Bt)
    assert (np.abs(got - exact6) <= 2e-7 * aa).all()


def test_split6_promotion_matters(E, oracle_mod):
    # one chunk over the whole K (no promotion) leaves the accumulation of the
    # large hh sums to the tensor core: several times the error of chunks of 64
    A, Bt = W.gemm_matrices(256, 256, 1536, seed=950)
    exact6 = oracle_mod.gemm(A, Bt, 3)
    e = {}
    for ck in (1, 1000):
        got, _ = run_gemm6(E, A, Bt, chunk_k=ck)
        e[ck] = np.linalg.norm(got - exact6) / np.linalg.norm(exact6)
    print("split6 normwise error vs its exact value: chunk 64: %.3e, whole K: %.3e" % (e[1], e[1000]))
    assert e[1000] > 3 * e[1], e


@pytest.mark.parametrize("sched,params,D,C", [("static", (), 1, 0), ("dynamic", (3,), 2, 0),
                                              ("hguided", (2.0, 1.0), 4, 0), ("monolithic", (), 0, 0)])
def test_split6_schedulers(E, oracle_mod, sched, params, D, C):
    A, Bt = W.gemm_matrices(640, 384, 256, seed=960)
    got, cov = run_gemm6(E, A, Bt, 0, sched, params, D, C, coverage=(sched != "monolithic"))
    exact6 = oracle_mod.gemm(A, Bt, 3)
    assert (np.abs(got - exact6) <= 2e-7 * absab(A, Bt)).all()
    if cov is not None:
        assert (cov.cpu().numpy() == 1).all()


def test_split6_full_size_sampled(E, oracle_mod):
    M = N = K = 8192
    A, Bt = W.gemm_matrices(M, N, K)
    rng = np.random.default_rng(4)
    ii = rng.integers(0, M, 512)
    jj = rng.integers(0, N, 512)
    got, _ = run_gemm6(E, A, Bt, 0, "hguided", (2.0, 1.0), 4, 0)
    g = got[ii, jj].astype(np.float64)
    del got
    ref1 = oracle_mod.gemm_entries(A, Bt, 1, ii, jj)
    ref6 = oracle_mod.gemm_entries(A, Bt, 3, ii, jj)
    aa = np.array([np.abs(A[i].astype(np.float64)) @ np.abs(Bt[j].astype(np.float64)) for i, j in zip(ii, jj)])
    assert (np.abs(g - ref6) <= 2e-7 * aa).all()
    rel = np.linalg.norm(g - ref1) / np.linalg.norm(ref1)
    print("split6 normwise error vs FP64 of FP32 inputs at 8192^3: %.3e" % rel)
    assert rel <= 1e-6, rel
