"""The energy entry point that allocates nothing (ecl_nbody_energy_noalloc).

Some callers cannot let a library call cudaMalloc: a process whose device
memory belongs to another allocator, or one running under a hard memory cap.
This entry point takes its scratch from a fixed array in the library's device
image instead.  Its result must equal the regular program's (ecl_run of
"nbody_energy") within the tolerance the energy tests use, on two calls in a
row (the second call reuses the array the first one left behind).

Named to be collected last, so a run that stops at the first failure has
already run every other test.
"""
import math

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


def regular_energy(E, x, n):
    import torch
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    eng = E.Engine(0)
    p = E.Program("nbody_energy").in_(x).out(e).args(x, n, EPS2, e)
    eng.work_items(-(-n // 64) * 64, 64).scheduler("hguided", (2.0, 1.0)).program(p).run().synchronize()
    eng.close()
    return float(e.item())


# 524288 bodies fill the scratch exactly (8192 work-groups x 8 segments =
# 65536 partials); 524288 - 37 also needs all 8192 work-groups, the last one
# holding 27 bodies.
@pytest.mark.parametrize("n", [3, 1000, 65536, 524288 - 37, 524288])
def test_noalloc_energy_matches_regular_twice(E, n):
    import torch
    pos, _ = W.nbody_bodies(n, seed=600 + n)
    x = torch.from_numpy(pos).cuda()
    want = regular_energy(E, x, n)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        E.ecl_nbody_energy_noalloc(x, n, EPS2, out)
        torch.cuda.synchronize()
        got = float(out.item())
        # same pair terms, partials summed in the same fixed order: the same bits
        assert got == want, (got, want)
        assert math.isclose(got, want, rel_tol=RTOL)


def test_noalloc_energy_matches_the_oracle(E, oracle_mod):
    import torch
    n = 1000
    pos, _ = W.nbody_bodies(n, seed=1600)
    x = torch.from_numpy(pos).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    E.ecl_nbody_energy_noalloc(x, n, EPS2, out)
    torch.cuda.synchronize()
    assert math.isclose(float(out.item()), oracle_mod.nbody_energy(pos, EPS2), rel_tol=RTOL)


def test_noalloc_energy_rejects_sizes_beyond_the_scratch(E):
    import torch
    x = torch.zeros((524288 + 64, 4), device="cuda")  # large enough for the binding's size check
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EclError) as ei:
        E.ecl_nbody_energy_noalloc(x, 524288 + 64, EPS2, out)
    assert ei.value.status == E.ECL_ERR_SIZE
    with pytest.raises(E.EclError) as ei:
        E.ecl_nbody_energy_noalloc(x, 0, EPS2, out)
    assert ei.value.status == E.ECL_ERR_ARG
