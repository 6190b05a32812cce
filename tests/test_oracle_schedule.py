"""Pins of the scheduler oracle (Sec. 5.3 rules) and of the library's host planner.

The oracle is pinned by hand-derived package sequences (each derivation is
written next to its case) and by exhaustive coverage checks on tiny ranges.
The library's planner (``ecl_plan``, pure host code) must then reproduce the
oracle exactly.
"""
import itertools
import math
import random

import pytest

from oracle import schedule as S


# ---------------------------------------------------------------- hand cases
def test_static_listing2_proportions():
    # Listing 2: 512000 bodies, lws 64 -> G = 8000 work-groups, props {0.08, 0.3}
    # for CPU, Phi, GPU: 0.08*8000 = 640, 0.3*8000 = 2400, the GPU the rest 4960.
    assert S.static(8000, 3, [0.08, 0.3]) == [(0, 640), (640, 2400), (3040, 4960)]
    # Static rev lays the same sizes out GPU first (Sec. 7.3).
    assert S.static(8000, 3, [0.08, 0.3], reverse=True) == [(7360, 640), (4960, 2400), (0, 4960)]


def test_static_equal_split_remainder_to_last():
    assert S.static(10, 3) == [(0, 3), (3, 3), (6, 4)]
    assert S.static(2, 4) == [(0, 0), (0, 0), (0, 0), (0, 2)]


def test_static_rejects_bad_props():
    with pytest.raises(ValueError):
        S.static(10, 3, [0.7, 0.5])
    with pytest.raises(ValueError):
        S.static(10, 3, [-0.1, 0.5])
    with pytest.raises(ValueError):
        S.static(10, 3, [0.5])


def test_dynamic_short_last_package():
    # ceil(10/4) = 3 work-groups per package -> 3, 3, 3, 1 (only 4 packages)
    assert S.dynamic(10, 4) == [(0, 3), (3, 3), (6, 3), (9, 1)]
    # ceil(10/6) = 2 -> five packages although six were asked for
    assert S.dynamic(10, 6) == [(0, 2), (2, 2), (4, 2), (6, 2), (8, 2)]
    # the Gaussian configuration: 8192 rows of 64 work-groups (lws 128), 256 packages of 32 rows
    pk = S.dynamic(8192 * 64, 256)
    assert len(pk) == 256 and all(ln == 32 * 64 for _, ln in pk)


def test_hguided_homogeneous_hand_sequence():
    # G = 40, n = 2, k = 1, equal powers: size = floor(G_r * 1 / (1 * 2 * 2)) = floor(G_r / 4)
    # 40->10, 30->7, 23->5, 18->4, 14->3, 11->2, 9->2, 7->1, then the minimum 1 until done.
    seq = [ln for _, _, ln in S.hguided(40, 2, k=1.0)]
    assert seq == [10, 7, 5, 4, 3, 2, 2, 1, 1, 1, 1, 1, 1, 1]


def test_hguided_heterogeneous_hand_sequence():
    # G = 100, powers (1, 3), k = 1, n = 2, sum P = 4, min_base 2 -> minimums (2, 6).
    # Requests alternate device 1, 0, 1, 0, ...:
    #  d1: floor(100*3/8)=37 | d0: floor(63/8)=7 | d1: floor(56*3/8)=21 | d0: floor(35/8)=4
    #  d1: floor(31*3/8)=11 | d0: floor(20/8)=2 | d1: floor(18*3/8)=6 | d0: floor(12/8)=1->2
    #  d1: floor(10*3/8)=3->6 | d0: 0->2 | d1: 0->6, clipped to the 2 left
    order = [1, 0] * 6
    got = [(d, ln) for d, _, ln in S.hguided(100, 2, k=1.0, min_base=2, powers=[1.0, 3.0],
                                              request_order=order)]
    assert got == [(1, 37), (0, 7), (1, 21), (0, 4), (1, 11), (0, 2), (1, 6), (0, 2), (1, 6),
                   (0, 2), (1, 2)]


def test_grain_units_and_ragged_tail():
    # G = 10 work-groups in units of 4 -> 3 units (4, 4, 2 work-groups)
    assert S.units_of(10, 4) == 3
    assert S.dynamic(10, 2, grain=4) == [(0, 8), (8, 2)]
    assert S.static(10, 2, grain=4) == [(0, 4), (4, 6)]


def test_hguided_min_sizes_grow_with_power():
    assert S.hguided_min(4, [1.0, 2.0, 0.5]) == [8, 16, 4]


# ---------------------------------------------------------------- exhaustive
def _all_plans(G, D, grain):
    yield S.static(G, D, grain=grain)
    yield S.static(G, D, grain=grain, reverse=True)
    if D >= 2:
        yield S.static(G, D, [0.25] * (D - 1), grain=grain)
    for pk in (1, 2, 3, 7):
        yield S.dynamic(G, pk, grain=grain)
    for k in (0.5, 1.0, 2.0, 3.0):
        for mb in (1, 2):
            yield [(o, l) for _, o, l in S.hguided(G, D, k=k, min_base=mb, grain=grain)]
    yield [(o, l) for _, o, l in S.hguided(G, D, k=2.0, powers=[1.0 + d for d in range(D)], grain=grain)]


@pytest.mark.parametrize("G", list(range(0, 65)))
def test_every_work_group_exactly_once(G):
    for D, grain in itertools.product((1, 2, 3, 5), (1, 2, 3)):
        for plan in _all_plans(G, D, grain):
            assert S.coverage(G, plan) == [1] * G, (G, D, grain, plan)
            # packages are contiguous and in offset order for queue plans
            assert sum(ln for _, ln in plan) == G


def test_homogeneous_hguided_sizes_never_grow():
    for G in (1, 17, 100, 1000, 65536):
        for D in (1, 3, 8, 152):
            for k in (0.5, 1, 2, 4):
                s = [ln for _, _, ln in S.hguided(G, D, k=k)]
                assert all(a >= b for a, b in zip(s, s[1:]))


def test_dynamic_package_count_closed_form():
    for U in range(1, 200):
        for pk in range(1, 40):
            n = len(S.dynamic(U, pk))
            assert n == math.ceil(U / math.ceil(U / pk))


# ---------------------------------------------------------------- library planner
@pytest.fixture(scope="module")
def ecl():
    import paper_1805_02755_gb300 as E
    from paper_1805_02755_gb300 import build as B
    B.build()
    return E


def _lib_plan(E, kind, params, G, grain, D):
    off, ln, dev = E.ecl_plan(kind, params, G, grain, D)
    return [(int(o), int(l)) for o, l in zip(off, ln)], [int(d) for d in dev]


def test_library_planner_matches_oracle(ecl):
    rnd = random.Random(1805)
    for _ in range(300):
        G = rnd.choice([1, 2, 7, 64, 100, 1000, 8000, 65536, 1 << 20])
        D = rnd.choice([1, 2, 3, 4, 8, 152, 1216])
        grain = rnd.choice([1, 1, 1, 4, 32])
        kind = rnd.choice(["static", "static_rev", "dynamic", "hguided"])
        if kind in ("static", "static_rev"):
            props = [] if rnd.random() < 0.5 or D == 1 else [0.5 / D] * (D - 1)
            got, dev = _lib_plan(ecl, kind, props, G, grain, D)
            want = S.static(G, D, props or None, reverse=(kind == "static_rev"), grain=grain)
            assert got == want
            assert dev == list(range(D))
        elif kind == "dynamic":
            npk = rnd.choice([1, 3, 50, 150, 256])
            got, _ = _lib_plan(ecl, kind, [npk], G, grain, D)
            assert got == S.dynamic(G, npk, grain=grain)
        else:
            k = rnd.choice([0.5, 1.0, 2.0, 3.0, 0.25])
            mb = rnd.choice([1, 2, 5])
            got, _ = _lib_plan(ecl, kind, [k, mb], G, grain, D)
            assert got == [(o, l) for _, o, l in S.hguided(G, D, k=k, min_base=mb, grain=grain)]


def test_library_planner_heterogeneous_matches_oracle(ecl):
    powers = [1.0, 3.0]
    got, dev = _lib_plan(ecl, "hguided", [1.0, 2.0] + powers, 100, 1, 2)
    want = S.hguided(100, 2, k=1.0, min_base=2, powers=powers)  # cyclic 0, 1, 0, ...
    assert list(zip(dev, got)) == [(d, (o, l)) for d, o, l in want]


def test_library_planner_rejects_bad_params(ecl):
    for kind, params, D in [("static", [0.7, 0.5], 3), ("static", [0.5], 4), ("dynamic", [0], 2),
                            ("dynamic", [2.5], 2), ("hguided", [0.0, 1], 2), ("hguided", [2, 0], 2),
                            ("hguided", [2, 1, 1.0], 2), ("hguided", [2, 1, 1.0, -1.0], 2)]:
        with pytest.raises(ecl.EclError) as ei:
            ecl.ecl_plan(kind, params, 100, 1, D)
        assert ei.value.status == ecl.ECL_ERR_SCHED
