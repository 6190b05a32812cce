"""Package sequences of the paper's three load-balancing schedulers (Sec. 5.3).

TEST INFRASTRUCTURE ONLY: the library never imports this module.

A scheduler cuts the NDRange of G work-groups into packages.  Sizes are
counted in *units* of ``grain`` consecutive work-groups (grain 1 for every
kernel except the row-tiled GEMM, whose unit is one full row of output
tiles); the last unit may be short when grain does not divide G.  A package
is returned as ``(offset_wg, length_wg)``.

Readings of the paper taken here:

* Static (Sec. 5.3 "Static"; Listing 2 gives n-1 proportions for n devices):
  device d < D-1 receives floor(props[d] * U) units, the product evaluated
  in IEEE double; the last device receives the rest.  Without proportions
  every device gets floor(U / D) and the last one the rest.  Offsets follow
  device order; "Static rev" (Sec. 7.3) keeps each device's size but lays
  the ranges out in reverse device order, so the last device's range starts
  at 0.
* Dynamic (Sec. 5.3 "Dynamic"): ``num_packages`` requested; every package
  has ceil(U / num_packages) units except a shorter last one, so fewer
  packages than requested can result (G=10, 4 packages -> 3,3,3,1).
* HGuided (Sec. 5.3, the packet-size equation):
  size_i = floor(G_r * P_i / (k * n * sum_j P_j)) units, evaluated in IEEE
  double in exactly that order ((G_r*P_i) / ((k*n)*sumP)), raised to the
  device's minimum package size and clipped to G_r; G_r (pending units)
  shrinks by every package handed out.  The minimum of device i is
  max(1, floor(min_base * P_i / min_j P_j + 0.5)); with equal powers every
  device's minimum is min_base.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

Package = Tuple[int, int]


def units_of(G: int, grain: int) -> int:
    """Number of scheduling units covering G work-groups."""
    if G < 0 or grain < 1:
        raise ValueError("G must be >= 0 and grain >= 1")
    return -(-G // grain)


def unit_range_to_wg(G: int, grain: int, u0: int, ulen: int) -> Package:
    """Convert a unit range to a work-group range, clipping the short tail."""
    off = min(G, u0 * grain)
    end = min(G, (u0 + ulen) * grain)
    return off, end - off


def static(G: int, devices: int, props: Optional[Sequence[float]] = None,
           reverse: bool = False, grain: int = 1) -> List[Package]:
    """One package per device, indexed by device (Sec. 5.3 "Static")."""
    if devices < 1:
        raise ValueError("at least one device")
    U = units_of(G, grain)
    if props is None or len(props) == 0:
        sizes = [U // devices] * (devices - 1)
    else:
        if len(props) not in (devices - 1, devices):
            raise ValueError("Static needs D-1 or D proportions")
        if any(p < 0 for p in props) or sum(props[: devices - 1]) > 1.0 + 1e-12:
            raise ValueError("proportions must be >= 0 and sum to at most 1")
        sizes = [math.floor(float(p) * float(U)) for p in props[: devices - 1]]
        if sum(sizes) > U:
            raise ValueError("proportions exceed the NDRange")
    sizes.append(U - sum(sizes))
    order = list(range(devices))
    if reverse:
        order.reverse()
    out: List[Package] = [(0, 0)] * devices
    u = 0
    for d in order:
        out[d] = unit_range_to_wg(G, grain, u, sizes[d])
        u += sizes[d]
    return out


def dynamic(G: int, num_packages: int, grain: int = 1) -> List[Package]:
    """Equal packages handed out in order (Sec. 5.3 "Dynamic")."""
    if num_packages < 1:
        raise ValueError("at least one package")
    U = units_of(G, grain)
    if U == 0:
        return []
    size = -(-U // num_packages)
    pk = []
    u = 0
    while u < U:
        ul = min(size, U - u)
        pk.append(unit_range_to_wg(G, grain, u, ul))
        u += ul
    return pk


def hguided_min(min_base: int, powers: Sequence[float]) -> List[int]:
    """Per-device minimum package size, growing with computing power."""
    pmin = min(powers)
    return [max(1, math.floor(float(min_base) * float(p) / float(pmin) + 0.5)) for p in powers]


def hguided_size(G_r: int, p_i: float, k: float, n: int, sum_p: float, min_i: int) -> int:
    """The HGuided packet-size equation with its lower bound and clip."""
    s = math.floor((float(G_r) * float(p_i)) / ((float(k) * float(n)) * float(sum_p)))
    return min(G_r, max(min_i, s))


def hguided(G: int, devices: int, k: float = 2.0, min_base: int = 1,
            powers: Optional[Sequence[float]] = None, grain: int = 1,
            request_order: Optional[Sequence[int]] = None) -> List[Tuple[int, int, int]]:
    """HGuided packages as (device, offset_wg, length_wg) in hand-out order.

    With equal powers the sizes depend on G_r only, so the sequence of
    (offset, length) does not depend on which device asks.  With unequal
    powers the caller gives the order in which devices asked
    (``request_order``); devices cycle 0..D-1 when it is omitted.
    """
    if devices < 1 or k <= 0 or min_base < 1:
        raise ValueError("bad HGuided parameters")
    if powers is None:
        powers = [1.0] * devices
    if len(powers) != devices or any(p <= 0 for p in powers):
        raise ValueError("one positive power per device")
    sum_p = 0.0
    for p in powers:
        sum_p += float(p)
    mins = hguided_min(min_base, powers)
    U = units_of(G, grain)
    G_r = U
    u = 0
    out = []
    t = 0
    while G_r > 0:
        if request_order is not None:
            if t >= len(request_order):
                raise ValueError("request order shorter than the package count")
            d = request_order[t]
        else:
            d = t % devices
        ul = hguided_size(G_r, powers[d], k, devices, sum_p, mins[d])
        off, ln = unit_range_to_wg(G, grain, u, ul)
        out.append((d, off, ln))
        u += ul
        G_r -= ul
        t += 1
    return out


def coverage(G: int, packages: Sequence[Package]) -> List[int]:
    """How many times each work-group is covered by the packages."""
    cov = [0] * G
    for off, ln in packages:
        for w in range(off, off + ln):
            cov[w] += 1
    return cov
