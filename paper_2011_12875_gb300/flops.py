"""Algorithmic floating-point work of one SNAP step, per kernel.

Counts the arithmetic the GPU algorithm must do, element by element, with
the conventions: real add or mul = 1 flop, fused multiply-add = 2, complex
multiply = 6, complex multiply-accumulate = 8, real-by-complex scale = 2.
Index arithmetic and loads are not counted.  Used for the roofline fraction
of the benchmark; the derivation is written out in the design notes.
"""
from __future__ import annotations

import heapq
from fractions import Fraction
from functools import lru_cache
from math import factorial


def half_layer(t: int):
    """(ma, mb) of the half layout of layer t (mb <= t/2)."""
    return [(ma, mb) for mb in range(t // 2 + 1) for ma in range(t + 1)]


@lru_cache(maxsize=None)
def ui_pair(twojmax: int) -> int:
    """compute_U, one neighbour pair, in the scaled form the library runs
    (u = S v, v_t[ma] = conj(a) v_{t-1}[ma] - conj(b) v_{t-1}[ma-1], with f_c
    carried in v from layer 0): a complex multiply (6) per term and the
    subtraction of the two terms (2), and the element added to the pair sum
    (2); before an even layer t, the seed of its middle column (layer t-1's
    column t/2: the mirror of column t/2 - 1 scaled by 1/sqrt(t/2), 2 for
    each of its t elements); S and w_self are applied once per atom, not
    per pair."""
    f = 2  # layer 0: f_c added to the sum
    for t in range(1, twojmax + 1):
        if t % 2 == 0:
            f += 2 * t
        for ma, mb in half_layer(t):
            nterm = (ma < t) + (ma > 0)
            f += 6 * nterm + 2 * (nterm - 1) + 2
    return f


@lru_cache(maxsize=None)
def de_pair(twojmax: int) -> int:
    """Fused dU + dE, one pair, in the scaled form (S folded into the
    weighted Y, so neither pass scales by roots).  Forward: the recursion and
    the seeds as in compute_U (layer 0 is v = 1, S = Re Yw_0: no arithmetic)
    and the Re(Yw conj v) accumulation (4) per element.
    Reverse, per element of layer t-1: conj(A) v and conj(B) v accumulated
    into g_a, g_b (8 + 8) and the new adjoint Yw + a A - b B (16); an element
    that also seeds the mirrored column of an even layer t adds the seed's
    scaling of v (2), the same two accumulations (16), a A2 - b B2 (14) and
    its scaled addition to the adjoint (4).  Final combination 3 x 10."""
    f = 0
    for t in range(1, twojmax + 1):
        if t % 2 == 0:
            f += 2 * t
        for ma, mb in half_layer(t):
            nterm = (ma < t) + (ma > 0)
            f += 6 * nterm + 2 * (nterm - 1) + 4
    for t in range(twojmax, 0, -1):
        tp = t - 1
        for m, mb in half_layer(tp):
            f += 32
            if t % 2 == 0 and mb == t // 2 - 1:
                f += 36
    return f + 30


def _half_elem(t: int, xa: int, xb: int) -> int:
    """Stored element of U_t[xa][xb] in the half layout, as 2 index + conj."""
    base = sum((tt // 2 + 1) * (tt + 1) for tt in range(t))
    if 2 * xb <= t:
        return 2 * (base + xb * (t + 1) + xa)
    return 2 * (base + (t - xb) * (t + 1) + (t - xa)) + 1


def _cover_size(edges) -> int:
    """Groups of one output: the greedy vertex cover of its terms (edges
    between stored elements) that takes the element with the most uncovered
    terms first (ties: the larger element), as the library's tables do."""
    inc = {}
    for k, (a, b) in enumerate(edges):
        inc.setdefault(a, []).append(k)
        if b != a:
            inc.setdefault(b, []).append(k)
    deg = {v: len(ks) for v, ks in inc.items()}
    heap = [(-d, -v) for v, d in deg.items()]
    heapq.heapify(heap)
    covered = [False] * len(edges)
    groups = 0
    while heap:
        d, v = heapq.heappop(heap)
        d, v = -d, -v
        if d != deg[v]:
            if deg[v] > 0:
                heapq.heappush(heap, (-deg[v], -v))
            continue
        if d == 0:
            break
        groups += 1
        for k in inc[v]:
            if covered[k]:
                continue
            covered[k] = True
            a, b = edges[k]
            o = b if a == v else a
            if o != v:
                deg[o] -= 1
        deg[v] = 0
    return groups


@lru_cache(maxsize=None)
def _cg_nonzero(t1: int, x1: int, t2: int, x2: int, t: int) -> bool:
    """Whether <j1 m1 j2 m2 | j m1+m2> is nonzero, decided exactly: with
    doubled ranks (t = 2j) and m1 = x1 - t1/2, m2 = x2 - t2/2, for a triangle
    (t1, t2, t) and |m1 + m2| <= j the coefficient is a nonzero factor times
    Racah's alternating sum of inverse factorial products, here summed in
    rationals."""
    a = (t1 + t2 - t) // 2          # j1 + j2 - j
    b = t1 - x1                     # j1 - m1
    c = x2                          # j2 + m2
    d = (t - t1 - t2) // 2 + x1     # j - j2 + m1
    e = (t - t1 + t2) // 2 - x2     # j - j1 - m2
    s = Fraction(0)
    for k in range(max(0, -d, -e), min(a, b, c) + 1):
        s += Fraction((-1) ** k, factorial(k) * factorial(a - k) * factorial(b - k) *
                      factorial(c - k) * factorial(d + k) * factorial(e + k))
    return s != 0


@lru_cache(maxsize=None)
def yi_atom(twojmax: int) -> int:
    """compute_Y, one atom.  For each half element (t, ma, mb) of Y, the terms
    beta~ C(ma1,ma2) C(mb1,mb2) U_t1[ma1][mb1] U_t2[ma2][mb2] of every triple
    (t1 >= t2) with output rank t.  When t1 == t2 the term with the factors
    swapped has the same coefficient, so the pair is one term.  Outputs below
    the centre of the middle column (2 mb = t, ma > mb) are mirrors that no
    contraction reads, and are not computed.  The terms of an output are
    grouped by a shared factor, Y += U[e] * sum_k coef_k U[e_k], the factors
    chosen by a greedy vertex cover.  Per term a real-by-complex
    scale-accumulate (4), per group a complex multiply-accumulate (8).  A
    term whose Clebsch-Gordan product vanishes (a selection rule or an
    accidental zero of Racah's sum) is no work and is not counted."""
    f = 0
    for t in range(twojmax + 1):
        for ma, mb in half_layer(t):
            if 2 * mb == t and ma > mb:
                continue
            pairs = set()
            for t1 in range(twojmax + 1):
                for t2 in range(t1 + 1):
                    if not (t1 - t2 <= t <= min(twojmax, t1 + t2)) or (t1 + t2 - t) % 2:
                        continue
                    dl = (t1 + t2 - t) // 2
                    for mb1 in range(max(0, mb + dl - t2), min(t1, mb + dl) + 1):
                        if not _cg_nonzero(t1, mb1, t2, mb + dl - mb1, t):
                            continue
                        for ma1 in range(max(0, ma + dl - t2), min(t1, ma + dl) + 1):
                            if not _cg_nonzero(t1, ma1, t2, ma + dl - ma1, t):
                                continue
                            x1 = _half_elem(t1, ma1, mb1)
                            x2 = _half_elem(t2, ma + dl - ma1, mb + dl - mb1)
                            pairs.add((min(x1, x2), max(x1, x2)) if t1 == t2 else (x1, x2))
            f += 4 * len(pairs) + 8 * _cover_size(sorted(pairs))
    return f


def step(twojmax: int, natoms: int, npairs: int) -> dict:
    """Flops of one step by stage, keyed by the library's stage names."""
    H = sum(len(half_layer(t)) for t in range(twojmax + 1))
    return {
        # the neighbour build fused with compute_U: the recursion and the slot
        # geometry (FP64 core, about 150 flops a slot); the build's distance
        # tests are not counted
        "neighbor_compute_ui": (ui_pair(twojmax) + 150) * npairs,
        "compute_yi": yi_atom(twojmax) * natoms,
        "fused_dE": de_pair(twojmax) * npairs,
        "energy_force_virial": natoms * 4 * H + npairs * 30,
    }
