"""Algorithmic floating-point work of one SNAP step, per kernel.

Counts the arithmetic the GPU algorithm must do, element by element, with
the conventions: real add or mul = 1 flop, fused multiply-add = 2, complex
multiply = 6, complex multiply-accumulate = 8, real-by-complex scale = 2.
Index arithmetic and loads are not counted.  Used for the roofline fraction
of the benchmark; the derivation is written out in the design notes.
"""
from __future__ import annotations

from functools import lru_cache


def half_layer(t: int):
    """(ma, mb) of the half layout of layer t (mb <= t/2)."""
    return [(ma, mb) for mb in range(t // 2 + 1) for ma in range(t + 1)]


@lru_cache(maxsize=None)
def ui_pair(twojmax: int) -> int:
    """compute_U, one neighbour pair: the layer recursion and the f_c u_t sum.
    Each term of an element is conj(a or b) * u_{t-1} (6) scaled by its root
    factor (2) and added (2); the element is then scaled by f_c and summed (4)."""
    f = 2  # layer 0: f_c added to U_0
    for t in range(1, twojmax + 1):
        for ma, mb in half_layer(t):
            nterm = (ma < t) + (ma > 0)
            f += 10 * nterm + 4
    return f


@lru_cache(maxsize=None)
def de_pair(twojmax: int) -> int:
    """Fused dU + dE, one pair: forward recursion (as compute_U, with the
    Re(Y conj u) accumulation, 4) and the reverse pass: per element of layer
    t-1 two root scalings (4), two conj(lambda) u products accumulated into
    g_a, g_b (16), a*A and b*B (12), the new adjoint (4); the mirrored column
    of even layers repeats the same work; final combination 3 x 10 (FP64)."""
    f = 2
    for t in range(1, twojmax + 1):
        for ma, mb in half_layer(t):
            nterm = (ma < t) + (ma > 0)
            f += 10 * nterm + 4
    for t in range(twojmax, 0, -1):
        tp = t - 1
        for m, mb in half_layer(tp):
            f += 36
            if t % 2 == 0 and mb == t // 2 - 1:
                f += 36
    return f + 30


def _half_elem(t: int, xa: int, xb: int):
    """Stored (index, conjugated) of U_t[xa][xb] in the half layout."""
    base = sum((tt // 2 + 1) * (tt + 1) for tt in range(t))
    if 2 * xb <= t:
        return (base + xb * (t + 1) + xa, 0)
    return (base + (t - xb) * (t + 1) + (t - xa), 1)


@lru_cache(maxsize=None)
def yi_atom(twojmax: int) -> int:
    """compute_Y, one atom.  For each half element (t, ma, mb) of Y, the terms
    beta~ C(ma1,ma2) C(mb1,mb2) U_t1[ma1][mb1] U_t2[ma2][mb2] of every triple
    (t1 >= t2) with output rank t, grouped by their first factor
    U_t1[ma1][mb1]: Y += U_t1[ma1][mb1] * sum_k coef_k U_t2,k.  When t1 == t2
    the term with the factors swapped has the same coefficient, so the pair
    is one term (the stored element with the lower index first).  Per term a
    real-by-complex scale-accumulate (4), per group a complex
    multiply-accumulate (8).  Terms and groups are counted structurally (a
    Clebsch-Gordan product that happens to vanish is still counted)."""
    f = 0
    for t in range(twojmax + 1):
        for ma, mb in half_layer(t):
            groups = set()
            pairs = set()
            for t1 in range(twojmax + 1):
                for t2 in range(t1 + 1):
                    if not (t1 - t2 <= t <= min(twojmax, t1 + t2)) or (t1 + t2 - t) % 2:
                        continue
                    dl = (t1 + t2 - t) // 2
                    for mb1 in range(max(0, mb + dl - t2), min(t1, mb + dl) + 1):
                        for ma1 in range(max(0, ma + dl - t2), min(t1, ma + dl) + 1):
                            x1 = _half_elem(t1, ma1, mb1)
                            x2 = _half_elem(t2, ma + dl - ma1, mb + dl - mb1)
                            if t1 == t2 and x2 < x1:
                                x1, x2 = x2, x1
                            pairs.add((t1, t2, x1, x2))
                            groups.add(x1)
            f += 4 * len(pairs) + 8 * len(groups)
    return f


def step(twojmax: int, natoms: int, npairs: int) -> dict:
    """Flops of one step by stage, keyed by the library's stage names."""
    H = sum(len(half_layer(t)) for t in range(twojmax + 1))
    return {
        # compute_U includes the slot geometry (FP64 core, about 150 flops a slot)
        "compute_ui": (ui_pair(twojmax) + 150) * npairs,
        "compute_yi": yi_atom(twojmax) * natoms,
        "fused_dE": de_pair(twojmax) * npairs,
        "energy_force_virial": natoms * 4 * H + npairs * 30,
    }
