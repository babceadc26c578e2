"""Algorithmic floating-point work of one SNAP step, per kernel.

Counts the arithmetic the GPU algorithm must do, element by element, with
the conventions: real add or mul = 1 flop, fused multiply-add = 2, complex
multiply = 6, complex multiply-accumulate = 8, real-by-complex scale = 2.
Index arithmetic and loads are not counted.  Used for the roofline fraction
of the benchmark; the derivation is written out in the design notes.
"""
from __future__ import annotations


def half_layer(t: int):
    """(ma, mb) of the half layout of layer t (mb <= t/2)."""
    return [(ma, mb) for mb in range(t // 2 + 1) for ma in range(t + 1)]


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


def yi_atom(twojmax: int) -> int:
    """compute_Y, one atom: for each half element of each Z^t_{t1 t2}, the
    double sum of CG-weighted products (8 per term: complex multiply 6, CG
    scale-accumulate 2... counted as 6 + 4), the mb1 scale-accumulate (4) and
    the beta-weighted add into Y (4)."""
    f = 0
    for t1 in range(twojmax + 1):
        for t2 in range(t1 + 1):
            for t in range(t1 - t2, min(twojmax, t1 + t2) + 1, 2):
                dl = (t1 + t2 - t) // 2
                for ma, mb in half_layer(t):
                    na = min(t1, ma + dl) - max(0, ma + dl - t2) + 1
                    nb = min(t1, mb + dl) - max(0, mb + dl - t2) + 1
                    if na <= 0 or nb <= 0:
                        continue
                    f += nb * (na * 10 + 4) + 4
    return f


def step(twojmax: int, natoms: int, npairs: int) -> dict:
    """Flops of one step by kernel (the FP64 geometry and force stages are
    small and counted separately)."""
    H = sum(len(half_layer(t)) for t in range(twojmax + 1))
    return {
        "compute_ui": ui_pair(twojmax) * npairs,
        "compute_yi": yi_atom(twojmax) * natoms,
        "fused_dE": de_pair(twojmax) * npairs,
        "force_virial": natoms * 4 * H + npairs * 30,
        "ck_geometry": npairs * 150,
    }
