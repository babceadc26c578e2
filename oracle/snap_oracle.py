"""ctypes wrapper around the FP64 C oracle (test infrastructure only).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  Every function returns numpy arrays in the
oracle's own layouts (full (t+1)x(t+1) matrices per layer t = 2j, row-major
[ma][mb], complex128), independent of the CUDA library's layouts.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.c_double
        i = ctypes.c_int
        p = ctypes.c_void_p
        L.orc_ncoeff.argtypes = [i]
        L.orc_ncoeff.restype = i
        L.orc_full_size.argtypes = [i]
        L.orc_full_size.restype = i
        L.orc_triples.argtypes = [i, p]
        L.orc_triples.restype = None
        L.orc_cg.argtypes = [i, i, i, i, i, i]
        L.orc_cg.restype = d
        L.orc_ulist_pair.argtypes = [i, d, d, d, d, d, d, i, p, p, p]
        L.orc_ulist_pair.restype = None
        L.orc_build_neighbors.argtypes = [i, p, p, d, i, p, p, p, p]
        L.orc_build_neighbors.restype = i
        L.orc_compute.argtypes = [i, d, d, d, i, d, p, i, i, p, p, p, p,
                                  p, p, p, p, p, p, p]
        L.orc_compute.restype = i
        L.orc_energy_from_u.argtypes = [i, p, p, p]
        L.orc_energy_from_u.restype = d
        L.orc_flops.argtypes = [i, p]
        L.orc_flops.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def ncoeff(twojmax: int) -> int:
    return lib().orc_ncoeff(twojmax)


def full_size(twojmax: int) -> int:
    return lib().orc_full_size(twojmax)


def triples(twojmax: int) -> np.ndarray:
    n = ncoeff(twojmax)
    out = np.zeros((n, 3), dtype=np.int32)
    lib().orc_triples(twojmax, _ptr(out))
    return out


def full_base(t: int) -> int:
    return sum((s + 1) ** 2 for s in range(t))


def block(arr: np.ndarray, t: int) -> np.ndarray:
    """View of layer t of a full-matrix array as a (t+1, t+1) matrix."""
    b = full_base(t)
    return arr[..., b:b + (t + 1) ** 2].reshape(arr.shape[:-1] + (t + 1, t + 1))


def cg(t1: int, m1x2: int, t2: int, m2x2: int, t: int, mx2: int) -> float:
    """<j1 m1 j2 m2 | j m> with doubled arguments (t = 2j, mx2 = 2m)."""
    return lib().orc_cg(t1, m1x2, t2, m2x2, t, mx2)


@dataclass
class Params:
    twojmax: int
    rcut: float = 4.73442
    rfac0: float = 0.99363
    rmin0: float = 0.0
    switchflag: int = 1
    wself: float = 1.0


def ulist_pair(p: Params, r, with_du: bool = False):
    """u_t (full, complex) of one neighbour vector r; optionally du_t/dr_d.

    Returns (u, du or None, geom) where geom = dict(a, b, fc, dfc, da, db).
    """
    nf = full_size(p.twojmax)
    u = np.zeros(2 * nf)
    du = np.zeros(3 * 2 * nf) if with_du else None
    g = np.zeros(20)
    lib().orc_ulist_pair(p.twojmax, float(r[0]), float(r[1]), float(r[2]), p.rcut,
                         p.rfac0, p.rmin0, p.switchflag, _ptr(u), _ptr(du), _ptr(g))
    uc = u.view(np.complex128)
    duc = du.view(np.complex128).reshape(3, nf) if with_du else None
    geom = dict(a=complex(g[0], g[1]), b=complex(g[2], g[3]), fc=g[4], dfc=g[5:8].copy(),
                da=g[8:14].view(np.complex128).copy(), db=g[14:20].view(np.complex128).copy())
    return uc, duc, geom


@dataclass
class Pairs:
    i: np.ndarray      # centre atom of each pair
    k: np.ndarray      # neighbour atom
    img: np.ndarray    # periodic image shift (n, 3) int
    rij: np.ndarray    # r_k + img*L - r_i  (n, 3)


def build_neighbors(pos: np.ndarray, box, rcut: float) -> Pairs:
    """Brute-force periodic neighbour list, grouped by centre atom."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    n = pos.shape[0]
    cap = max(64, 64 * n)
    while True:
        pi = np.zeros(cap, dtype=np.int32)
        pk = np.zeros(cap, dtype=np.int32)
        img = np.zeros((cap, 3), dtype=np.int32)
        rij = np.zeros((cap, 3))
        np_ = lib().orc_build_neighbors(n, _ptr(pos), _ptr(box), rcut, cap, _ptr(pi),
                                        _ptr(pk), _ptr(img), _ptr(rij))
        if np_ >= 0:
            return Pairs(pi[:np_].copy(), pk[:np_].copy(), img[:np_].copy(), rij[:np_].copy())
        cap = -np_


@dataclass
class Result:
    E: np.ndarray            # per-atom energy (n,)
    B: np.ndarray | None     # bispectrum (n, ncoeff)
    U: np.ndarray | None     # Ulisttot (n, nfull) complex
    Y: np.ndarray | None     # adjoint Y (n, nfull) complex
    dedr: np.ndarray         # dE_i/dr_ik per pair (npairs, 3)
    F: np.ndarray | None     # forces (n, 3), only for a full evaluation
    W: np.ndarray | None     # virial (6,) xx yy zz xy xz yz


def compute(p: Params, beta, n: int, pairs: Pairs, need=None, want_UY: bool = False,
            want_B: bool = False) -> Result:
    """Run the oracle on a given pair list.

    need: optional boolean mask of centre atoms to evaluate (E, U, Y, B and the
    dedr of their pairs); forces and virial are only produced when need is None.
    """
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    nc = ncoeff(p.twojmax)
    if beta.shape != (nc + 1,):
        raise ValueError(f"beta must have {nc + 1} entries")
    nf = full_size(p.twojmax)
    npairs = len(pairs.i)
    pi = np.ascontiguousarray(pairs.i, dtype=np.int32)
    pk = np.ascontiguousarray(pairs.k, dtype=np.int32)
    rij = np.ascontiguousarray(pairs.rij, dtype=np.float64)
    needa = None if need is None else np.ascontiguousarray(need, dtype=np.uint8)
    E = np.zeros(n)
    B = np.zeros((n, nc)) if want_B else None
    U = np.zeros((n, 2 * nf)) if want_UY else None
    Y = np.zeros((n, 2 * nf)) if want_UY else None
    dedr = np.zeros((npairs, 3))
    F = np.zeros((n, 3)) if need is None else None
    W = np.zeros(6) if need is None else None
    rc = lib().orc_compute(p.twojmax, p.rcut, p.rfac0, p.rmin0, p.switchflag, p.wself,
                           _ptr(beta), n, npairs, _ptr(pi), _ptr(pk), _ptr(rij), _ptr(needa),
                           _ptr(E), _ptr(B), _ptr(U), _ptr(Y), _ptr(dedr), _ptr(F), _ptr(W))
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return Result(E, B, None if U is None else U.view(np.complex128),
                  None if Y is None else Y.view(np.complex128), dedr, F, W)


def energy_from_u(twojmax: int, beta, U: np.ndarray, want_Y: bool = False):
    """E(U) for one atom from explicit full matrices (complex, length nfull)."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    Uc = np.ascontiguousarray(U, dtype=np.complex128)
    Y = np.zeros(2 * full_size(twojmax)) if want_Y else None
    E = lib().orc_energy_from_u(twojmax, _ptr(beta), _ptr(Uc.view(np.float64)), _ptr(Y))
    return (E, Y.view(np.complex128)) if want_Y else E


def evaluate(p: Params, beta, pos, box, need=None, want_UY=False, want_B=False):
    """Neighbour build plus compute, for convenience. Returns (pairs, result)."""
    pairs = build_neighbors(pos, box, p.rcut)
    res = compute(p, beta, pos.shape[0], pairs, need=need, want_UY=want_UY, want_B=want_B)
    return pairs, res


def forces_for_atoms(p: Params, beta, pos, box, atoms, pairs: Pairs | None = None):
    """Forces on selected atoms only, evaluating just the atoms they touch.

    F_a = sum_{pairs (a,k)} dedr - sum_{pairs (k,a)} dedr needs E_i for i = a
    and for every neighbour of a.
    """
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    if pairs is None:
        pairs = build_neighbors(pos, box, p.rcut)
    atoms = np.asarray(atoms)
    need = np.zeros(n, dtype=bool)
    need[atoms] = True
    sel = np.isin(pairs.i, atoms)
    need[pairs.k[sel]] = True
    res = compute(p, beta, n, pairs, need=need)
    F = np.zeros((len(atoms), 3))
    for idx, a in enumerate(atoms):
        F[idx] += res.dedr[pairs.i == a].sum(axis=0)
        F[idx] -= res.dedr[pairs.k == a].sum(axis=0)
    return F, res, pairs


def threads() -> int:
    """OpenMP threads the oracle will use (OMP_NUM_THREADS or all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def flops(twojmax: int) -> dict:
    """Floating-point work of the oracle's own unreduced evaluation (counted
    by walking its loops): compute_U per pair, B + product-rule Y per atom,
    dU + dE/dr per pair."""
    out = np.zeros(3)
    lib().orc_flops(twojmax, _ptr(out))
    return {"compute_u_pair": float(out[0]), "y_b_atom": float(out[1]), "du_de_pair": float(out[2])}
