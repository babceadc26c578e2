"""Helpers shared by the GPU parity tests: layout conversion and pair matching.

These only re-index arrays; they hold no SNAP arithmetic.
"""
import numpy as np

from oracle import snap_oracle as O


def half_to_full(half: np.ndarray, twojmax: int, half_index) -> np.ndarray:
    """[n][H][2] half-layout (library) -> [n][nfull] complex full matrices
    (oracle layout), filling the other columns with
    M[t-ma][t-mb] = (-1)^(ma+mb) conj(M[ma][mb])."""
    n = half.shape[0]
    hc = half[..., 0] + 1j * half[..., 1]
    out = np.zeros((n, O.full_size(twojmax)), dtype=complex)
    for t in range(twojmax + 1):
        fb = O.full_base(t)
        for ma in range(t + 1):
            for mb in range(t + 1):
                if 2 * mb <= t:
                    v = hc[:, half_index(twojmax, t, ma, mb)]
                else:
                    s = (-1) ** (ma + mb)
                    v = s * np.conj(hc[:, half_index(twojmax, t, t - ma, t - mb)])
                out[:, fb + ma * (t + 1) + mb] = v
    return out


def gpu_pairs(s, n):
    """Slots of the library's neighbour table as {(i, k, ix, iy, iz): slot}."""
    from paper_2011_12875_gb300 import snap
    cnt = s.get_buffer(snap.BUF_NBR_CNT)
    K = s.get_buffer(snap.BUF_NBR_IDX).size // n
    idx = s.get_buffer(snap.BUF_NBR_IDX).reshape(n, K)
    img = s.get_buffer(snap.BUF_NBR_IMG).reshape(n, K, 3)
    keys = {}
    for i in range(n):
        for q in range(cnt[i]):
            keys[(i, int(idx[i, q]), *map(int, img[i, q]))] = i * K + q
    return keys, K, cnt


def oracle_pairs(pairs):
    return {(int(pairs.i[q]), int(pairs.k[q]), *map(int, pairs.img[q])): q
            for q in range(len(pairs.i))}


def rel_err(got, want):
    scale = np.abs(want).max()
    return float(np.abs(np.asarray(got) - np.asarray(want)).max() / (scale if scale > 0 else 1.0))
