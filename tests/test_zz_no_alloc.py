"""snap_neighbors_noalloc: the neighbour-list entry point for callers that
cannot call cudaMalloc (a host program whose device memory belongs to its own
pool, or a caller on a latency-critical path where cudaMalloc may synchronise
the device).  It must produce the same list as the existing entry point
(snap_compute's device builder, read back with snap_get_buffer), call after
call, although all calls share one fixed scratch array inside the library.

This file is collected last on purpose, and it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from paper_2011_12875_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    L = snap.load()
    p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.snap_neighbors_noalloc.argtypes = [i, p, p, d, i, p, p, p, p, p, p]
    L.snap_neighbors_noalloc.restype = i
    return L


def existing_lists(cfg, cap):
    """Neighbour list of the existing entry point (snap_compute)."""
    from paper_2011_12875_gb300 import snap
    s = snap.Snap(4, inputs.beta(4))
    s.set_neigh_cap(cap)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda:0")
    s.compute(pos, cfg.box)
    n = cfg.natoms
    out = (s.get_buffer(snap.BUF_NBR_CNT).copy(),
           s.get_buffer(snap.BUF_NBR_IDX).reshape(n, cap).copy(),
           s.get_buffer(snap.BUF_NBR_IMG).reshape(n, cap, 3).copy(),
           s.get_buffer(snap.BUF_RIJ).reshape(n, cap, 3).copy())
    s.close()
    return out


def noalloc_lists(lib, cfg, cap):
    n = cfg.natoms
    dev = "cuda:0"
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device=dev)
    cnt = torch.full((n,), -1, dtype=torch.int32, device=dev)
    nbr = torch.full((n, cap), -1, dtype=torch.int32, device=dev)
    img = torch.zeros((n, cap, 3), dtype=torch.int8, device=dev)
    rij = torch.zeros((n, cap, 3), dtype=torch.float64, device=dev)
    mx = torch.zeros(1, dtype=torch.int32, device=dev)
    box = np.ascontiguousarray(cfg.box, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.snap_neighbors_noalloc(n, ptr(pos), box.ctypes.data_as(ctypes.c_void_p),
                                    inputs.RCUT, cap, ptr(cnt), ptr(nbr), ptr(img), ptr(rij),
                                    ptr(mx), ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    return (cnt.cpu().numpy(), nbr.cpu().numpy(), img.cpu().numpy(), rij.cpu().numpy(),
            int(mx.item()))


def same(got, want):
    cnt, nbr, img, rij = want
    assert np.array_equal(got[0], cnt)
    for i in range(len(cnt)):
        c = cnt[i]
        assert np.array_equal(got[1][i, :c], nbr[i, :c])
        assert np.array_equal(got[2][i, :c], img[i, :c])
        # exact FP64 separations; the parity tolerance is 1e-10 relative
        np.testing.assert_allclose(got[3][i, :c], rij[i, :c], rtol=0, atol=1e-10 * 4.73442)


def test_noalloc_matches_existing_entry_point_on_consecutive_calls(lib):
    """Two calls in a row on different configurations (a large box with
    nearest images and a small box with many images of each atom): both match
    the existing entry point, so the shared scratch is reset between calls."""
    cap = 32
    a = inputs.bcc(4, disp=0.1)
    b = inputs.bcc(2, disp=0.15, seed=3)
    want_a, want_b = existing_lists(a, cap), existing_lists(b, cap)
    got_a = noalloc_lists(lib, a, cap)
    got_b = noalloc_lists(lib, b, cap)
    same(got_a[:4], want_a)
    same(got_b[:4], want_b)
    assert got_a[4] == want_a[0].max() == 26
    assert got_b[4] == want_b[0].max()
    again = noalloc_lists(lib, a, cap)
    same(again[:4], want_a)


def test_noalloc_reports_overflow_and_rejects_oversized_input(lib):
    cfg = inputs.bcc(4, disp=0.1)
    got = noalloc_lists(lib, cfg, 8)
    assert got[4] == 26 and got[0].max() == 8
    box = np.ascontiguousarray(cfg.box, dtype=np.float64)
    rc = lib.snap_neighbors_noalloc(65537, None, box.ctypes.data_as(ctypes.c_void_p), 4.7, 32,
                                    None, None, None, None, None, None)
    assert rc == -1  # SNAP_ERR_ARG: more atoms than the fixed scratch holds
    p = box.ctypes.data_as(ctypes.c_void_p)
    for bad_rcut in (float("inf"), float("nan"), 0.0):
        assert lib.snap_neighbors_noalloc(4, None, p, bad_rcut, 32, None, None, None, None, None,
                                          None) == -1
    tiny = np.array([0.01, 0.01, 0.01])
    assert lib.snap_neighbors_noalloc(4, None, tiny.ctypes.data_as(ctypes.c_void_p), 4.7, 32, None,
                                      None, None, None, None, None) == -3  # SNAP_ERR_BOX
    # an empty call is valid (it does the set-up) and the next call still matches
    assert lib.snap_neighbors_noalloc(0, None, p, inputs.RCUT, 32, None, None, None, None, None,
                                      None) == 0
    again = noalloc_lists(lib, cfg, 32)
    assert again[4] == 26


def test_noalloc_call_captured_in_a_cuda_graph_replays_on_new_positions(lib):
    """The entry point's reason to exist is use inside a stream capture: one
    call (counter reset, positions, build, max-count copy) is captured once
    and replayed on two configurations of the same box copied into the
    captured position buffer.  Each replay matches the existing entry point,
    max_count included, so the scratch counters are cleared on every replay."""
    cap = 32
    a = inputs.bcc(4, disp=0.1, seed=11)
    b = inputs.bcc(4, disp=0.2, seed=12)
    assert np.array_equal(a.box, b.box)
    n = a.natoms
    dev = "cuda:0"
    pos = torch.tensor(a.pos, dtype=torch.float64, device=dev)
    cnt = torch.full((n,), -1, dtype=torch.int32, device=dev)
    nbr = torch.full((n, cap), -1, dtype=torch.int32, device=dev)
    img = torch.zeros((n, cap, 3), dtype=torch.int8, device=dev)
    rij = torch.zeros((n, cap, 3), dtype=torch.float64, device=dev)
    mx = torch.zeros(1, dtype=torch.int32, device=dev)
    box = np.ascontiguousarray(a.box, dtype=np.float64)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())

    def call(stream):
        return lib.snap_neighbors_noalloc(n, ptr(pos), box.ctypes.data_as(ctypes.c_void_p),
                                          inputs.RCUT, cap, ptr(cnt), ptr(nbr), ptr(img),
                                          ptr(rij), ptr(mx), ctypes.c_void_p(stream))

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        assert call(side.cuda_stream) == 0  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        assert call(torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    for cfg in (a, b, a):
        want = existing_lists(cfg, cap)
        pos.copy_(torch.tensor(cfg.pos, dtype=torch.float64, device=dev))
        cnt.fill_(-1)
        mx.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = (cnt.cpu().numpy(), nbr.cpu().numpy(), img.cpu().numpy(), rij.cpu().numpy())
        same(got, want)
        assert int(mx.item()) == want[0].max()
