"""Thin Python binding of the C ABI in include/snap_gb300.h.

Argument marshalling only: every step of the SNAP evaluation runs in the CUDA
library ``_build/libsnap_gb300.so``.  PyTorch supplies device memory and the
current CUDA stream.  If the library cannot be loaded this module raises; it
has no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsnap_gb300.so")

FP64 = 0
MIXED = 1

OK = 0
ERR_ARG = -1
ERR_NEIGH_OVERFLOW = -2
ERR_BOX = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_NOMEM = -6
ERR_NEIGH_ASYM = -7

KNOB_COL_WARPS = 0
KNOB_YI_WAVES = 1
KNOB_YI_LAYOUT = 2
KNOB_PERSIST = 3
KNOB_DE_ATOMS = 4
KNOB_BI_LAYOUT = 5

BUF_NBR_CNT = 0
BUF_NBR_IDX = 1
BUF_NBR_IMG = 2
BUF_NBR_REV = 3
BUF_RIJ = 4
BUF_ULISTTOT = 5
BUF_YLIST = 6
BUF_DEDR = 7

EXPORTS = ("snap_num_coeff", "snap_create", "snap_set_beta", "snap_set_neigh_cap",
           "snap_neigh_max", "snap_compute", "snap_compute_async", "snap_sync",
           "snap_compute_host", "snap_get_buffer", "snap_half_index", "snap_half_size",
           "snap_destroy", "snap_last_error", "snap_profile", "snap_profile_read",
           "snap_stage_name", "snap_launches_per_call", "snap_compute_bispectrum",
           "snap_compute_bispectrum_async",
           "snap_bispectrum_deriv", "snap_force_weighted", "snap_generation",
           "snap_compute_batch", "snap_set_tuning", "snap_get_tuning", "snap_autotune",
           "snap_neighbors_noalloc", "snap_yi_host", "snap_bi_host", "snap_test_stage_timeout",
           "snap_probe_fma", "snap_bispectrum_deriv_batch", "snap_set_knob", "snap_get_knob")
NSTAGES = 5

_lib = None


class SnapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"snap error {code}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load the CUDA library (raises OSError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    i, d, p, ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
    L.snap_num_coeff.argtypes = [i]
    L.snap_num_coeff.restype = i
    L.snap_create.argtypes = [i, d, d, d, i, p, i, ctypes.POINTER(p)]
    L.snap_create.restype = i
    L.snap_set_beta.argtypes = [p, p]
    L.snap_set_beta.restype = i
    L.snap_set_neigh_cap.argtypes = [p, i]
    L.snap_set_neigh_cap.restype = i
    L.snap_neigh_max.argtypes = [p]
    L.snap_neigh_max.restype = i
    L.snap_compute.argtypes = [p, i, p, p, p, p, p, i, p, p, p, p]
    L.snap_compute.restype = i
    L.snap_compute_async.argtypes = [p, i, p, p, p, p, p, i, p, p, p, p]
    L.snap_compute_async.restype = i
    L.snap_sync.argtypes = [p, p]
    L.snap_sync.restype = i
    L.snap_profile.argtypes = [p, i]
    L.snap_profile.restype = i
    L.snap_profile_read.argtypes = [p, p, p, i]
    L.snap_profile_read.restype = i
    L.snap_stage_name.argtypes = [i]
    L.snap_stage_name.restype = ctypes.c_char_p
    L.snap_launches_per_call.argtypes = [p]
    L.snap_launches_per_call.restype = i
    L.snap_compute_bispectrum.argtypes = [p, i, p, p, p, p, p, i, p, p]
    L.snap_compute_bispectrum.restype = i
    L.snap_compute_bispectrum_async.argtypes = [p, i, p, p, p, p, p, i, p, p]
    L.snap_compute_bispectrum_async.restype = i
    L.snap_bispectrum_deriv.argtypes = [p, i, p, p, p, p, p, i, p, p, p]
    L.snap_bispectrum_deriv.restype = i
    L.snap_force_weighted.argtypes = [p, p, p, p]
    L.snap_force_weighted.restype = i
    L.snap_generation.argtypes = [p]
    L.snap_generation.restype = ctypes.c_longlong
    L.snap_compute_batch.argtypes = [p, i, p, p, p, p, p, p, i, p]
    L.snap_compute_batch.restype = i
    L.snap_bispectrum_deriv_batch.argtypes = [p, i, p, p, p, p, p, p]
    L.snap_bispectrum_deriv_batch.restype = i
    L.snap_set_knob.argtypes = [p, i, i]
    L.snap_set_knob.restype = i
    L.snap_get_knob.argtypes = [p, i, p]
    L.snap_get_knob.restype = i
    L.snap_set_tuning.argtypes = [p, i, i, i]
    L.snap_set_tuning.restype = i
    L.snap_test_stage_timeout.argtypes = [p, i]
    L.snap_test_stage_timeout.restype = i
    L.snap_get_tuning.argtypes = [p, p, p, p]
    L.snap_get_tuning.restype = i
    L.snap_autotune.argtypes = [p, i, p, p, p, p, p, p, i, p, p]
    L.snap_autotune.restype = i
    L.snap_compute_host.argtypes = [p, i, p, p, p, p, p, p]
    L.snap_compute_host.restype = i
    L.snap_get_buffer.argtypes = [p, i, p, ctypes.c_size_t]
    L.snap_get_buffer.restype = ll
    L.snap_half_index.argtypes = [i, i, i, i]
    L.snap_half_index.restype = i
    L.snap_half_size.argtypes = [i]
    L.snap_half_size.restype = i
    L.snap_yi_host.argtypes = [i, i, p, p, p]
    L.snap_yi_host.restype = i
    L.snap_bi_host.argtypes = [i, i, p, p]
    L.snap_bi_host.restype = i
    L.snap_probe_fma.argtypes = [i, i, p, p]
    L.snap_probe_fma.restype = i
    L.snap_destroy.argtypes = [p]
    L.snap_destroy.restype = i
    L.snap_last_error.argtypes = [p]
    L.snap_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def probe_fma(precision: int, iters: int = 1 << 16, stream=None) -> float:
    """Measured FMA peak (TFLOP/s) of the current device in the working
    precision of `precision` (snap_probe_fma)."""
    import torch
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    out = ctypes.c_double()
    rc = load().snap_probe_fma(precision, iters, ctypes.byref(out), ctypes.c_void_p(st))
    if rc != OK:
        raise SnapError(rc, "snap_probe_fma failed")
    return out.value


def num_coeff(twojmax: int) -> int:
    return load().snap_num_coeff(twojmax)


def half_size(twojmax: int) -> int:
    return load().snap_half_size(twojmax)


def half_index(twojmax: int, t: int, ma: int, mb: int) -> int:
    return load().snap_half_index(twojmax, t, ma, mb)


def yi_host(twojmax: int, beta, u_half, precision: int = MIXED) -> np.ndarray:
    """compute_Y's term list for one atom on the host in FP64 (snap_yi_host):
    u_half [H][2] -> Y [H][2], half layout.  No GPU work."""
    H = half_size(twojmax)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    u = np.ascontiguousarray(u_half, dtype=np.float64).reshape(H, 2)
    y = np.zeros((H, 2))
    rc = load().snap_yi_host(twojmax, precision, _np_ptr(beta), _np_ptr(u), _np_ptr(y))
    if rc != 0:
        raise SnapError(rc, "snap_yi_host: invalid argument")
    return y


def bi_host(twojmax: int, u_half, layout: int = 0) -> np.ndarray:
    """The bispectrum kernels' record words for one atom walked on the host in
    FP64 (snap_bi_host): u_half [H][2] -> B [ncoeff].  layout 0: sign-flip
    words, 1: conjugate-plane words.  No GPU work."""
    H = half_size(twojmax)
    u = np.ascontiguousarray(u_half, dtype=np.float64).reshape(H, 2)
    b = np.zeros(num_coeff(twojmax))
    rc = load().snap_bi_host(twojmax, layout, _np_ptr(u), _np_ptr(b))
    if rc != 0:
        raise SnapError(rc, "snap_bi_host: invalid argument")
    return b


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _t_ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Snap:
    """One SNAP potential (2J, R_cut, rfac0, rmin0, switching, beta) on the
    current CUDA device, in FP64 or mixed precision."""

    def __init__(self, twojmax: int, beta, rcut: float = 4.73442, rfac0: float = 0.99363,
                 rmin0: float = 0.0, switchflag: int = 1, precision: int = FP64):
        self._lib = load()
        self.twojmax = twojmax
        self.precision = precision
        self._hp = {}      # host-array addresses (compute_host)
        self._boxes = {}   # boxes as float64 arrays (compute_host)
        b = np.ascontiguousarray(beta, dtype=np.float64)
        nc = self._lib.snap_num_coeff(twojmax)
        if nc < 0 or b.shape != (nc + 1,):
            raise ValueError(f"beta must have 1 + {nc} entries for twojmax={twojmax}")
        h = ctypes.c_void_p()
        rc = self._lib.snap_create(twojmax, rcut, rfac0, rmin0, switchflag, _np_ptr(b), precision,
                                   ctypes.byref(h))
        if rc != OK:
            raise SnapError(rc, self._lib.snap_last_error(None).decode())
        self._h = h

    def _check(self, rc: int):
        if rc != OK:
            raise SnapError(rc, self._lib.snap_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.snap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_beta(self, beta):
        b = np.ascontiguousarray(beta, dtype=np.float64)
        self._check(self._lib.snap_set_beta(self._h, _np_ptr(b)))

    def set_neigh_cap(self, cap: int):
        self._check(self._lib.snap_set_neigh_cap(self._h, cap))

    def neigh_max(self) -> int:
        return self._lib.snap_neigh_max(self._h)

    def compute(self, pos, box, energy=None, forces=None, virial=None, neighbors=None,
                stream=None, wait=True):
        """Evaluate on device tensors (torch, float64, [N,3] positions).

        box: 3 box lengths (host sequence).  neighbors: optional (cnt, idx, img)
        device tensors (int32 [N], int32 [N,cap], int8 [N,cap,3]).
        Returns (energy [N], forces [N,3], virial [6]) tensors.
        """
        import torch
        if pos.dtype != torch.float64 or not pos.is_cuda or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous float64 CUDA tensor")
        n = pos.shape[0]
        dev = pos.device
        if energy is None:
            energy = torch.empty(n, dtype=torch.float64, device=dev)
        if forces is None:
            forces = torch.empty((n, 3), dtype=torch.float64, device=dev)
        if virial is None:
            virial = torch.empty(6, dtype=torch.float64, device=dev)
        boxa = np.ascontiguousarray(box, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        cnt = idx = img = None
        cap = 0
        if neighbors is not None:
            cnt, idx, img = neighbors
            cap = idx.shape[1]
        fn = self._lib.snap_compute if wait else self._lib.snap_compute_async
        self._check(fn(self._h, n, _t_ptr(pos), _np_ptr(boxa), _t_ptr(cnt), _t_ptr(idx),
                       _t_ptr(img), cap, _t_ptr(energy), _t_ptr(forces), _t_ptr(virial),
                       ctypes.c_void_p(stream)))
        return energy, forces, virial

    def bispectrum(self, pos, box, out=None, neighbors=None, stream=None, wait=True):
        """Bispectrum components B [N, N_B] (float64 device tensor).  With
        wait=False the call returns once enqueued; device-side errors come
        from the next sync()."""
        import torch
        if pos.dtype != torch.float64 or not pos.is_cuda or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous float64 CUDA tensor")
        n = pos.shape[0]
        nc = self._lib.snap_num_coeff(self.twojmax)
        if out is None:
            out = torch.empty((n, nc), dtype=torch.float64, device=pos.device)
        boxa = np.ascontiguousarray(box, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream(pos.device).cuda_stream
        cnt = idx = img = None
        cap = 0
        if neighbors is not None:
            cnt, idx, img = neighbors
            cap = idx.shape[1]
        fn = self._lib.snap_compute_bispectrum if wait else self._lib.snap_compute_bispectrum_async
        self._check(fn(
            self._h, n, _t_ptr(pos), _np_ptr(boxa), _t_ptr(cnt), _t_ptr(idx), _t_ptr(img), cap,
            _t_ptr(out), ctypes.c_void_p(stream)))
        return out

    def bispectrum_deriv(self, pos, box, g, out=None, neighbors=None, stream=None):
        """dB[i, l] = sum_k g_k . dB_l(i)/dr_k for a displacement field g [N, 3]."""
        import torch
        for t in (pos, g):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("pos and g must be contiguous float64 CUDA tensors")
        n = pos.shape[0]
        nc = self._lib.snap_num_coeff(self.twojmax)
        if out is None:
            out = torch.empty((n, nc), dtype=torch.float64, device=pos.device)
        boxa = np.ascontiguousarray(box, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream(pos.device).cuda_stream
        cnt = idx = img = None
        cap = 0
        if neighbors is not None:
            cnt, idx, img = neighbors
            cap = idx.shape[1]
        self._check(self._lib.snap_bispectrum_deriv(
            self._h, n, _t_ptr(pos), _np_ptr(boxa), _t_ptr(cnt), _t_ptr(idx), _t_ptr(img), cap,
            _t_ptr(g), _t_ptr(out), ctypes.c_void_p(stream)))
        return out

    def force_weighted(self, weight, out=None, stream=None):
        """Gradient of sum_i w_i E_i w.r.t. positions for the last evaluation."""
        import torch
        if weight.dtype != torch.float64 or not weight.is_cuda or not weight.is_contiguous():
            raise ValueError("weight must be a contiguous float64 CUDA tensor")
        n = weight.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=weight.device)
        if stream is None:
            stream = torch.cuda.current_stream(weight.device).cuda_stream
        self._check(self._lib.snap_force_weighted(self._h, _t_ptr(weight), _t_ptr(out),
                                                  ctypes.c_void_p(stream)))
        return out

    def _batch_args(self, pos, natoms, boxes, energy, forces, virial):
        import torch
        if pos.dtype != torch.float64 or not pos.is_cuda or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous float64 CUDA tensor")
        na = np.ascontiguousarray(natoms, dtype=np.int32)
        bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        if bx.shape[0] != na.shape[0] or int(na.sum()) != pos.shape[0]:
            raise ValueError("natoms, boxes and pos do not describe the same batch")
        n, dev = pos.shape[0], pos.device
        if energy is None:
            energy = torch.empty(n, dtype=torch.float64, device=dev)
        if forces is None:
            forces = torch.empty((n, 3), dtype=torch.float64, device=dev)
        if virial is None:
            virial = torch.empty((na.shape[0], 6), dtype=torch.float64, device=dev)
        return na, bx, energy, forces, virial

    def compute_batch(self, pos, natoms, boxes, energy=None, forces=None, virial=None,
                      use_graph=True, stream=None, wait=True):
        """Evaluate a batch of configurations (atoms concatenated in pos).

        Returns (energy [N], forces [N,3], virial [nconf,6]).  With use_graph
        the launch sequence is captured once per batch shape and replayed.
        """
        import torch
        na, bx, energy, forces, virial = self._batch_args(pos, natoms, boxes, energy, forces, virial)
        if stream is None:
            stream = torch.cuda.current_stream(pos.device).cuda_stream
        self._check(self._lib.snap_compute_batch(
            self._h, len(na), _np_ptr(na), _np_ptr(bx), _t_ptr(pos), _t_ptr(energy),
            _t_ptr(forces), _t_ptr(virial), int(bool(use_graph)), ctypes.c_void_p(stream)))
        if wait:
            self.sync(stream)
        self._batch_keep = (na, bx)
        return energy, forces, virial

    def bispectrum_deriv_batch(self, pos, natoms, boxes, g, out=None, stream=None, wait=True):
        """snap_bispectrum_deriv over a batch of configurations (see
        compute_batch for the layout): dB [sum natoms, N_B]."""
        import torch
        na, bx, _, _, _ = self._batch_args(pos, natoms, boxes, None, None, None)
        if g.dtype != torch.float64 or not g.is_cuda or not g.is_contiguous() or g.shape != pos.shape:
            raise ValueError("g must be a contiguous float64 CUDA tensor shaped like pos")
        nc = self._lib.snap_num_coeff(self.twojmax)
        if out is None:
            out = torch.empty((pos.shape[0], nc), dtype=torch.float64, device=pos.device)
        if stream is None:
            stream = torch.cuda.current_stream(pos.device).cuda_stream
        self._check(self._lib.snap_bispectrum_deriv_batch(
            self._h, len(na), _np_ptr(na), _np_ptr(bx), _t_ptr(pos), _t_ptr(g), _t_ptr(out),
            ctypes.c_void_p(stream)))
        self._batch_keep = (na, bx)
        if wait:
            self.sync(stream)
        return out

    def set_tuning(self, col_warps: int, yi_waves: int, yi_layout: int = 0):
        """Launch-shape tunables (see snap_set_tuning); yi_layout 0 = warp of
        32 atoms, 1 = warp per atom."""
        self._check(self._lib.snap_set_tuning(self._h, col_warps, yi_waves, yi_layout))

    def set_knob(self, knob: int, value: int):
        """One tunable (KNOB_*; see snap_set_knob)."""
        self._check(self._lib.snap_set_knob(self._h, knob, value))

    def get_knob(self, knob: int) -> int:
        v = ctypes.c_int()
        self._check(self._lib.snap_get_knob(self._h, knob, ctypes.byref(v)))
        return v.value

    def test_stage_timeout(self, on: bool):
        """Test hook (snap_test_stage_timeout): staging copies are not issued,
        so their bounded waits run out and calls raise SnapError
        (ERR_TIMEOUT) until it is switched off again."""
        self._check(self._lib.snap_test_stage_timeout(self._h, int(bool(on))))

    def get_tuning(self):
        """(col_warps, yi_waves, yi_layout)."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.snap_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, pos, natoms, boxes, reps: int = 5, stream=None):
        """Pick the fastest launch shape for this batch; returns its median ms."""
        import torch
        na, bx, energy, forces, virial = self._batch_args(pos, natoms, boxes, None, None, None)
        if stream is None:
            stream = torch.cuda.current_stream(pos.device).cuda_stream
        best = ctypes.c_double()
        self._check(self._lib.snap_autotune(
            self._h, len(na), _np_ptr(na), _np_ptr(bx), _t_ptr(pos), _t_ptr(energy), _t_ptr(forces),
            _t_ptr(virial), reps, ctypes.byref(best), ctypes.c_void_p(stream)))
        return best.value

    def generation(self) -> int:
        return int(self._lib.snap_generation(self._h))

    def sync(self, stream=None):
        """Wait for the stream; raise if the last asynchronous compute failed."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._check(self._lib.snap_sync(self._h, ctypes.c_void_p(stream)))

    def profile(self, enable: bool):
        self._check(self._lib.snap_profile(self._h, int(enable)))

    def profile_read(self):
        """{stage name: (total ms, calls)} of the per-stage CUDA-event timing."""
        ms = np.zeros(NSTAGES)
        calls = np.zeros(NSTAGES, dtype=np.int64)
        rc = self._lib.snap_profile_read(self._h, _np_ptr(ms), _np_ptr(calls), NSTAGES)
        if rc < 0:
            self._check(rc)
        return {self._lib.snap_stage_name(k).decode(): (float(ms[k]), int(calls[k]))
                for k in range(NSTAGES)}

    def launches_per_call(self) -> int:
        return self._lib.snap_launches_per_call(self._h)

    def _host_ptr(self, a):
        """Address of a host array's data.  Arrays passed again (the usual loop
        over steps with the same buffers) take it from a cache that holds a
        reference to each array, so its buffer cannot move or be freed while
        cached (numpy cannot resize an array that has other references)."""
        if a is None:
            return None
        hit = self._hp.get(id(a))
        if hit is not None and hit[0] is a:
            return hit[1]
        if len(self._hp) >= 16:
            self._hp.clear()
        p = a.ctypes.data
        self._hp[id(a)] = (a, p)
        return p

    def compute_host(self, pos: np.ndarray, box, stream=None, want_energy=True, want_virial=True,
                     out=None):
        """Evaluate from HOST numpy arrays (copies in and out inside the call)."""
        if not (isinstance(pos, np.ndarray) and pos.dtype == np.float64 and pos.flags.c_contiguous):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        n = pos.shape[0]
        if out is None:
            E = np.empty(n) if want_energy else None
            F = np.empty((n, 3))
            W = np.empty(6) if want_virial else None
        else:
            E, F, W = out
        key = tuple(float(x) for x in box)
        boxa = self._boxes.get(key)
        if boxa is None:
            if len(self._boxes) >= 16:
                self._boxes.clear()
            boxa = self._boxes[key] = np.array(key, dtype=np.float64)
        hp = self._host_ptr
        self._check(self._lib.snap_compute_host(
            self._h, n, hp(pos), hp(boxa), hp(E), hp(F), hp(W), stream or 0))
        return E, F, W

    def get_buffer(self, which: int) -> np.ndarray:
        """Internal buffer of the last compute, as a host numpy array."""
        nbytes = self._lib.snap_get_buffer(self._h, which, None, 0)
        if nbytes < 0:
            self._check(int(nbytes))
        raw = np.empty(max(int(nbytes), 1), dtype=np.uint8)
        rc = self._lib.snap_get_buffer(self._h, which, _np_ptr(raw), raw.nbytes)
        if rc < 0:
            self._check(int(rc))
        raw = raw[:int(nbytes)]
        dt = {BUF_NBR_CNT: np.int32, BUF_NBR_IDX: np.int32, BUF_NBR_IMG: np.int8,
              BUF_NBR_REV: np.int32, BUF_RIJ: np.float64, BUF_ULISTTOT: np.float64,
              BUF_YLIST: np.float64, BUF_DEDR: np.float64}[which]
        return raw.view(dt)
