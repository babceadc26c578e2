"""The C-ABI library loads and exports every symbol its header declares, and
its host-only entry points answer without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snap_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    return snap.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(snap_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("snap_create", "snap_compute", "snap_destroy", "snap_num_coeff",
                 "snap_set_beta", "snap_last_error", "snap_compute_host"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2011_12875_gb300 import build, snap
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (snap_[a-z_0-9]+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(snap.EXPORTS) <= exported


def test_host_only_entry_points(lib):
    from paper_2011_12875_gb300 import snap
    assert snap.num_coeff(8) == 55 and snap.num_coeff(14) == 204
    assert snap.num_coeff(0) == 1 and snap.num_coeff(15) == -1 and snap.num_coeff(-1) == -1
    assert snap.half_size(8) == 155 and snap.half_size(14) == 652
    # half layout: t-major, then mb, then ma, dense
    seen = []
    for t in range(9):
        for mb in range(t // 2 + 1):
            for ma in range(t + 1):
                seen.append(snap.half_index(8, t, ma, mb))
    assert seen == list(range(155))
    assert snap.half_index(8, 4, 0, 3) == -1 and snap.half_index(8, 9, 0, 0) == -1


def test_create_validates_arguments_before_the_gpu(lib):
    import numpy as np
    from paper_2011_12875_gb300 import snap
    beta = np.zeros(56)
    bad = [dict(twojmax=15), dict(rcut=0.0), dict(rfac0=1.5), dict(rmin0=-1.0),
           dict(switchflag=2), dict(precision=7)]
    for b in bad:
        kw = dict(twojmax=8, rcut=4.7, rfac0=0.99, rmin0=0.0, switchflag=1, precision=0)
        kw.update(b)
        h = ctypes.c_void_p()
        nb = np.zeros(snap.num_coeff(kw["twojmax"]) + 1 if kw["twojmax"] <= 14 else 1)
        rc = lib.snap_create(kw["twojmax"], kw["rcut"], kw["rfac0"], kw["rmin0"],
                             kw["switchflag"], nb.ctypes.data_as(ctypes.c_void_p),
                             kw["precision"], ctypes.byref(h))
        assert rc == snap.ERR_ARG, b
        assert not h.value
        assert lib.snap_last_error(None)


def test_create_without_gpu_reports_cuda_error(lib):
    import numpy as np
    import torch
    from paper_2011_12875_gb300 import snap
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(snap.SnapError) as ei:
        snap.Snap(8, np.zeros(56))
    assert ei.value.code == snap.ERR_CUDA


def test_noalloc_refuses_bad_boxes_and_cutoffs_before_the_gpu(lib):
    """The allocation-free neighbour list checks its box and cutoff on the
    host: a box so short against rcut that the image loop would run away, a
    non-finite box and a non-finite or non-positive rcut are refused before
    any CUDA call (this runs without a GPU)."""
    import numpy as np
    from paper_2011_12875_gb300 import snap
    p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.snap_neighbors_noalloc.argtypes = [i, p, p, d, i, p, p, p, p, p, p]
    lib.snap_neighbors_noalloc.restype = i

    def call(box, rcut, n=4):
        b = np.ascontiguousarray(box, dtype=np.float64)
        return lib.snap_neighbors_noalloc(n, None, b.ctypes.data_as(p), rcut, 32,
                                          None, None, None, None, None, None)
    # 0.01 A box against a 4.7 A cutoff: 471 shifts a side
    assert call([0.01, 0.01, 0.01], 4.7) == snap.ERR_BOX
    # short along one axis only: more than 100 shifts
    assert call([0.04, 50.0, 50.0], 4.7) == snap.ERR_BOX
    # 0.5 A box: 11 shifts a side, 23^3 images per atom (> 4096)
    assert call([0.5, 0.5, 0.5], 4.7) == snap.ERR_BOX
    assert call([np.inf, 5.0, 5.0], 4.7) == snap.ERR_BOX
    assert call([np.nan, 5.0, 5.0], 4.7) == snap.ERR_BOX
    assert call([5.0, 0.0, 5.0], 4.7) == snap.ERR_BOX
    for rc in (np.inf, -np.inf, np.nan, 0.0, -1.0):
        assert call([5.0, 5.0, 5.0], rc) == snap.ERR_ARG, rc
    # finite but absurd: every box is too short for it
    assert call([5.0, 5.0, 5.0], 1e300) == snap.ERR_BOX
