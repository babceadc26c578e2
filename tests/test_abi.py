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
