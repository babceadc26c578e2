"""The bounded staging wait of compute_Y and of the bispectrum kernels runs
out without faulting or hanging the GPU: with the test hook on, the TMA copy
is registered on its mbarrier but never issued (nothing is in flight), the
wait gives up after its time limit, the call returns SNAP_ERR_TIMEOUT, and
the same context computes correct results once the hook is off."""
import time

import numpy as np
import pytest

from paper_2011_12875_gb300 import inputs
from tests.parity_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snapmod():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    snap.load()
    return snap


@pytest.mark.parametrize("prec", [0, 1])
def test_staging_wait_times_out_and_context_recovers(snapmod, prec):
    cfg = inputs.bcc(2, disp=0.1, seed=51)   # 16 atoms: one 32-atom block, one wave
    s = snapmod.Snap(8, inputs.beta(8), precision=prec)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda:0")
    E0, F0, W0 = [x.cpu().numpy().copy() for x in s.compute(pos, cfg.box)]
    s.test_stage_timeout(True)
    t0 = time.perf_counter()
    with pytest.raises(snapmod.SnapError) as ei:
        s.compute(pos, cfg.box)
    waited = time.perf_counter() - t0
    assert ei.value.code == snapmod.ERR_TIMEOUT
    assert waited < 30.0
    with pytest.raises(snapmod.SnapError) as ei:
        s.bispectrum(pos, cfg.box)
    assert ei.value.code == snapmod.ERR_TIMEOUT
    s.test_stage_timeout(False)
    for _ in range(3):  # direct, then captured and replayed
        E1, F1, W1 = [x.cpu().numpy().copy() for x in s.compute(pos, cfg.box)]
        assert np.array_equal(E1, E0) and np.array_equal(F1, F0) and np.array_equal(W1, W0)
    B = s.bispectrum(pos, cfg.box).cpu().numpy()
    assert rel_err(inputs.beta(8)[0] + B @ inputs.beta(8)[1:], E0) < (1e-12 if prec == 0 else 1e-5)
    s.close()
