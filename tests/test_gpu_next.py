"""GPU parity of the widened rows: bispectrum output, weighted forces
(autograd backward) and the force-matching derivative d(F.g)/d(beta).

Each is checked against the FP64 oracle, at 1e-10 relative for the FP64
path and at the mixed tolerances of test_gpu_parity.py for the mixed path.
"""
import numpy as np
import pytest

from oracle import snap_oracle as O
from paper_2011_12875_gb300 import inputs
from tests.parity_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_B_TOL = 2e-5


@pytest.fixture(scope="module")
def snapmod():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    snap.load()
    return snap


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("twojmax", [0, 1, 2, 3, 4, 5, 6, 7, 8, 14])
def test_bispectrum_parity(snapmod, twojmax, prec):
    """B[i][l] = Re Z^j_{j1j2} : conj(U_j) (Eq. z) for every atom and component."""
    cfg = inputs.bcc(2, disp=0.15, seed=3)
    beta = inputs.beta(twojmax)
    p = O.Params(twojmax)
    _, ref = O.evaluate(p, beta, cfg.pos, cfg.box, want_B=True)
    s = snapmod.Snap(twojmax, beta, precision=prec)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda:0")
    B = s.bispectrum(pos, cfg.box).cpu().numpy()
    s.close()
    assert B.shape == ref.B.shape
    assert rel_err(B, ref.B) <= (FP64_TOL if prec == 0 else MIXED_B_TOL)


def test_bispectrum_full_size_and_energy_identity(snapmod):
    """2000 atoms, 2J = 8: B against the oracle on every atom, and
    E_i = beta_0 + beta . B_i against the energy path."""
    w = inputs.WORKLOADS["bcc10_2j8"]
    cfg, beta = w.config(), w.beta()
    s = snapmod.Snap(8, beta)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device="cuda:0")
    B = s.bispectrum(pos, cfg.box).cpu().numpy()
    E, _, _ = s.compute(pos, cfg.box)
    s.close()
    _, ref = O.evaluate(O.Params(8), beta, cfg.pos, cfg.box, want_B=True)
    assert rel_err(B, ref.B) <= FP64_TOL
    np.testing.assert_allclose(beta[0] + B @ beta[1:], E.cpu().numpy(), rtol=1e-12)
