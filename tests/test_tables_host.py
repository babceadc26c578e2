"""compute_Y's term list against the oracle's Y, on the host (no GPU).

The library walks a reduced term list for Eq. (y) of Sec. III: the two terms
of a t1 == t2 triple with swapped factors are kept as one, each output's
terms are grouped by a shared factor, and the outputs below the centre of the
middle column (2 mb = t, ma > mb) are left at zero because no contraction
reads them.  snap_yi_host evaluates exactly that list in FP64.  For a U with
the inversion symmetry M[t-ma][t-mb] = (-1)^(ma+mb) conj(M[ma][mb]) it must
give the oracle's Y (every triple product of the full matrices multiplied
out) on every element it computes, and the oracle's Y must have the same
symmetry, which the library's Y export uses to fill in the skipped outputs.
"""
import numpy as np
import pytest

from oracle import snap_oracle as O
from paper_2011_12875_gb300 import inputs
from tests.parity_util import half_to_full


@pytest.fixture(scope="module")
def snapmod():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    snap.load()
    return snap


def symmetric_u(snap, twojmax, rng):
    """Random half layout whose middle columns obey the inversion symmetry
    (their lower half mirrors the upper one, the centre is real)."""
    H = snap.half_size(twojmax)
    h = rng.uniform(-1.0, 1.0, (H, 2))
    for t in range(0, twojmax + 1, 2):
        mb = t // 2
        c = snap.half_index(twojmax, t, mb, mb)
        h[c, 1] = 0.0
        for ma in range(mb + 1, t + 1):
            e, m = snap.half_index(twojmax, t, ma, mb), snap.half_index(twojmax, t, t - ma, mb)
            s = -1.0 if (ma + mb) & 1 else 1.0
            h[e] = (s * h[m, 0], -s * h[m, 1])
    return h


def full_pos(t, ma, mb):
    return O.full_base(t) + ma * (t + 1) + mb


@pytest.mark.parametrize("twojmax", [2, 5, 8, 10])
@pytest.mark.parametrize("precision", [0, 1])
def test_reduced_term_list_gives_the_oracle_y(snapmod, twojmax, precision):
    rng = np.random.default_rng(700 + twojmax)
    beta = inputs.beta(twojmax, seed=11 + twojmax)
    h = symmetric_u(snapmod, twojmax, rng)
    U = half_to_full(h[None], twojmax, snapmod.half_index)[0]
    _, Yo = O.energy_from_u(twojmax, beta, U, want_Y=True)
    y = snapmod.yi_host(twojmax, beta, h, precision=precision)
    yc = y[:, 0] + 1j * y[:, 1]
    scale = np.abs(Yo).max()
    worst = 0.0
    for t in range(twojmax + 1):
        for mb in range(t // 2 + 1):
            for ma in range(t + 1):
                e = snapmod.half_index(twojmax, t, ma, mb)
                if 2 * mb == t and ma > mb:
                    assert yc[e] == 0.0  # skipped: no contraction reads it
                    continue
                worst = max(worst, abs(yc[e] - Yo[full_pos(t, ma, mb)]) / scale)
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("twojmax", [4, 8])
def test_oracle_y_has_the_mirror_the_export_fills_in(twojmax):
    """Y[ma][t/2] = (-1)^(ma + t/2) conj(Y[t-ma][t/2]) below the centre of the
    middle column, for the Y of a U with the inversion symmetry (a physical
    Ulisttot, so the symmetry is the one the library relies on)."""
    cfg = inputs.bcc(2, disp=0.1, seed=71)
    beta = inputs.beta(twojmax, seed=3)
    _, ref = O.evaluate(O.Params(twojmax), beta, cfg.pos, cfg.box, want_UY=True)
    for a in range(3):
        Y = ref.Y[a]
        scale = np.abs(Y).max()
        for t in range(0, twojmax + 1, 2):
            mb = t // 2
            for ma in range(mb + 1, t + 1):
                s = -1.0 if (ma + mb) & 1 else 1.0
                want = s * np.conj(Y[full_pos(t, t - ma, mb)])
                assert abs(Y[full_pos(t, ma, mb)] - want) <= 1e-12 * scale


@pytest.mark.parametrize("twojmax", [2, 5, 8, 10])
@pytest.mark.parametrize("layout", [0, 1])
def test_bispectrum_words_give_the_oracle_b(snapmod, twojmax, layout):
    """The bispectrum kernels' record words (factor offsets, conjugation by
    flag or by the conjugate plane, the step to each group's output element,
    chunks of whole groups), walked on the host, give the oracle's B_l (Eq. z
    with every triple product of the full matrices multiplied out) for a U
    with the inversion symmetry.  The oracle's B_l is its energy with beta the
    l-th unit vector (E is linear in beta, beta_0 = 0)."""
    rng = np.random.default_rng(900 + twojmax)
    h = symmetric_u(snapmod, twojmax, rng)
    U = half_to_full(h[None], twojmax, snapmod.half_index)[0]
    nc = O.ncoeff(twojmax)
    want = np.empty(nc)
    for l in range(nc):
        beta = np.zeros(nc + 1)
        beta[1 + l] = 1.0
        want[l] = O.energy_from_u(twojmax, beta, U)
    got = snapmod.bi_host(twojmax, h, layout=layout)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-12 * scale, np.abs(got - want).max() / scale


def test_bispectrum_words_reject_bad_arguments(snapmod):
    h = np.zeros((snapmod.half_size(4), 2))
    with pytest.raises(snapmod.SnapError):
        snapmod.bi_host(4, h, layout=2)
