"""Pins of the FP64 oracle against what the mathematics fixes (no GPU needed).

The paper (arXiv:2011.12875) prints no worked numerical values, so the oracle
is pinned by closed forms, textbook tables, invariants and finite
differences, each chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import snap_oracle as O
from paper_2011_12875_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.Generator(np.random.PCG64(2024))


def rand_vec(rmax=4.5, rmin=1.0):
    while True:
        v = rng.uniform(-rmax, rmax, 3)
        if rmin < np.linalg.norm(v) < rmax:
            return v


# ---------------------------------------------------------------- CG tables

def test_cg_textbook_values():
    """Spot values from the standard Clebsch-Gordan table (Eq. z couples with them)."""
    n = 0
    with open(os.path.join(GOLDEN, "cg_textbook.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            *ints, expr = line.split()
            t1, m1, t2, m2, t, m = map(int, ints)
            want = eval(expr, {"sqrt": math.sqrt})
            assert O.cg(t1, m1, t2, m2, t, m) == pytest.approx(want, abs=1e-14)
            n += 1
    assert n >= 15


@pytest.mark.parametrize("t1,t2", [(1, 1), (2, 1), (3, 2), (4, 4), (7, 5), (8, 6)])
def test_cg_orthogonality(t1, t2):
    """sum_{m1,m2} <j1m1j2m2|JM><j1m1j2m2|J'M'> = delta_JJ' delta_MM' (unitary)."""
    cols = []
    for t in range(abs(t1 - t2), t1 + t2 + 1, 2):
        for mm in range(-t, t + 1, 2):
            col = np.array([[O.cg(t1, m1, t2, m2, t, mm)
                             for m2 in range(-t2, t2 + 1, 2)] for m1 in range(-t1, t1 + 1, 2)])
            cols.append(col.ravel())
    C = np.array(cols)
    assert C.shape[0] == (t1 + 1) * (t2 + 1)
    np.testing.assert_allclose(C @ C.T, np.eye(C.shape[0]), atol=1e-13)


# ------------------------------------------------- hyperspherical harmonics

@pytest.mark.parametrize("twojmax", [8, 14])
def test_u_unitary(twojmax):
    """Every u_t of a single neighbour is unitary and |a|^2 + |b|^2 = 1."""
    p = O.Params(twojmax)
    for _ in range(3):
        u, _, g = O.ulist_pair(p, rand_vec())
        assert abs(g["a"]) ** 2 + abs(g["b"]) ** 2 == pytest.approx(1.0, abs=1e-15)
        for t in range(twojmax + 1):
            m = O.block(u, t)
            np.testing.assert_allclose(m @ m.conj().T, np.eye(t + 1), atol=2e-13)


def sym_power(g2, t):
    """Closed form of the spin-t/2 representation: the action of the 2x2 matrix
    g2 on homogeneous polynomials of degree t in (x, y), in the orthonormal
    basis sqrt(C(t,m)) x^(t-m) y^m.  Written independently of the oracle."""
    out = np.zeros((t + 1, t + 1), dtype=complex)
    gx = np.array([g2[0, 0], g2[1, 0]])   # image of x: coefficients of (x, y)
    gy = np.array([g2[0, 1], g2[1, 1]])   # image of y
    for mb in range(t + 1):
        poly = np.array([1.0 + 0j])        # coefficients in powers of y (x implicit)
        for _ in range(t - mb):
            poly = np.convolve(poly, gx)
        for _ in range(mb):
            poly = np.convolve(poly, gy)
        for ma in range(t + 1):
            out[ma, mb] = poly[ma] * math.sqrt(math.comb(t, mb) / math.comb(t, ma))
    return out


@pytest.mark.parametrize("t", [1, 2, 3, 4, 5, 6, 8])
def test_u_closed_form(t):
    """The layer recursion reproduces the symmetric power of u_1 (Wigner's
    closed form for SU(2) in Cayley-Klein parameters), and u_1 = [[a*, b], [-b*, a]]."""
    p = O.Params(max(t, 1))
    for _ in range(3):
        u, _, g = O.ulist_pair(p, rand_vec())
        a, b = g["a"], g["b"]
        u1 = np.array([[np.conj(a), b], [-np.conj(b), a]])
        np.testing.assert_allclose(O.block(u, 1), u1, atol=1e-15)
        np.testing.assert_allclose(O.block(u, t), sym_power(u1, t), atol=1e-13)


def test_u_homomorphism():
    """u_t(g1) u_t(g2) = u_t(g1 g2): the recursion yields a representation."""
    t = 6
    p = O.Params(t)
    u_a, _, ga = O.ulist_pair(p, rand_vec())
    u_b, _, gb = O.ulist_pair(p, rand_vec())
    m = lambda g: np.array([[np.conj(g["a"]), g["b"]], [-np.conj(g["b"]), g["a"]]])
    prod = m(ga) @ m(gb)
    np.testing.assert_allclose(O.block(u_a, t) @ O.block(u_b, t), sym_power(prod, t), atol=1e-13)


def test_ck_derivatives_fd():
    """da/dr, db/dr, df_c/dr and du/dr against central differences."""
    p = O.Params(6)
    r = rand_vec(4.6, 2.0)
    u, du, g = O.ulist_pair(p, r, with_du=True)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        up, _, gp = O.ulist_pair(p, r + e)
        um, _, gm = O.ulist_pair(p, r - e)
        assert (gp["a"] - gm["a"]) / (2 * h) == pytest.approx(g["da"][d], abs=1e-8)
        assert (gp["b"] - gm["b"]) / (2 * h) == pytest.approx(g["db"][d], abs=1e-8)
        assert (gp["fc"] - gm["fc"]) / (2 * h) == pytest.approx(g["dfc"][d], abs=1e-8)
        np.testing.assert_allclose((up - um) / (2 * h), du[d], atol=2e-7)


# ---------------------------------------------------------- bispectrum / E

def unit_beta(twojmax, l):
    b = np.zeros(O.ncoeff(twojmax) + 1)
    b[1 + l] = 1.0
    return b


@pytest.mark.parametrize("twojmax", [4, 7])
def test_single_rotation_bispectrum(twojmax):
    """For U = u(g) of ONE rotation, the CG product of u_j1 and u_j2 is u_j, so
    B_{j1j2j} = u_j : u_j^* = 2j + 1 for every component.  Pins the CG
    coefficients, their index pairing in Eq. (z) and the recursion jointly."""
    p = O.Params(twojmax)
    u, _, _ = O.ulist_pair(p, rand_vec())
    tr = O.triples(twojmax)
    for l in range(len(tr)):
        B = O.energy_from_u(twojmax, unit_beta(twojmax, l), u)
        assert B == pytest.approx(tr[l, 2] + 1, abs=1e-11), tuple(tr[l])


def test_ncoeff():
    """0 <= 2j2 <= 2j1 <= 2j <= 2J gives 55 components at 2J = 8, 204 at 2J = 14
    (Sec. II-C)."""
    assert O.ncoeff(8) == 55 and O.ncoeff(14) == 204
    assert inputs.ncoeff(8) == 55 and inputs.ncoeff(14) == 204


def cluster(n=9, seed=7, spread=3.0):
    """Isolated cluster (huge box: no periodic images)."""
    g = np.random.Generator(np.random.PCG64(seed))
    while True:
        pos = g.uniform(0, spread, (n, 3)) + 50.0
        d = np.linalg.norm(pos[:, None] - pos[None], axis=-1) + 10 * np.eye(n)
        if d.min() > 1.4:
            return pos, np.array([200.0, 200.0, 200.0])


def test_twojmax0_closed_form():
    """2J = 0: U_0 = 1 + sum f_c, B_000 = U_0^3, E = beta0 + beta1 U_0^3 and
    dE_i/dr_ik = 3 beta1 U_0^2 df_c/dr r_hat."""
    p = O.Params(0)
    pos, box = cluster()
    beta = np.array([0.3, -0.7])
    pairs, res = O.evaluate(p, beta, pos, box)
    r = np.linalg.norm(pairs.rij, axis=1)
    w = np.pi * r / p.rcut
    fc = 0.5 * (np.cos(w) + 1.0)
    dfc = -0.5 * np.pi / p.rcut * np.sin(w)
    U0 = 1.0 + np.bincount(pairs.i, weights=fc, minlength=len(pos))
    np.testing.assert_allclose(res.E, beta[0] + beta[1] * U0 ** 3, rtol=1e-13)
    want = (3 * beta[1] * U0[pairs.i] ** 2 * dfc / r)[:, None] * pairs.rij
    np.testing.assert_allclose(res.dedr, want, rtol=1e-12, atol=1e-14)


def random_rotation(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("twojmax", [5, 8])
def test_rotation_translation_invariance(twojmax):
    """B and E_i are invariant and F rotates with the cluster."""
    p = O.Params(twojmax)
    pos, box = cluster()
    beta = inputs.beta(twojmax)
    c = pos.mean(0)
    _, r0 = O.evaluate(p, beta, pos, box, want_B=True)
    R = random_rotation(11)
    pos_r = (pos - c) @ R.T + c + np.array([1.3, -0.4, 2.2])
    _, r1 = O.evaluate(p, beta, pos_r, box, want_B=True)
    np.testing.assert_allclose(r1.B, r0.B, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(r1.E, r0.E, rtol=1e-12)
    np.testing.assert_allclose(r1.F, r0.F @ R.T, atol=1e-10 * np.abs(r0.F).max())


def fd_derivative(f, h):
    """Five-point central difference: exact for polynomials up to degree 4."""
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


@pytest.mark.parametrize("twojmax", [2, 3, 4])
def test_adjoint_matches_energy_gradient(twojmax):
    """Y (Eq. y) equals dE/dRe U + i dE/dIm U, entry by entry, at a Ulisttot of
    several neighbours.  E is cubic in U, so the five-point difference is exact."""
    p = O.Params(twojmax)
    pos, box = cluster()
    beta = inputs.beta(twojmax)
    _, res = O.evaluate(p, beta, pos, box, want_UY=True)
    U = res.U[0].copy()
    E0, Y = O.energy_from_u(twojmax, beta, U, want_Y=True)
    assert E0 == pytest.approx(res.E[0], rel=1e-13)
    np.testing.assert_allclose(Y, res.Y[0], atol=1e-12)
    scale = np.abs(Y).max()
    for e in range(len(U)):
        for unit in (1.0, 1j):
            def f(h):
                V = U.copy()
                V[e] += unit * h
                return O.energy_from_u(twojmax, beta, V)
            g = fd_derivative(f, 1e-3)
            want = Y[e].real if unit == 1.0 else Y[e].imag
            assert g == pytest.approx(want, abs=1e-9 * scale), (e, unit)


@pytest.mark.parametrize("twojmax", [4, 8])
def test_euler_identity_and_symmetry(twojmax):
    """E - beta0 is a cubic form in U, so Re sum conj(Y) U = 3 (E - beta0);
    Y carries the same inversion symmetry as U."""
    p = O.Params(twojmax)
    pos, box = cluster()
    beta = inputs.beta(twojmax)
    _, res = O.evaluate(p, beta, pos, box, want_UY=True)
    for i in range(3):
        lhs = np.real(np.sum(np.conj(res.Y[i]) * res.U[i]))
        assert lhs == pytest.approx(3 * (res.E[i] - beta[0]), rel=1e-12)
        for t in range(twojmax + 1):
            for M in (O.block(res.U[i], t), O.block(res.Y[i], t)):
                sgn = np.array([[(-1) ** (a + b) for b in range(t + 1)] for a in range(t + 1)])
                np.testing.assert_allclose(M[::-1, ::-1], sgn * np.conj(M), atol=1e-11 * (1 + np.abs(M).max()))


def test_linear_in_beta():
    """E is affine and F linear in beta (exact up to rounding)."""
    p = O.Params(6)
    cfg = inputs.bcc(2, disp=0.1)
    b1 = inputs.beta(6, seed=1)
    b2 = inputs.beta(6, seed=2)
    _, r1 = O.evaluate(p, b1, cfg.pos, cfg.box, want_B=True)
    _, r2 = O.evaluate(p, b2, cfg.pos, cfg.box)
    _, r12 = O.evaluate(p, b1 + b2, cfg.pos, cfg.box)
    np.testing.assert_allclose(r12.E, r1.E + r2.E, rtol=1e-12)
    np.testing.assert_allclose(r12.F, r1.F + r2.F, atol=1e-11 * np.abs(r12.F).max())
    np.testing.assert_allclose(r1.E, b1[0] + r1.B @ b1[1:], rtol=1e-12)


def total_energy(p, beta, pos, box):
    _, r = O.evaluate(p, beta, pos, box)
    return r.E.sum()


@pytest.mark.parametrize("ncell,twojmax", [(2, 8), (3, 6)])
def test_forces_are_minus_energy_gradient(ncell, twojmax):
    """F = -dE_total/dr by central differences (h = 1e-5 A) in a periodic box
    smaller than 2 rcut (several images of one atom are neighbours); sum F = 0."""
    p = O.Params(twojmax)
    cfg = inputs.bcc(ncell, disp=0.15, seed=99)
    beta = inputs.beta(twojmax)
    _, r = O.evaluate(p, beta, cfg.pos, cfg.box)
    scale = np.abs(r.F).max()
    np.testing.assert_allclose(r.F.sum(0), 0.0, atol=1e-11 * scale * len(cfg.pos))
    h = 1e-5
    for a in (0, 3, len(cfg.pos) - 1):
        for d in range(3):
            def f(s):
                q = cfg.pos.copy()
                q[a, d] += s
                return total_energy(p, beta, q, cfg.box)
            fd = -(f(h) - f(-h)) / (2 * h)
            assert fd == pytest.approx(r.F[a, d], abs=2e-6 * scale), (a, d)


def test_virial_is_strain_derivative():
    """W_ab = -dE/d(eps_ab) under r -> (I + eps) r: all nine components on an
    isolated cluster, the diagonal ones in a periodic box (box scales too)."""
    p = O.Params(6)
    beta = inputs.beta(6)
    h = 1e-6
    pos, box = cluster()
    _, r = O.evaluate(p, beta, pos, box)
    W = r.W
    full = np.array([[W[0], W[3], W[4]], [W[3], W[1], W[5]], [W[4], W[5], W[2]]])
    scale = np.abs(W).max()
    for a in range(3):
        for b in range(3):
            def f(s):
                eps = np.eye(3)
                eps[a, b] += s
                return total_energy(p, beta, pos @ eps.T, box)
            fd = -(f(h) - f(-h)) / (2 * h)
            assert fd == pytest.approx(full[a, b], abs=1e-6 * scale), (a, b)
    cfg = inputs.bcc(2, disp=0.1)
    _, r = O.evaluate(p, beta, cfg.pos, cfg.box)
    for a in range(3):
        def f(s):
            sc = np.ones(3)
            sc[a] += s
            return total_energy(p, beta, cfg.pos * sc, cfg.box * sc)
        fd = -(f(h) - f(-h)) / (2 * h)
        assert fd == pytest.approx(r.W[a], abs=1e-6 * np.abs(r.W).max()), a


def test_perfect_lattice():
    """Ideal BCC: 26 neighbours each, all E_i equal, all forces zero."""
    p = O.Params(8)
    cfg = inputs.bcc(3, disp=0.0)
    pairs, r = O.evaluate(p, inputs.beta(8), cfg.pos, cfg.box)
    assert np.all(np.bincount(pairs.i) == 26)
    assert np.ptp(r.E) < 1e-11 * np.abs(r.E).max()
    assert np.abs(r.F).max() < 1e-10 * np.abs(r.E).max()


def test_neighbor_list_brute_force():
    """The oracle's image enumeration matches a direct numpy enumeration on a
    box smaller than 2 rcut (54 atoms, L = 9.54 A)."""
    cfg = inputs.bcc(3, disp=0.1, strain=0.02, seed=5)
    pairs = O.build_neighbors(cfg.pos, cfg.box, inputs.RCUT)
    got = set()
    for q in range(len(pairs.i)):
        got.add((pairs.i[q], pairs.k[q], *pairs.img[q]))
    want = set()
    rng_s = range(-2, 3)
    for i in range(cfg.natoms):
        for k in range(cfg.natoms):
            for s in np.array(np.meshgrid(rng_s, rng_s, rng_s)).reshape(3, -1).T:
                if i == k and not s.any():
                    continue
                if np.linalg.norm(cfg.pos[k] + s * cfg.box - cfg.pos[i]) < inputs.RCUT:
                    want.add((i, k, *s))
    assert got == want


def test_oracle_flop_counter_walks_the_nonzero_cg_terms():
    """orc_flops counts 47 flops per nonzero term of the oracle's triple
    products: the number of terms with both Clebsch-Gordan factors nonzero,
    counted here with sympy's CG (an independent routine), for 2J up to 4;
    and the recursion's terms (two per element but the edges) for U and dU."""
    sympy = pytest.importorskip("sympy")
    from sympy.physics.quantum.cg import CG
    from sympy import Rational as Q
    for J in range(0, 5):
        nterm = 0
        for t1 in range(J + 1):
            for t2 in range(t1 + 1):
                for t in range(t1 - t2, min(J, t1 + t2) + 1, 2):
                    if t < t1:
                        continue
                    nz = {}
                    for x1 in range(t1 + 1):
                        for x2 in range(t2 + 1):
                            m = (2 * x1 - t1) + (2 * x2 - t2)
                            if abs(m) > t:
                                continue
                            v = CG(Q(t1, 2), Q(2 * x1 - t1, 2), Q(t2, 2), Q(2 * x2 - t2, 2), Q(t, 2), Q(m, 2)).doit()
                            nz[(x1, x2)] = v != 0
                    good = [k for k, v in nz.items() if v]
                    nterm += len(good) ** 2
        rec = sum((ma < t) + (ma > 0) for t in range(1, J + 1) for mb in range(t) for ma in range(t + 1))
        nfull = sum((t + 1) ** 2 for t in range(J + 1))
        f = O.flops(J)
        assert f["y_b_atom"] == 47 * nterm, J
        assert f["compute_u_pair"] == 12 * rec + 4 * nfull
        assert f["du_de_pair"] == 12 * rec + 54 * rec + 30 * nfull


def z_full(t1, t2, t, Ua, Ub):
    """Z^t_{t1 t2}[ma][mb] = sum CG CG Ua_t1[ma1][mb1] Ub_t2[ma2][mb2]
    (Eq. z), full matrices, written out here on its own."""
    dl = (t1 + t2 - t) // 2
    A, Bm = O.block(Ua, t1), O.block(Ub, t2)
    Z = np.zeros((t + 1, t + 1), dtype=complex)
    for ma in range(t + 1):
        for mb in range(t + 1):
            s = 0j
            for ma1 in range(max(0, ma + dl - t2), min(t1, ma + dl) + 1):
                ma2 = ma + dl - ma1
                ca = O.cg(t1, 2 * ma1 - t1, t2, 2 * ma2 - t2, t, 2 * ma - t)
                for mb1 in range(max(0, mb + dl - t2), min(t1, mb + dl) + 1):
                    mb2 = mb + dl - mb1
                    cb = O.cg(t1, 2 * mb1 - t1, t2, 2 * mb2 - t2, t, 2 * mb - t)
                    s += ca * cb * A[ma1, mb1] * Bm[ma2, mb2]
            Z[ma, mb] = s
    return Z


@pytest.mark.parametrize("twojmax", [2, 4])
def test_direct_db_route_gives_the_adjoint_forces(twojmax):
    """The second route of the forces (Eq. dbidrk): dB_l^i/dr_ik by the
    product rule on B_l = Re Z : conj(U) with dU of the one pair, then
    dE_i/dr_ik = sum_l beta_l dB_l^i/dr_ik.  It equals the oracle's adjoint
    dE_i/dr_ik (Eq. snapforce2, through Y) pair by pair, and dB agrees with
    central differences of the oracle's B in the pair's separation."""
    p = O.Params(twojmax)
    cfg = inputs.bcc(2, disp=0.15, seed=31)
    beta = inputs.beta(twojmax)
    pairs = O.build_neighbors(cfg.pos, cfg.box, p.rcut)
    n = cfg.natoms
    res = O.compute(p, beta, n, pairs, want_UY=True, want_B=True)
    tr = O.triples(twojmax)
    i = 3
    Ui = res.U[i]
    for q in np.flatnonzero(pairs.i == i)[:6]:
        u, du, g = O.ulist_pair(p, pairs.rij[q], with_du=True)
        dB = np.zeros((len(tr), 3))
        for d in range(3):
            dU = g["dfc"][d] * u + g["fc"] * du[d]
            for l, (t1, t2, t) in enumerate(tr):
                Z = z_full(t1, t2, t, Ui, Ui)
                dZ = z_full(t1, t2, t, dU, Ui) + z_full(t1, t2, t, Ui, dU)
                dB[l, d] = np.real(np.sum(dZ * np.conj(O.block(Ui, t))) +
                                   np.sum(Z * np.conj(O.block(dU, t))))
        dE = beta[1:] @ dB
        scale = max(1.0, np.abs(res.dedr).max())
        np.testing.assert_allclose(dE, res.dedr[q], rtol=0, atol=1e-11 * scale)
        # dB against central differences of the oracle's B_l^i
        need = np.zeros(n, dtype=bool)
        need[i] = True
        h = 1e-5
        for d in range(3):
            Bpm = []
            for sgn in (1.0, -1.0):
                rij = pairs.rij.copy()
                rij[q, d] += sgn * h
                moved = O.Pairs(pairs.i, pairs.k, pairs.img, rij)
                Bpm.append(O.compute(p, beta, n, moved, need=need, want_B=True).B[i])
            fd = (Bpm[0] - Bpm[1]) / (2 * h)
            np.testing.assert_allclose(dB[:, d], fd, rtol=0, atol=1e-7 * max(1.0, np.abs(fd).max()))


@pytest.mark.parametrize("twojmax", [3, 8])
def test_isolated_cluster_has_no_net_force_or_torque(twojmax):
    """The energy of an isolated cluster is invariant under translation and
    rotation, so the forces sum to zero and so do their torques r x F."""
    p = O.Params(twojmax)
    pos, box = cluster()
    _, r = O.evaluate(p, inputs.beta(twojmax), pos, box)
    scale = np.abs(r.F).max() * len(pos)
    assert scale > 0
    np.testing.assert_allclose(r.F.sum(0), 0.0, atol=1e-12 * scale)
    c = pos - pos.mean(0)
    torque = np.cross(c, r.F).sum(0)
    np.testing.assert_allclose(torque, 0.0, atol=1e-12 * scale * np.abs(c).max())
