"""The per-pair flop counts behind the roofline (``flops.ui_pair``,
``flops.de_pair``) against a counted run of the same algorithm (no GPU).

The run below executes the scaled recursion u = S v (Eq. hysphrecur with the
root factors absorbed in S_t(ma, mb) = sqrt((t-ma)! ma! / (t-mb)!)) on the
half layout, and the reverse pass of the fused dU + dE (Eq. snapforce2 via
the adjoint), with every arithmetic operation tallied under the counting
conventions of ``flops.py``: real add or multiply 1, fused multiply-add 2,
complex multiply 6, complex multiply-accumulate 8, real-by-complex scale 2.
The run is pinned to the oracle before its tally is trusted:
  * forward: S v equals the oracle's u_t (Eq. u) at every half element;
  * reverse: dE/dr of E = f_c Re sum conj(Yw) v equals central differences
    of the same E through the oracle's Cayley-Klein geometry (Sec. II).
A count in ``flops.py`` that drops or adds a term then fails the equality.
compute_Y's count (``flops.yi_atom``) leaves out terms whose Clebsch-Gordan
product vanishes; its exact zero test is pinned to the oracle's CG values.
"""
import math

import numpy as np
import pytest

from oracle import snap_oracle as O
from paper_2011_12875_gb300 import flops


class Tally:
    def __init__(self):
        self.n = 0

    def cmul(self, x, y):          # complex multiply
        self.n += 6
        return x * y

    def cadd(self, x, y):          # complex add or subtract (sign in y)
        self.n += 2
        return x + y

    def scale(self, r, x):         # real-by-complex scale
        self.n += 2
        return r * x

    def cmac(self, acc, x, y):     # complex multiply-accumulate
        self.n += 8
        return acc + x * y

    def redot(self, acc, y, v):    # acc + Re(conj(y) v): two fused multiply-adds
        self.n += 4
        return acc + (y.real * v.real + y.imag * v.imag)


def half(t):
    return [(ma, mb) for mb in range(t // 2 + 1) for ma in range(t + 1)]


def forward(J, a, b, tal, v0, per_elem):
    """Scaled recursion over the half layout; the middle column of each even
    layer t reads the seed: layer t-1's column t/2, the mirror of column
    t/2 - 1 times 1/sqrt(t/2), formed once (t elements)."""
    ca, cb = a.conjugate(), b.conjugate()
    v = [{(0, 0): v0}]
    per_elem(0, (0, 0), v0, layer0=True)
    for t in range(1, J + 1):
        prev = dict(v[t - 1])
        if t % 2 == 0:
            mc, tp = t // 2, t - 1
            q = 1.0 / math.sqrt(mc)
            for m in range(t):
                sig = -q if (m + mc) % 2 else q
                prev[(m, mc)] = tal.scale(sig, v[tp][(tp - m, tp - mc)].conjugate())
        cur = {}
        for ma, mb in half(t):
            x = None
            if ma < t:
                x = tal.cmul(ca, prev[(ma, mb)])
            if ma > 0:
                y = tal.cmul(-cb, prev[(ma - 1, mb)])
                x = y if x is None else tal.cadd(x, y)
            cur[(ma, mb)] = x
            per_elem(t, (ma, mb), x, layer0=False)
        v.append(cur)
    return v


def count_ui(J, a=0.6 + 0.3j, b=0.2 - 0.5j, fc=0.7):
    """compute_U, one pair: f_c carried in v from layer 0, each element
    added to the pair's running sum."""
    tal = Tally()
    acc = {}

    def add(t, e, x, layer0):
        acc[(t, e)] = tal.cadd(acc.get((t, e), 0j), x)

    v = forward(J, a, b, tal, complex(fc), add)
    return tal.n, v


def dE_pair(J, geom, Yw, tal):
    """Fused dU + dE of one pair: forward (v and S = Re sum conj(Yw) v), the
    reverse over layers, and dE/dr_d = dfc_d S + f_c (Re g_a Re da_d +
    Im g_a Im da_d + Re g_b Re db_d + Im g_b Im db_d)."""
    a, b = geom["a"], geom["b"]
    S = [0.0]

    def acc(t, e, x, layer0):
        if layer0:
            S[0] = Yw[0][e].real  # v_0 = 1: no arithmetic
        else:
            S[0] = tal.redot(S[0], Yw[t][e], x)

    v = forward(J, a, b, tal, 1 + 0j, acc)
    lam = dict(Yw[J])
    ga, gb = 0j, 0j
    for t in range(J, 0, -1):
        tp = t - 1
        mc = t // 2
        nl_all = {}
        for m, mb in half(tp):
            u = v[tp][(m, mb)]
            A, B = lam[(m, mb)], lam[(m + 1, mb)]
            ga = tal.cmac(ga, A.conjugate(), u)
            gb = tal.cmac(gb, -B.conjugate(), u)
            nl = tal.cadd(tal.cadd(Yw[tp][(m, mb)], tal.cmul(a, A)), tal.cmul(-b, B))
            if t % 2 == 0 and mb == mc - 1:
                q = 1.0 / math.sqrt(mc)
                sig = -q if (m + mc - 1) % 2 else q
                vm = tal.scale(sig, u.conjugate())
                mp = tp - m
                A2, B2 = lam[(mp, mc)], lam[(mp + 1, mc)]
                ga = tal.cmac(ga, A2.conjugate(), vm)
                gb = tal.cmac(gb, -B2.conjugate(), vm)
                l2 = tal.cadd(tal.cmul(a, A2), tal.cmul(-b, B2))
                nl = tal.cadd(nl, tal.scale(sig, l2.conjugate()))
            nl_all[(m, mb)] = nl
        lam = nl_all
    dedr = np.zeros(3)
    for d in range(3):
        da, db = geom["da"][d], geom["db"][d]
        tal.n += 10
        dedr[d] = geom["dfc"][d] * S[0] + geom["fc"] * (
            ga.real * da.real + ga.imag * da.imag + gb.real * db.real + gb.imag * db.imag)
    return dedr, S[0], v


def scale_S(t, ma, mb):
    f = math.factorial
    return math.sqrt(f(t - ma) * f(ma) / f(t - mb))


def random_Yw(J, rng):
    return [{e: complex(*rng.normal(size=2)) for e in half(t)} for t in range(J + 1)]


@pytest.mark.parametrize("J", range(0, 15))
def test_counted_run_equals_flops_py(J):
    rng = np.random.Generator(np.random.PCG64(100 + J))
    n_ui, _ = count_ui(J)
    assert n_ui == flops.ui_pair(J)
    geom = dict(a=0.6 + 0.3j, b=0.2 - 0.5j, fc=0.7, dfc=np.array([0.1, -0.2, 0.3]),
                da=np.array([0.1 + 0.2j, -0.3j, 0.5]), db=np.array([0.2, 0.1 - 0.1j, -0.4j]))
    tal = Tally()
    dE_pair(J, geom, random_Yw(J, rng), tal)
    assert tal.n == flops.de_pair(J)


@pytest.mark.parametrize("J", [1, 4, 5, 8])
def test_counted_forward_is_the_oracle_u(J):
    """S_t(ma, mb) v_t[ma][mb] is the oracle's u_t[ma][mb] (f_c = 1 here)."""
    p = O.Params(J)
    r = np.array([1.3, -2.1, 1.7])
    u, _, g = O.ulist_pair(p, r)
    _, v = count_ui(J, g["a"], g["b"], 1.0)
    for t in range(J + 1):
        ut = O.block(u, t)
        for (ma, mb), x in v[t].items():
            assert abs(scale_S(t, ma, mb) * x - ut[ma, mb]) < 1e-13, (t, ma, mb)


@pytest.mark.parametrize("J", [2, 5, 8])
def test_counted_reverse_is_the_gradient(J):
    """dE/dr of the counted reverse pass against central differences of
    E(r) = f_c(r) Re sum conj(Yw) v(a(r), b(r)) through the oracle geometry."""
    rng = np.random.Generator(np.random.PCG64(7 + J))
    p = O.Params(J)
    Yw = random_Yw(J, rng)
    r = np.array([1.9, 1.1, -2.4])
    _, _, g = O.ulist_pair(p, r)
    dedr, _, _ = dE_pair(J, g, Yw, Tally())

    def energy(rr):
        _, _, gg = O.ulist_pair(p, rr)
        _, S, _ = dE_pair(J, gg, Yw, Tally())
        return gg["fc"] * S

    h = 1e-5
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (energy(r + e) - energy(r - e)) / (2 * h)
        assert abs(fd - dedr[d]) < 1e-7 * max(1.0, abs(fd)), (d, fd, dedr[d])


def test_y_count_zero_decision_matches_the_oracle_cg():
    """compute_Y's count leaves out terms whose Clebsch-Gordan product
    vanishes; its exact zero test agrees with the oracle's Racah CG (in
    FP64: an accidental zero comes out below 1e-12) on every coefficient
    the 2J <= 14 term lists use."""
    J = 14
    nz = zero = 0
    for t in range(J + 1):
        for t1 in range(J + 1):
            for t2 in range(t1 + 1):
                if not (t1 - t2 <= t <= min(J, t1 + t2)) or (t1 + t2 - t) % 2:
                    continue
                for x1 in range(t1 + 1):
                    for x2 in range(t2 + 1):
                        m = (2 * x1 - t1) + (2 * x2 - t2)
                        if abs(m) > t:
                            continue
                        want = abs(O.cg(t1, 2 * x1 - t1, t2, 2 * x2 - t2, t, m)) > 1e-12
                        assert flops._cg_nonzero(t1, x1, t2, x2, t) == want, (t1, x1, t2, x2, t)
                        nz += want
                        zero += not want
    assert nz > 0 and zero > 0
