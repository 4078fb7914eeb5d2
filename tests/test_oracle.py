"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle against something other than itself: a published
closed form, a symmetry of the S-matrix, an independent brute-force
computation, or a count printed in the paper (tests/golden).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_form, color, topology
from paper_2510_05392_gb300 import phasespace as ps

GS = math.sqrt(4 * math.pi * 0.118)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_complexity.json")


def _events(ng, nevt, seed, sqrts=1500.0):
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    return ps.generate(nevt, ng, sqrts, seed, **kw)


# ---------------------------------------------------------------- colour ----

def test_color_matrix_two_gluons_closed_form():
    # C_F^2 N = 16/3 on the diagonal, (C_F - C_A/2) C_F N = -2/3 off it
    Chat, D, perms = color.color_matrix(2)
    assert D == 3
    assert Chat == [[16, -2], [-2, 16]]
    assert perms == [(0, 1), (1, 0)]


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_color_matrix_trace_pin(n):
    # Tr C = n! C_F^n N: every diagonal entry is Tr(t^a1..t^an t^an..t^a1)
    from fractions import Fraction
    Chat, D, _ = color.color_matrix(n)
    assert Fraction(sum(Chat[i][i] for i in range(len(Chat))), D) == \
        math.factorial(n) * 3 * Fraction(4, 3) ** n


def _gell_mann():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / math.sqrt(3)
    l[7][2, 2] = -2 / math.sqrt(3)
    return l / 2


@pytest.mark.parametrize("n", [2, 3, 4])
def test_color_matrix_brute_force_traces(n):
    """Sum explicit Gell-Mann generators over every colour index."""
    t = _gell_mann()
    perms = color.gluon_orderings(n)
    rows = []
    for s in perms:
        # T_s[a_1..a_n] = t^{a_s1} ... t^{a_sn} for every assignment of a's
        acc = None
        for pos in range(n):
            g = s[pos]
            shape = [1] * n + [3, 3]
            shape[g] = 8
            tg = t.reshape(shape)
            acc = tg if acc is None else np.einsum("...ij,...jk->...ik", acc, tg)
        acc = np.broadcast_to(acc, [8] * n + [3, 3])
        rows.append(acc.reshape(-1))
    T = np.array(rows)
    C_bf = (T.conj() @ T.T)
    assert np.abs(C_bf.imag).max() < 1e-12
    Chat, D, p2 = color.color_matrix(n)
    assert list(p2) == list(perms)
    np.testing.assert_allclose(C_bf.real, np.array(Chat) / D, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_color_matrix_symmetric_psd(n):
    Chat, D, _ = color.color_matrix(n)
    C = np.array(Chat, dtype=float)
    assert np.array_equal(C, C.T)
    assert np.linalg.eigvalsh(C).min() > -1e-9 * np.abs(C).max()


# ------------------------------------------------------------ diagrams -----

@pytest.mark.parametrize("n", [3, 4, 5])
def test_color_matrix_relabelling_equals_entrywise(n):
    """The n! -trace construction used beyond 6 gluons reproduces the
    entry-by-entry trace evaluation exactly."""
    full, D, _ = color.color_matrix(n)
    rel, D2, _ = color.color_matrix_relabelled(n)
    assert D == D2
    assert np.array_equal(np.array(full, dtype=np.int64), rel)


def test_color_matrix_seven_gluons():
    """2 -> 7 (5040 flows): symmetric, and every diagonal entry is the
    textbook sum over colours of |(t^a1 ... t^a7)_ij|^2 = N C_F^7."""
    from fractions import Fraction
    Chat, D, perms = color.color_matrix(7)
    assert Chat.shape == (5040, 5040) and len(perms) == 5040
    assert np.array_equal(Chat, Chat.T)
    diag = np.diag(Chat)
    assert (diag == diag[0]).all()
    assert Fraction(int(diag[0]), D) == 3 * Fraction(4, 3) ** 7


def test_counts_against_paper_table():
    g = json.load(open(GOLDEN))["processes"]
    for proc, row in g.items():
        n = oracle.ngluons(proc)
        assert len(color.gluon_orderings(n)) == row["colors"]
        assert 2 ** (n + 2) == row["helicities"]
        if n <= 6:
            assert topology.count_diagrams(n) == row["diagrams"], proc


# ------------------------------------------------------- matrix elements ---

def test_closed_form_ggtt_zero_width():
    p = _events(0, 256, 101, sqrts=1000.0)
    a = oracle.me(p, wt=0.0)
    b = closed_form.ggqq_averaged(p, 173.0, GS)
    # both sides round differently; near-collinear tops amplify it to ~1e-13
    assert np.abs(a / b - 1).max() < 1e-12
    assert np.median(np.abs(a / b - 1)) < 1e-14


def test_closed_form_massless_limit():
    # m -> 0 reduces Combridge to the textbook g g -> q qbar result
    p = ps.generate(64, 0, 1000.0, 5, mt=0.0)
    # put the final state exactly on the light cone (RAMBO leaves p^2 ~ 1e-10)
    p[:, 2:, 0] = np.sqrt((p[:, 2:, 1:] ** 2).sum(-1))
    a = oracle.me(p, mt=0.0, wt=0.0)
    s = 2 * (p[:, 0, 0] * p[:, 1, 0] - (p[:, 0, 1:] * p[:, 1, 1:]).sum(1))
    t = -2 * (p[:, 0, 0] * p[:, 2, 0] - (p[:, 0, 1:] * p[:, 2, 1:]).sum(1))
    u = -2 * (p[:, 1, 0] * p[:, 2, 0] - (p[:, 1, 1:] * p[:, 2, 1:]).sum(1))
    textbook = GS ** 4 * ((t * t + u * u) / (6 * t * u) - 3 * (t * t + u * u) / (8 * s * s))
    # t = -2 p1.p3 loses digits as s/|t| grows (near-collinear events): scale the bound
    cond = s / np.minimum(np.abs(t), np.abs(u))
    assert np.all(np.abs(a / textbook - 1) < 1e-13 * cond)
    assert np.median(np.abs(a / textbook - 1)) < 1e-14


def _mdot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


@pytest.mark.parametrize("ng", [0, 1, 2, 3, 4, 5])
def test_parke_taylor_massless_quark_line(ng):
    """Massless limit (m_t = Gamma_t = 0) of every colour-ordered amplitude
    against the Parke-Taylor formula for a quark pair and n gluons (Berends and
    Giele 1987; Mangano and Parke, Phys. Rep. 200 (1991) 301), up to 7 gluons.

    All particles are taken outgoing: incoming momenta k = -p, incoming
    helicities flipped.  The flow (t^s1 ... t^sn)_{i_t, i_tbar} belongs to the
    cyclic order tbar, t, g_s1, ..., g_sn.  Where exactly one gluon j has the
    helicity of one member f of the (opposite-helicity) quark pair and every
    other gluon the opposite one (MHV and its parity conjugate),
        |A_s|^2 = 2^n s_fj^3 s_f'j / (s_tbar,t s_t,s1 s_s1,s2 ... s_sn,tbar),
    s_ab = |2 k_a.k_b|; the formula is written for generators with
    Tr(T^a T^b) = delta^ab, and the flows here use t^a = T^a / sqrt(2), hence
    2^n.  Quark pairs of equal helicity, and gluons all of one helicity, give
    zero (helicity selection rules).  This fixes the absolute normalisation,
    the phase-free magnitude of each ordering and the orientation of the flows
    for every gluon multiplicity, independently of the width reading."""
    n = ng + 2
    npar = n + 2
    nevt = 2 if ng < 4 else 1
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    p = ps.generate(nevt, ng, 1000.0 if ng < 4 else 2000.0, 800 + ng, mt=0.0, **kw)
    p[:, 2:, 0] = np.sqrt((p[:, 2:, 1:] ** 2).sum(-1))      # exactly on the light cone
    _, _, perms = oracle.color_data(n)
    glu = np.array([0, 1] + list(range(4, npar)))            # particle index of each gluon
    order = glu[np.asarray(perms)]                           # [n!][n] particle indices
    T, TB = 2, 3
    mhv, zero = [], []
    for h in range(1 << npar):
        lam = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
        out = [-l if i < 2 else l for i, l in enumerate(lam)]
        neg = [g for g in glu if out[g] < 0]
        pos = [g for g in glu if out[g] > 0]
        if out[T] == out[TB] or not neg or not pos:
            zero.append(h)
        elif len(neg) == 1 or len(pos) == 1:
            j = neg[0] if len(neg) == 1 else pos[0]
            f = T if out[T] == out[j] else TB
            mhv.append((h, j, f, TB if f == T else T))
    assert len(mhv) == (4 if n == 2 else 4 * n)
    if ng >= 4:
        zero = zero[:: max(1, len(zero) // 8)]
    for e in range(nevt):
        k = p[e].copy()
        k[:2] *= -1
        S = np.abs(2 * _mdot(k[:, None, :], k[None, :, :]))
        chain = S[TB, T] * S[T, order[:, 0]] * S[order[:, -1], TB]
        for a in range(n - 1):
            chain = chain * S[order[:, a], order[:, a + 1]]
        scale = 0.0
        for h, j, f, fp in mhv:
            A = oracle.amplitudes(p[e], h, mt=0.0, wt=0.0)
            pt = 2.0 ** n * S[f, j] ** 3 * S[fp, j] / chain
            assert np.abs(np.abs(A) ** 2 / pt - 1).max() < 1e-9, (h, j, f)
            scale = max(scale, np.abs(A).max())
        for h in zero:
            assert np.abs(oracle.amplitudes(p[e], h, mt=0.0, wt=0.0)).max() <= 1e-12 * scale, h


@pytest.mark.parametrize("ng", [0, 1, 2, 3, 4, 5])
def test_gauge_invariance_every_ordering(ng):
    """eps_i -> k_i makes every colour-ordered amplitude vanish (zero width);
    up to 7 gluons (5040 orderings)."""
    n = ng + 2
    p = _events(ng, 2 if ng < 4 else 1, 200 + ng, 1500.0 if ng < 4 else 2000.0)
    nhel = 1 << (n + 2)
    for e in range(len(p)):
        # scale: the largest amplitude of this event over the helicities (a
        # strided subset of them beyond 5 gluons)
        hs = range(0, nhel, 1 if ng < 4 else 16)
        ref = max(np.abs(oracle.amplitudes(p[e], h, wt=0.0)).max() for h in hs)
        for h in sorted({0, 1, nhel // 3, nhel - 1}):
            for leg in range(n):
                ip = leg if leg < 2 else leg + 2
                g = oracle.amplitudes(p[e], h, gauge_leg=leg, wt=0.0)
                assert np.abs(g).max() / p[e, ip, 0] <= 1e-10 * ref


def _boost(beta):
    beta = np.asarray(beta, float)
    b2 = beta @ beta
    g = 1 / math.sqrt(1 - b2)
    L = np.eye(4)
    L[0, 0] = g
    L[0, 1:] = L[1:, 0] = g * beta
    L[1:, 1:] += (g - 1) * np.outer(beta, beta) / b2
    return L


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_lorentz_invariance_zero_width(ng):
    p = _events(ng, 4 if ng < 3 else 2, 300 + ng)
    rng = np.random.default_rng(ng)
    m = oracle.me(p, wt=0.0)
    for _ in range(2):
        beta = rng.uniform(-0.5, 0.5, 3)
        L = _boost(beta)
        # also rotate: random orthogonal 3x3
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        R = np.eye(4)
        R[1:, 1:] = q * np.sign(np.linalg.det(q))
        pb = p @ (L @ R).T
        mb = oracle.me(pb, wt=0.0)
        assert np.abs(mb / m - 1).max() < 1e-11


@pytest.mark.parametrize("ng", [1, 2, 3])
def test_bose_symmetry_with_width(ng):
    p = _events(ng, 4 if ng < 3 else 2, 400 + ng)
    m = oracle.me(p)
    sw = p[:, [1, 0, 2, 3] + list(range(4, 4 + ng))]
    assert np.abs(oracle.me(sw) / m - 1).max() < 1e-12
    for perm in list(itertools.permutations(range(4, 4 + ng)))[1:3]:
        q = p[:, [0, 1, 2, 3] + list(perm)]
        assert np.abs(oracle.me(q) / m - 1).max() < 1e-12


def test_bose_symmetry_seven_gluons():
    """g g -> t t~ + 5 g: exchanging the incoming gluons or two final gluons
    leaves |M|^2 unchanged (one event, about 15 s of oracle time)."""
    p = ps.generate(1, 5, 2000.0, 424242, ptmin=20.0, drmin=0.4)
    m = oracle.me(p)
    assert m[0] > 0
    assert abs(oracle.me(p[:, [1, 0] + list(range(2, 9))])[0] / m[0] - 1) < 1e-12
    assert abs(oracle.me(p[:, [0, 1, 2, 3, 8, 5, 6, 7, 4]])[0] / m[0] - 1) < 1e-12


def test_helicity_sum_equals_total():
    p = _events(1, 3, 500)
    m, mh = oracle.me(p, per_helicity=True)
    np.testing.assert_allclose(mh.sum(1), m, rtol=1e-14)


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_helicity_mask_all_good(ng):
    # table "complexity": all helicities contribute for these processes
    p = _events(ng, 16, 600 + ng)
    mask = oracle.good_helicity_mask(p)
    assert mask.all()


def test_width_is_a_small_effect():
    p = _events(2, 4, 700)
    r = oracle.me(p) / oracle.me(p, wt=0.0)
    assert np.all(np.abs(r - 1) < 1e-2)
