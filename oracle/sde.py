"""Single Feynman diagrams and single-diagram-enhancement weights (oracle).

TEST INFRASTRUCTURE ONLY: tests/ import this module; the library never does.
It shares no code with the CUDA path or with its process compiler.

What it computes.  The paper's process table (table "complexity", row (3))
counts the "SDE channels", the diagrams that MadEvent's single diagram
enhancement uses: 3 / 15 / 105 / 945 for 2 to 5 gluons; its sigmaKin also
takes an event-by-event channel identifier for that algorithm (Sec. 2.2).
Those counts are the tree diagrams built from three-point vertices only
((2n-1)!! for n gluons): a diagram with a four-gluon vertex is no channel.
For channel c the weight of an event is

    w_c = sum_h |D_c,h|^2 / sum_h sum_c' |D_c',h|^2

over the good helicities h and the channels c', with D_c,h the amplitude of
diagram c alone, its colour factor written in the colour-flow basis
(t^{a_s1} ... t^{a_sn})_{i3 j4}, where for one top line and gluons every
entry is 0 or of modulus one (f^abc t^c = -i [t^a, t^b]).  The helicity-
summed |D_c|^2 are MadEvent's multi-channel numerators; their sum over the
channels is the denominator.

Method (plain, slow, FP64).  The diagrams are the labelled trees of the
brute-force enumeration in topology.py that obey the QCD vertex rules.  Each
diagram's value is the product of the textbook full-colour Feynman rules
(metric +---, Feynman gauge, all momenta into a vertex):
  quark-gluon vertex   i g gamma^mu t^a
  3-gluon vertex       g f^abc [g^mn (k-p)^r + g^nr (p-q)^m + g^rm (q-k)^n]
  4-gluon vertex       -i g^2 [f^abe f^cde (g^mr g^ns - g^ms g^nr)
                              + f^ace f^bde (g^mn g^rs - g^ms g^nr)
                              + f^ade f^bce (g^mn g^rs - g^mr g^ns)]
  gluon propagator     -i g_mn delta^ab / k^2
  top propagator       i (qslash + m) / (q^2 - m^2 + i m Gamma)
with g = 1 and the external states of bg.c (oracle.externals), evaluated with
explicit 4x4 gamma matrices.  A four-gluon vertex gives three terms, one per
colour structure.  The colour factor of each term is built from the
Gell-Mann matrices (t^a = lambda^a / 2, f^abc = -2i Tr([t^a, t^b] t^c)) as a
tensor over every colour index and projected onto the colour flows by least
squares.  Summing all terms with their flow coefficients gives the
colour-ordered amplitudes; tests/test_oracle_sde.py checks them against the
Berends-Giele recursion of bg.c.

Colour factors are built for up to 4 gluons (tensors of 8^n * 9 entries).
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

from . import topology

MT, WT = 173.0, 1.4915
MAX_GLUONS = 4

# ------------------------------------------------------------- SU(3) -----


def _gell_mann():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


T = _gell_mann() / 2.0
# f^abc = -2i Tr([t^a, t^b] t^c)
F = -2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T))


# ------------------------------------------------------------ diagrams ---

def _gluon(ip: int) -> int:
    """Gluon index (particle order g1 g2 g5 ...) of particle index ip."""
    return ip if ip < 2 else ip - 2


def _tree_specs(edges, nleaf):
    """The top line of one tree and the gluon sub-tree hanging from each of
    its vertices, from ubar(p3) to v(p4).  A sub-tree is ('e', g),
    ('v3', child, child) or ('v4', child, child, child)."""
    adj = {}
    for u, v in edges:
        adj.setdefault(u, []).append(v)
        adj.setdefault(v, []).append(u)
    # path from the top (leaf 2) to the antitop (leaf 3)
    prev = {2: None}
    todo = [2]
    while todo:
        x = todo.pop()
        for y in adj[x]:
            if y not in prev:
                prev[y] = x
                todo.append(y)
    path = [3]
    while path[-1] != 2:
        path.append(prev[path[-1]])
    path.reverse()

    def sub(w, parent):
        if w < nleaf:
            return ("e", _gluon(w))
        kids = tuple(sub(c, w) for c in adj[w] if c != parent)
        return (("v3",) if len(kids) == 2 else ("v4",)) + kids

    line = []
    for j in range(1, len(path) - 1):
        v = path[j]
        g = [c for c in adj[v] if c not in (path[j - 1], path[j + 1])]
        assert len(g) == 1
        line.append(sub(g[0], v))
    return tuple(line)


def _n_v4(spec) -> int:
    if spec[0] == "e":
        return 0
    return (spec[0] == "v4") + sum(_n_v4(c) for c in spec[1:])


@lru_cache(maxsize=None)
def diagrams(n: int):
    """Every tree diagram of g g -> t t~ + (n-2) g as its top-line sub-trees
    (tuple of specs, see _tree_specs), in the enumeration order of
    topology.py."""
    nleaf = n + 2
    out = []
    for edges in topology._trees(nleaf):
        if topology._is_qcd(edges, nleaf):
            out.append(_tree_specs(edges, nleaf))
    return out


def _terms_of(line):
    """Diagram terms: every choice of colour structure (0, 1, 2) at each
    four-gluon vertex; a term is the line with 'v4' nodes tagged by choice."""
    def alts(spec):
        if spec[0] == "e":
            return [spec]
        kids = [alts(c) for c in spec[1:]]
        out = []
        for combo in itertools.product(*kids):
            if spec[0] == "v3":
                out.append(("v3",) + combo)
            else:
                for k in range(3):
                    out.append(("v4", k) + combo)
        return out
    return [tuple(t) for t in itertools.product(*[alts(s) for s in line])]


# ---------------------------------------------------------------- colour --

def _colour_tensor(n: int, term) -> np.ndarray:
    """Colour factor of a diagram term as a tensor [8]*n + [3, 3] over the
    gluon colours (particle order) and the top / antitop colour indices."""
    ops, subs = [], []
    nxt = [n]

    def new():
        nxt[0] += 1
        return nxt[0] - 1

    def walk(spec):
        if spec[0] == "e":
            return spec[1]
        if spec[0] == "v3":
            a, b = walk(spec[1]), walk(spec[2])
            e = new()
            ops.append(F)
            subs.append([a, b, e])
            return e
        k = spec[1]
        a, b, c = walk(spec[2]), walk(spec[3]), walk(spec[4])
        d, e = new(), new()
        pairs = [((a, b), (c, d)), ((a, c), (b, d)), ((a, d), (b, c))][k]
        ops.extend([F, F])
        subs.extend([[pairs[0][0], pairs[0][1], e], [pairs[1][0], pairs[1][1], e]])
        return d

    labels = [walk(s) for s in term]
    q = [new() for _ in range(len(term) + 1)]
    for j, x in enumerate(labels):
        ops.append(T)
        subs.append([x, q[j], q[j + 1]])
    args = []
    for o, s in zip(ops, subs):
        args += [o, s]
    return np.einsum(*args, list(range(n)) + [q[0], q[-1]], optimize=True)


def flow_orderings(n: int):
    """Colour flows: orderings of the gluons in lexicographic permutation
    order (the order of color.color_matrix)."""
    return list(itertools.permutations(range(n)))


@lru_cache(maxsize=None)
def _flow_basis(n: int):
    rows = []
    for s in flow_orderings(n):
        ops = []
        q = list(range(n, 2 * n + 1))
        for j, g in enumerate(s):
            ops += [T, [g, q[j], q[j + 1]]]
        rows.append(np.einsum(*ops, list(range(n)) + [q[0], q[-1]]).ravel())
    Fm = np.array(rows)                  # [ncolor][8^n * 9]
    sv = np.linalg.svd(Fm, compute_uv=False)
    if sv[-1] < 1e-8 * sv[0]:
        raise RuntimeError("colour flows are not linearly independent")
    return Fm, np.linalg.pinv(Fm.T)      # pinv: [ncolor][8^n * 9]


@lru_cache(maxsize=None)
def terms(n: int):
    """All diagram terms of n gluons: list of (diagram index, term line,
    trivalent (no four-gluon vertex), flow coefficients x [ncolor]) with the
    term's colour factor = sum_s x_s (t^{a_s1}...t^{a_sn})_{i3 j4}; every x_s
    is rounded to 0, +-1 or +-i after checking the projection is exact."""
    if n > MAX_GLUONS:
        raise ValueError(f"colour factors are built for up to {MAX_GLUONS} gluons")
    Fm, pinv = _flow_basis(n)
    out = []
    for d, line in enumerate(diagrams(n)):
        triv = sum(_n_v4(s) for s in line) == 0
        for t in _terms_of(line):
            c = _colour_tensor(n, t).ravel()
            x = pinv @ c
            xr = np.round(x.real) + 1j * np.round(x.imag)
            if np.abs(x - xr).max() > 1e-10 or np.abs(c - Fm.T @ xr).max() > 1e-10:
                raise RuntimeError("colour factor is not a unit-coefficient flow combination")
            if not np.all(np.isin(np.abs(xr), [0.0, 1.0])):
                raise RuntimeError("flow coefficient of modulus other than 0 or 1")
            out.append((d, t, triv, xr))
    return out


# ------------------------------------------------------------- Lorentz ----

_G = np.zeros((4, 4, 4), dtype=complex)   # gamma^mu, chiral representation
_s = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
_G[0][:2, 2:] = _s[0]
_G[0][2:, :2] = _s[0]
for _k in range(1, 4):
    _G[_k][:2, 2:] = _s[_k]
    _G[_k][2:, :2] = -_s[_k]
_METRIC = np.array([1.0, -1.0, -1.0, -1.0])


def _dot(a, b):
    return np.einsum("...m,m,...m->...", a, _METRIC, b)


def _slash(a):
    """a_slash = gamma^mu a_mu for a batch of upper-index vectors [B][4]."""
    return np.einsum("...m,m,mij->...ij", a, _METRIC, _G)


def _current(spec, eps, kin):
    """Off-shell gluon current (propagator included) and incoming momentum of
    a sub-tree for a batch: (J [B][4], K [B][4])."""
    if spec[0] == "e":
        return eps[spec[1]], kin[spec[1]]
    if spec[0] == "v3":
        J1, K1 = _current(spec[1], eps, kin)
        J2, K2 = _current(spec[2], eps, kin)
        W = (_dot(J1, J2)[..., None] * (K1 - K2) + J2 * _dot(K1 + 2 * K2, J1)[..., None]
             - J1 * _dot(2 * K1 + K2, J2)[..., None])
        P = K1 + K2
        return -1j * W / _dot(P, P)[..., None], P
    k = spec[1]
    (J1, K1), (J2, K2), (J3, K3) = [_current(c, eps, kin) for c in spec[2:]]
    d12, d13, d23 = _dot(J1, J2)[..., None], _dot(J1, J3)[..., None], _dot(J2, J3)[..., None]
    S = [d13 * J2 - d23 * J1, d12 * J3 - d23 * J1, d12 * J3 - d13 * J2][k]
    P = K1 + K2 + K3
    return -S / _dot(P, P)[..., None], P


def _term_value(term, eps, kin, ub, v, p3, mt, wt):
    U = ub
    Ksum = 0.0
    for j, spec in enumerate(term):
        J, K = _current(spec, eps, kin)
        U = 1j * np.einsum("bi,bij->bj", U, _slash(J))
        Ksum = Ksum + K
        if j < len(term) - 1:
            q = p3 - Ksum
            M = _slash(q.astype(complex)) + mt * np.eye(4)
            den = _dot(q, q) - mt * mt + 1j * mt * wt
            U = 1j * np.einsum("bi,bij->bj", U, M) / den[:, None]
    return np.einsum("bi,bi->b", U, v)


def _batch(momenta, hels):
    """External states for every (event, helicity) pair, batched."""
    from . import externals
    eps, kin, ub, v, p3 = [], [], [], [], []
    for p in momenta:
        for h in hels:
            e, k, u, w = externals(p, h)
            eps.append(e)
            kin.append(k)
            ub.append(u)
            v.append(w)
            p3.append(p[2])
    eps = np.transpose(np.array(eps), (1, 0, 2))   # [n][B][4]
    kin = np.transpose(np.array(kin), (1, 0, 2))
    return eps, kin, np.array(ub), np.array(v), np.array(p3)


def term_amplitudes(momenta, hels, mt=MT, wt=WT):
    """Values of every diagram term (no couplings) for events [nevt][npar][4]
    and helicity indices: complex [nterms][nevt][len(hels)]."""
    momenta = np.asarray(momenta, dtype=np.float64)
    n = momenta.shape[1] - 2
    eps, kin, ub, v, p3 = _batch(momenta, hels)
    vals = [_term_value(t, eps, kin, ub, v, p3, mt, wt) for _, t, _, _ in terms(n)]
    return np.array(vals).reshape(len(vals), len(momenta), len(hels))


def colour_ordered(momenta, hels, mt=MT, wt=WT):
    """Colour-ordered amplitudes from the diagrams: A_s = sum_t x_t,s L_t,
    complex [nevt][len(hels)][ncolor]."""
    n = np.asarray(momenta).shape[1] - 2
    L = term_amplitudes(momenta, hels, mt, wt)
    X = np.array([x for _, _, _, x in terms(n)])      # [nterms][ncolor]
    return np.einsum("teh,ts->ehs", L, X)


# -------------------------------------------------------------- channels --

def channel_code(x) -> tuple:
    """A channel's colour factor as codes per flow, normalised so that its
    first non-zero coefficient is +1: 0 absent, 1 for +1, 2 for -1, 3 for +i,
    4 for -i."""
    nz = np.flatnonzero(np.abs(x) > 0.5)
    y = x / x[nz[0]]
    code = {1: 1, -1: 2, 1j: 3, -1j: 4}
    return tuple(0 if abs(c) < 0.5 else code[complex(round(c.real), round(c.imag))] for c in y)


@lru_cache(maxsize=None)
def channels(n: int):
    """The single-diagram-enhancement channels of n gluons: the trivalent
    diagrams, ordered by their colour codes (channel_code, lexicographic).
    Returns (term indices into terms(n), codes [nchannel][ncolor] int8)."""
    T_ = terms(n)
    tri = [(channel_code(x), i) for i, (_, _, triv, x) in enumerate(T_) if triv]
    tri.sort()
    keys = [k for k, _ in tri]
    if len(set(keys)) != len(keys):
        raise RuntimeError("two channels share a colour factor")
    return [i for _, i in tri], np.array(keys, dtype=np.int8)


def sde_weights(momenta, hel_mask=None, mt=MT, wt=WT):
    """Channel weights w_c [nevt][nchannel] (channel order of channels(n)),
    summed over the helicities with hel_mask[h] != 0 (all when None)."""
    momenta = np.asarray(momenta, dtype=np.float64)
    n = momenta.shape[1] - 2
    nhel = 1 << (n + 2)
    hels = [h for h in range(nhel) if hel_mask is None or hel_mask[h]]
    idx, _ = channels(n)
    L = term_amplitudes(momenta, hels, mt, wt)[idx]      # [nchannel][nevt][nh]
    num = (np.abs(L) ** 2).sum(axis=2).T                  # [nevt][nchannel]
    return num / num.sum(axis=1, keepdims=True)
