"""Exact SU(3) colour matrix of the colour-flow basis (oracle; test infrastructure).

Only tests/, the smoke check and the benchmark's CPU-baseline leg use this
module.  It shares nothing with the CUDA path's own colour builder.

Definition (the paper's colour sum, Sec. 3.3, Eq. "jcj": |M|^2 = J^H C J with a
real symmetric colour matrix C over the colour flows):
for the single top line with n gluons, the flows are the strings
(t^{a_s1} ... t^{a_sn})_{i j} for all orderings s of the gluons, and

    C_st = sum over all colour indices of conj((T^s)_ij) (T^t)_ij
         = Tr(t^{a_sn} ... t^{a_s1} t^{a_t1} ... t^{a_tn}).

Each trace is evaluated exactly by the SU(N) Fierz identity
    sum_a t^a_ij t^a_kl = 1/2 (delta_il delta_kj - delta_ij delta_kl / N),
applied to one repeated index at a time:
    Tr(X a Y a Z)        = 1/2 [Tr(Y) Tr(XZ) - Tr(XYZ)/N]
    Tr(X a Y) Tr(Z a W)  = 1/2 [Tr(YXWZ) - Tr(YX) Tr(WZ)/N]
with Tr(empty) = N.  Results are fractions; D is the least common denominator
and C_hat = D C is integer.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from functools import lru_cache

NC = 3


def _canon_word(w):
    """Rotate a cyclic word to its lexicographically smallest rotation."""
    if not w:
        return ()
    return min(tuple(w[i:] + w[:i]) for i in range(len(w)))


def _canon(traces):
    """Canonical form of a product of traces: relabel indices in order of first
    appearance, canonical rotation of each word, sorted word list."""
    # relabel by first appearance over the concatenation (order-dependent but
    # deterministic; memoisation only needs equal inputs to map equally)
    words = [tuple(w) for w in traces if len(w) > 0]
    nempty = sum(1 for w in traces if len(w) == 0)
    relabel = {}
    out = []
    for w in words:
        nw = []
        for x in w:
            if x not in relabel:
                relabel[x] = len(relabel)
            nw.append(relabel[x])
        out.append(_canon_word(tuple(nw)))
    return tuple(sorted(out)), nempty


@lru_cache(maxsize=None)
def _eval(traces) -> Fraction:
    """Value of a product of traces (tuple of non-empty words; every label
    occurs exactly twice in total), summed over all colour labels."""
    if not traces:
        return Fraction(1)
    # pick the first label of the first word
    w0 = traces[0]
    a = w0[0]
    pos = [i for i, x in enumerate(w0) if x == a]
    rest = list(traces[1:])
    half = Fraction(1, 2)
    if len(pos) == 2:
        # same word: w0 = a Y a Z  (X empty after rotation to start at a)
        i, j = pos
        Y = w0[i + 1:j]
        XZ = w0[j + 1:] + w0[:i]
        t1 = [Y, XZ] + rest
        t2 = [w0[:i] + Y + w0[j + 1:]] + rest
        return half * (_val(t1) - _val(t2) / NC)
    # label a appears once in w0 and once in another word
    for k, w1 in enumerate(rest):
        if a in w1:
            break
    else:
        raise ValueError("unpaired colour label")
    others = rest[:k] + rest[k + 1:]
    # Tr(a Y) with X empty (w0 starts with a): Tr(X a Y) = Tr(a Y X)
    Y = w0[1:]
    X = ()
    j = w1.index(a)
    Z, W = w1[:j], w1[j + 1:]
    t1 = [Y + X + W + Z] + others
    t2 = [Y + X, W + Z] + others
    return half * (_val(t1) - _val(t2) / NC)


def _val(traces) -> Fraction:
    words, nempty = _canon(traces)
    return Fraction(NC) ** nempty * _eval(words)


def trace_value(word) -> Fraction:
    """sum over colours of Tr(t^{w0} t^{w1} ...), each label twice."""
    return _val([tuple(word)])


def gluon_orderings(n: int):
    """Colour-flow orderings of n gluons (indices 0..n-1 in particle order
    g1, g2, g5, ...): all permutations, in itertools order."""
    return list(itertools.permutations(range(n)))


def _lex_rank(P):
    """Lexicographic rank of each row of P (permutations of range(n)), i.e.
    its index in itertools.permutations order (Lehmer code)."""
    import numpy as np
    m, n = P.shape
    rank = np.zeros(m, dtype=np.int64)
    used = np.zeros((m, n), dtype=bool)
    rows = np.arange(m)
    for k in range(n):
        smaller_unused = (~used) & (np.arange(n)[None, :] < P[:, k:k + 1])
        rank = rank * (n - k) + smaller_unused.sum(axis=1)
        used[rows, P[:, k]] = True
    return rank


def color_matrix_relabelled(n: int):
    """The same matrix from n! traces instead of (n!)^2.

    The gluon labels are summed dummies, so renaming them by the inverse of
    ordering s leaves C_st unchanged and turns s into the identity:
    C_st = C_(id, r) with r_k = (position of t_k in s).  Returns
    (C_hat int64 array [n!][n!], D, perms).
    """
    import numpy as np
    perms = gluon_orderings(n)
    base = [trace_value(tuple(reversed(range(n))) + tuple(r)) for r in perms]
    D = 1
    for x in base:
        D = D * x.denominator // math.gcd(D, x.denominator)
    base_hat = np.array([int(x * D) for x in base], dtype=np.int64)
    P = np.array(perms, dtype=np.int64)
    m = len(perms)
    Chat = np.empty((m, m), dtype=np.int64)
    for s in range(m):
        pos = np.empty(n, dtype=np.int64)
        pos[P[s]] = np.arange(n)          # pos[a] = position of label a in s
        Chat[s] = base_hat[_lex_rank(pos[P])]
    return Chat, D, perms


def color_matrix(n: int):
    """Exact colour matrix for n gluons.

    Returns (C_hat, D, perms): C_hat (n! x n! integers) with D the common
    denominator (C = C_hat / D), perms the orderings.  Up to 6 gluons every
    entry is its own trace (lists of ints); beyond that the (n!)^2 traces are
    out of reach in Python and the relabelling identity of
    color_matrix_relabelled is used (an int64 array; the identity is checked
    against the entry-by-entry evaluation for small n in the tests).
    """
    if n > 6:
        return color_matrix_relabelled(n)
    perms = gluon_orderings(n)
    m = len(perms)
    C = [[None] * m for _ in range(m)]
    for s in range(m):
        rs = tuple(reversed(perms[s]))
        for t in range(m):
            C[s][t] = trace_value(rs + tuple(perms[t]))
    D = 1
    for row in C:
        for x in row:
            D = D * x.denominator // math.gcd(D, x.denominator)
    Chat = [[int(x * D) for x in row] for row in C]
    return Chat, D, perms
