"""Exact colour matrix for the CUDA path's colour sum.

The paper's colour sum is the quadratic form J^H C J over the colour flows
(Sec. 3.3, Eq. "jcj"), with C real and symmetric.  For one top line and n
gluons the flows are the generator strings (t^{a_s1}...t^{a_sn})_{ij}, and
C_st = sum over colours of Tr(t^{a_sn}...t^{a_s1} t^{a_t1}...t^{a_tn}).

Evaluation used here: write the trace as a closed chain of 2n generators
with index slots (in_p, out_p) glued out_p = in_{p+1}.  Replacing every
paired product sum_a t^a_{ij} t^a_{kl} by its completeness relation
1/2 (d_il d_kj - d_ij d_kl / N) gives 2^n terms; each term is
(1/2)^n (-1/N)^(#second choices) N^(#index loops), the loops counted with a
union-find over the slots.  Relabelling the summed colour indices shows
C_st depends only on the relative permutation s^-1 t, so only n! traces are
evaluated.  C_hat = D C with D the least common denominator.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

N = 3


def _find(par, x):
    while par[x] != x:
        par[x] = par[par[x]]
        x = par[x]
    return x


def chain_trace(word) -> Fraction:
    """sum over colours of Tr(t^{word[0]} ... t^{word[-1]}); each label twice."""
    L = len(word)
    pos = {}
    for p, a in enumerate(word):
        pos.setdefault(a, []).append(p)
    pairs = list(pos.values())
    if any(len(v) != 2 for v in pairs):
        raise ValueError("every colour label must occur exactly twice")
    total = Fraction(0)
    # slots: in_p = 2p, out_p = 2p+1
    for choice in itertools.product((0, 1), repeat=len(pairs)):
        par = list(range(2 * L))

        def union(a, b):
            ra, rb = _find(par, a), _find(par, b)
            if ra != rb:
                par[ra] = rb

        for p in range(L):
            union(2 * p + 1, 2 * ((p + 1) % L))      # out_p = in_{p+1}
        nsecond = 0
        for (p, q), c in zip(pairs, choice):
            if c == 0:      # d_{in_p out_q} d_{in_q out_p}
                union(2 * p, 2 * q + 1)
                union(2 * q, 2 * p + 1)
            else:           # -1/N d_{in_p out_p} d_{in_q out_q}
                union(2 * p, 2 * p + 1)
                union(2 * q, 2 * q + 1)
                nsecond += 1
        loops = len({_find(par, x) for x in range(2 * L)})
        total += Fraction(-1, N) ** nsecond * Fraction(N) ** loops
    return total / 2 ** len(pairs)


def relative_row(n: int):
    """(row, D): row[k] = D * C_(id, r) for the k-th ordering r in
    itertools.permutations order, so that C_st = row[rank(r)] with
    r_k = (position in s of t_k).  n! traces."""
    perms = list(itertools.permutations(range(n)))
    base = [chain_trace(tuple(reversed(range(n))) + tuple(r)) for r in perms]
    D = 1
    for x in base:
        D = D * x.denominator // math.gcd(D, x.denominator)
    return [int(x * D) for x in base], D


def colour_matrix(n: int):
    """(C_hat rows as ints, D, orderings) for n gluons, orderings in
    itertools.permutations order of range(n)."""
    perms = list(itertools.permutations(range(n)))
    # f(r) for the relative permutation r = s^-1 t: relabel so s = identity
    base = {}
    for r in perms:
        word = tuple(reversed(range(n))) + tuple(r)
        base[r] = chain_trace(word)
    inv = {}
    for s in perms:
        si = [0] * n
        for k, a in enumerate(s):
            si[a] = k
        inv[s] = tuple(si)
    C = []
    for s in perms:
        si = inv[s]
        # C_st = f(r) with r_k = position in s of t_k
        C.append([base[tuple(si[a] for a in t)] for t in perms])
    D = 1
    for row in C:
        for x in row:
            D = D * x.denominator // math.gcd(D, x.denominator)
    return [[int(x * D) for x in row] for row in C], D, perms
