"""Feynman diagrams of g g -> t t~ + (n-2) g with full-colour QCD vertices.

This is the "Feynman diagrams -> wavefunctions -> amplitudes -> jamps" half of
the paper's method (Sec. 2.2, the sigmaKin / calculate_wavefunctions
structure; Sec. 4.2-4.3 on diagram groups).  Every tree diagram is a top line (ubar(p3) ...
v(p4)) with an ordered sequence of gluon sub-trees attached to it; gluon
sub-trees are built from 3- and 4-gluon vertices.  Sub-trees ("internal
wavefunctions") are shared between diagrams, as in HELAS/ALOHA.

Colour.  Each wavefunction carries a colour operator: a linear combination
of strings of generators t^{a_i}.  With Tr(t^a t^b) = delta^ab/2 and
f^abc t^c = -i [t^a, t^b]:
  3-vertex current (X, Y):   Lorentz V3(X, Y) / P^2, colour -[X, Y]
  4-vertex currents (X,Y,Z): Lorentz L_k / P^2 with colours
      L_1 = (X.Z) Y - (Y.Z) X   colour [[X,Y],Z]
      L_2 = (X.Y) Z - (Y.Z) X   colour [[X,Z],Y]
      L_3 = (X.Y) Z - (X.Z) Y   colour [[Y,Z],X]
  top line with k attachments: ubar B1slash (q1slash+m) B2slash ... Bkslash v
      / prod_j (q_j^2 - m^2 + i m w), colour i^(2k-1) Theta_B1 ... Theta_Bk
(all factors i of vertices and propagators moved into the colour
coefficients, so the Lorentz arithmetic has real scalar factors only).
A diagram's colour expands into strings over all n gluons; each string is a
colour flow ("jamp") and the coefficient is one of +-1, +-i.

Gluon indices 0..n-1 follow particle order (g1, g2, g5, g6, ...).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from functools import lru_cache

# ---------------------------------------------------------------- colour ----
# A colour operator is a dict {string (tuple of gluon indices): complex coeff}
# with coefficients in {+-1, +-i} times small integers.


def c_mul(a: dict, b: dict) -> dict:
    out = {}
    for sa, ca in a.items():
        for sb, cb in b.items():
            s = sa + sb
            out[s] = out.get(s, 0) + ca * cb
    return {s: c for s, c in out.items() if c != 0}


def c_add(*terms) -> dict:
    out = {}
    for coef, op in terms:
        for s, c in op.items():
            out[s] = out.get(s, 0) + coef * c
    return {s: c for s, c in out.items() if c != 0}


def c_comm(a: dict, b: dict) -> dict:
    return c_add((1, c_mul(a, b)), (-1, c_mul(b, a)))


# -------------------------------------------------------- wavefunctions -----

@dataclass(eq=False)
class Current:
    """A gluon wavefunction: external polarisation or off-shell current."""
    idx: int
    gset: frozenset            # gluons it contains
    kind: str                  # 'ext', 'v3', 'v4'
    args: tuple = ()           # child Currents (ordered X, Y[, Z])
    term: int = 0              # 4-vertex structure 1..3
    color: dict = field(default_factory=dict)


@dataclass(eq=False)
class Diagram:
    """Ordered attachments B1..Bk along the top line; one Lorentz term."""
    idx: int                   # diagram-term index
    diagram: int               # diagram index (4-vertex terms share it)
    blocks: tuple              # tuple of Currents
    color: dict                # colour operator over full strings


def _splits2(s):
    """Unordered splits of a frozenset into two non-empty parts (X holds min)."""
    items = sorted(s)
    first, rest = items[0], items[1:]
    for r in range(0, len(rest)):
        for comb in itertools.combinations(rest, r):
            X = frozenset((first,) + comb)
            Y = s - X
            if Y:
                yield X, Y


def _splits3(s):
    """Unordered splits into three non-empty parts, canonically ordered by min."""
    items = sorted(s)
    n = len(items)
    for labels in itertools.product(range(3), repeat=n):
        # canonical: first occurrence order 0, 1, 2
        seen = []
        for l in labels:
            if l not in seen:
                seen.append(l)
        if seen != [0, 1, 2]:
            continue
        parts = [frozenset(x for x, l in zip(items, labels) if l == k) for k in range(3)]
        yield tuple(parts)


class Process:
    """All wavefunctions and diagram terms of g g -> t t~ + (n-2) g."""

    def __init__(self, n: int):
        if n < 2:
            raise ValueError("need at least two gluons")
        self.n = n
        self.npar = n + 2
        self.currents: list[Current] = []
        self._by_set: dict = {}
        self.full = frozenset(range(n))
        for g in range(n):
            c = Current(len(self.currents), frozenset([g]), "ext", (), 0, {(g,): 1})
            self.currents.append(c)
            self._by_set[c.gset] = [c]
        # currents on every proper or full subset, by increasing size
        for size in range(2, n + 1):
            for comb in itertools.combinations(range(n), size):
                self._build(frozenset(comb))
        self.diagrams: list[Diagram] = []
        self.ndiagrams = 0
        self._enumerate_diagrams()

    def _new(self, gset, kind, args, term, color):
        c = Current(len(self.currents), gset, kind, args, term, color)
        self.currents.append(c)
        self._by_set.setdefault(gset, []).append(c)
        return c

    def _build(self, s):
        for X, Y in _splits2(s):
            for cx in self._by_set[X]:
                for cy in self._by_set[Y]:
                    col = c_add((-1, c_comm(cx.color, cy.color)))
                    self._new(s, "v3", (cx, cy), 0, col)
        for X, Y, Z in _splits3(s):
            for cx in self._by_set[X]:
                for cy in self._by_set[Y]:
                    for cz in self._by_set[Z]:
                        a, b, c = cx.color, cy.color, cz.color
                        self._new(s, "v4", (cx, cy, cz), 1, c_comm(c_comm(a, b), c))
                        self._new(s, "v4", (cx, cy, cz), 2, c_comm(c_comm(a, c), b))
                        self._new(s, "v4", (cx, cy, cz), 3, c_comm(c_comm(b, c), a))

    def currents_on(self, s):
        return self._by_set.get(frozenset(s), [])

    def _enumerate_diagrams(self):
        n = self.n
        # ordered set partitions of all gluons into blocks, a tree per block
        def ordered_partitions(rem):
            if not rem:
                yield ()
                return
            items = sorted(rem)
            for r in range(1, len(items) + 1):
                for comb in itertools.combinations(items, r):
                    B = frozenset(comb)
                    for rest in ordered_partitions(rem - B):
                        yield (B,) + rest

        seen_diag = {}
        for parts in ordered_partitions(self.full):
            k = len(parts)
            phase = 1j ** (2 * k - 1)
            for blocks in itertools.product(*[self._by_set[B] for B in parts]):
                col = {(): phase}
                for b in blocks:
                    col = c_mul(col, b.color)
                # diagram identity: blocks with 4-vertex terms collapsed
                key = tuple(_tree_key(b) for b in blocks)
                if key not in seen_diag:
                    seen_diag[key] = len(seen_diag)
                self.diagrams.append(Diagram(len(self.diagrams), seen_diag[key], blocks, col))
        self.ndiagrams = len(seen_diag)

    # ----------------------------------------------------------- stats ----
    def stats(self):
        strings = sum(len(d.color) for d in self.diagrams)
        return dict(n=self.n, ndiagrams=self.ndiagrams, nterms=len(self.diagrams),
                    ncurrents=len(self.currents), jamp_updates=strings)


def _tree_key(c: Current):
    if c.kind == "ext":
        return ("e", min(c.gset))
    return (c.kind,) + tuple(_tree_key(a) for a in c.args)


@lru_cache(maxsize=None)
def process(n: int) -> Process:
    return Process(n)
