"""Brute-force count of tree Feynman diagrams for g g -> t t~ + (n-2) g (oracle).

Test infrastructure only; independent of the process compiler's own diagram
generator.  The paper's process-complexity table (table "complexity" in
Sec. 3, row "Feynman diagrams") gives 3 / 16 / 123 / 1240 / 15495
diagrams for 2 to 6 gluons, each 4-gluon vertex counted once.

Method: every unrooted tree with labelled leaves and internal vertices of
degree 3 or 4 is generated exactly once by inserting leaves in label order
(a new leaf either subdivides an existing edge or joins an existing degree-3
vertex).  A tree is a QCD diagram when every internal vertex is allowed:
an edge is a top line when exactly one of the two top legs lies on one side
of it, otherwise a gluon line; degree-3 vertices need 0 (ggg) or 2 (t t~ g)
top lines, degree-4 vertices need 0 (gggg).
"""
from __future__ import annotations


def _trees(nleaf: int):
    """Yield edge lists of all trees on leaves 0..nleaf-1 with internal
    vertices of degree 3 or 4 (internal vertices numbered from nleaf)."""
    if nleaf < 3:
        raise ValueError("need at least 3 legs")
    start = [(0, nleaf), (1, nleaf), (2, nleaf)]

    def grow(edges, k, next_node):
        if k == nleaf:
            yield edges
            return
        # subdivide an edge
        for i, (u, v) in enumerate(edges):
            w = next_node
            ne = edges[:i] + edges[i + 1:] + [(u, w), (w, v), (k, w)]
            yield from grow(ne, k + 1, next_node + 1)
        # attach to an internal vertex of degree 3
        deg = {}
        for u, v in edges:
            deg[u] = deg.get(u, 0) + 1
            deg[v] = deg.get(v, 0) + 1
        for c in sorted(deg):
            if c >= nleaf and deg[c] == 3:
                yield from grow(edges + [(k, c)], k + 1, next_node)

    yield from grow(start, 3, nleaf + 1)


def _is_qcd(edges, nleaf, t_leg=2, tb_leg=3):
    adj = {}
    for u, v in edges:
        adj.setdefault(u, []).append(v)
        adj.setdefault(v, []).append(u)

    def side_leaves(u, v):
        # leaves reachable from v without crossing back to u
        seen, stack, out = {u, v}, [v], set()
        while stack:
            x = stack.pop()
            if x < nleaf:
                out.add(x)
            for y in adj[x]:
                if y not in seen:
                    seen.add(y)
                    stack.append(y)
        return out

    for c, nb in adj.items():
        if c < nleaf:
            continue
        nferm = 0
        for v in nb:
            s = side_leaves(c, v)
            if (t_leg in s) != (tb_leg in s):
                nferm += 1
        if len(nb) == 3 and nferm not in (0, 2):
            return False
        if len(nb) == 4 and nferm != 0:
            return False
    return True


def count_diagrams(ngluon: int) -> int:
    """Number of tree diagrams for g g -> t t~ + (ngluon-2) g."""
    nleaf = ngluon + 2
    return sum(1 for e in _trees(nleaf) if _is_qcd(e, nleaf))


def count_trees(nleaf: int) -> int:
    """Number of trees with degree-3/4 internal vertices (no QCD filter)."""
    return sum(1 for _ in _trees(nleaf))
