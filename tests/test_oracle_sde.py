"""Pins of the single-diagram oracle (oracle/sde.py), no GPU.

Each check compares the diagram-by-diagram evaluation with something it
does not share code with: the Berends-Giele colour-ordered amplitudes of
bg.c (themselves pinned by tests/test_oracle.py), the paper's channel counts
(tests/golden), a selection rule of the three-gluon vertex, and the
symmetries of the physics (rotations, relabelling the incoming gluons).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import sde
from paper_2510_05392_gb300 import phasespace as ps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_complexity.json")


def _events(n, nevt, seed):
    if n == 2:
        return ps.generate(nevt, 0, 1000.0, seed)
    return ps.generate(nevt, n - 2, 1500.0, seed, ptmin=20.0, drmin=0.4)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_counts_against_paper_table(n):
    """Diagrams 3 / 16 / 123 and single-diagram-enhancement channels
    3 / 15 / 105 (table "complexity", rows 2 and 3)."""
    row = json.load(open(GOLDEN))["processes"]["g g > t t~" + " g" * (n - 2)]
    assert len(sde.diagrams(n)) == row["diagrams"]
    assert len(sde.channels(n)[0]) == row["sde_channels"]


@pytest.mark.parametrize("n", [2, 3, 4])
def test_diagrams_sum_to_berends_giele_amplitudes(n):
    """sum over diagram terms of (flow coefficient x value) equals every
    colour-ordered amplitude of the Berends-Giele recursion, per helicity
    (a dropped term, a wrong sign, vertex or propagator anywhere fails)."""
    mom = _events(n, 2, 300 + n)
    hels = list(range(1 << (n + 2)))
    A = sde.colour_ordered(mom, hels)
    for e in range(len(mom)):
        for h in hels:
            ref = oracle.amplitudes(mom[e], h)
            assert np.abs(A[e, h] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [2, 3, 4])
def test_three_gluon_vertex_selection_rule(n):
    """In the centre-of-mass frame with the beams along z and transverse
    polarisations (eps^0 = 0), a three-gluon vertex joining the two incoming
    gluons reduces to (eps1.eps2)(k1 - k2), and eps1.eps2 = 0 for opposite
    gluon helicities: every diagram with that vertex vanishes there and not
    for equal helicities."""
    def joins_beams(spec):
        if spec[0] == "e":
            return False
        kids = spec[1:] if spec[0] == "v3" else spec[2:]
        if spec[0] == "v3" and {kids[0], kids[1]} == {("e", 0), ("e", 1)}:
            return True
        return any(joins_beams(k) for k in kids)

    mom = _events(n, 2, 400 + n)
    npar = n + 2
    hels = list(range(1 << npar))
    L = sde.term_amplitudes(mom, hels)
    idx = [i for i, (_, t, triv, _) in enumerate(sde.terms(n)) if triv and any(joins_beams(s) for s in t)]
    assert idx
    opp = [h for h in hels if ((h >> (npar - 1)) & 1) != ((h >> (npar - 2)) & 1)]
    same = [h for h in hels if h not in opp]
    scale = np.abs(L).max()
    assert np.abs(L[idx][:, :, opp]).max() <= 1e-14 * scale
    assert np.abs(L[idx][:, :, same]).max() >= 1e-3 * scale


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


@pytest.mark.parametrize("n", [2, 3, 4])
def test_rotation_invariance_per_diagram_and_helicity(n):
    """Rotating every momentum maps each helicity state onto itself up to a
    phase (eps^0 = 0 survives rotations), so |D_t,h|^2 of every diagram term
    and helicity is unchanged."""
    mom = _events(n, 2, 500 + n)
    R = _rotation(np.random.default_rng(n))
    rot = mom.copy()
    rot[..., 1:] = mom[..., 1:] @ R.T
    hels = list(range(1 << (n + 2)))
    a = np.abs(sde.term_amplitudes(mom, hels)) ** 2
    b = np.abs(sde.term_amplitudes(rot, hels)) ** 2
    assert np.abs(a - b).max() <= 1e-11 * a.max()


def _relabelled_channel(n, swap):
    """Channel index map under relabelling the gluons by ``swap`` (gluon
    index -> gluon index): the colour factor of the relabelled diagram is the
    flow vector with its orderings relabelled."""
    _, codes = sde.channels(n)
    perms = sde.flow_orderings(n)
    pos = {p: i for i, p in enumerate(perms)}
    val = {1: 1, 2: -1, 3: 1j, 4: -1j}
    key = {tuple(c): i for i, c in enumerate(codes)}
    out = []
    for c in codes:
        x = np.zeros(len(perms), dtype=complex)
        for s, k in enumerate(c):
            if k:
                x[pos[tuple(swap[g] for g in perms[s])]] = val[int(k)]
        out.append(key[sde.channel_code(x)])
    return np.array(out)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_bose_symmetry_of_channel_weights(n):
    """Exchanging the incoming gluons (momenta p1 <-> p2) maps every diagram
    onto the diagram with the gluon labels exchanged: the channel weights are
    permuted accordingly (t- and u-channel exchange places for g g -> t t~)."""
    mom = _events(n, 3, 600 + n)
    sw = mom.copy()
    sw[:, [0, 1]] = mom[:, [1, 0]]
    w = sde.sde_weights(mom)
    ws = sde.sde_weights(sw)
    swap = list(range(n))
    swap[0], swap[1] = 1, 0
    m = _relabelled_channel(n, swap)
    assert sorted(m) == list(range(len(m)))
    assert np.abs(ws[:, m] - w).max() <= 1e-12
    assert np.abs(np.sort(w, axis=1) - np.sort(ws, axis=1)).max() <= 1e-12
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=1e-13)
