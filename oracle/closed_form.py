"""Closed-form spin- and colour-averaged |M|^2 for g g -> Q Qbar (oracle pin).

Test infrastructure only.  Combridge (Nucl. Phys. B151 (1979) 429); in the
form of Ellis, Stirling, Webber, "QCD and collider physics", eq. (10.12):

    |M|^2 / g^4 = (1/(6 t1 t2) - 3/8) (t1^2 + t2^2 + rho - rho^2 / (4 t1 t2))

with t1 = 2 p1.p3 / s, t2 = 2 p2.p3 / s, rho = 4 m^2 / s, averaged over the
initial spins and colours and summed over the final ones.  It is the n = 2
case of the matrix element the paper computes (its smallest process, g g ->
t t~, table "complexity"), at zero top width.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(axis=-1)


def ggqq_averaged(mom: np.ndarray, m: float, gs: float) -> np.ndarray:
    """mom: [nevt][4][4] (g1, g2, Q, Qbar); returns averaged |M|^2 [nevt]."""
    p1, p2, p3 = mom[:, 0], mom[:, 1], mom[:, 2]
    s = 2.0 * _dot(p1, p2)
    t1 = 2.0 * _dot(p1, p3) / s
    t2 = 2.0 * _dot(p2, p3) / s
    rho = 4.0 * m * m / s
    return gs ** 4 * (1.0 / (6.0 * t1 * t2) - 3.0 / 8.0) * (
        t1 * t1 + t2 * t2 + rho - rho * rho / (4.0 * t1 * t2))
