"""Seeded synthetic phase-space points for g g -> t t~ + n g.

This module produces the *inputs* of the matrix-element calculation and holds
none of its arithmetic.  Both the CUDA path and the CPU oracle are fed from
here, so neither side generates its own momenta.

Generator chain (all vectorised numpy, deterministic for a given seed):

* Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11).  The key is the
  64-bit seed, the counter is (candidate index lo, candidate index hi, block,
  0), so candidate ``c`` always sees the same numbers whatever the batch size.
* Massless RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986)
  359) followed by the standard rescaling to massive final states: the common
  momentum factor xi solves sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt(s) by
  Newton iteration.
* Cuts on the final-state gluons only: pT > ptmin for every gluon and
  Delta R > drmin between every gluon pair (Delta phi wrapped into (-pi, pi]).
  A failing candidate is dropped and the next counter value is tried; the
  accepted events keep candidate order.

Particle order in the output is (g1, g2, t, t~, g5, ..., g_npar), with the two
beams along +z and -z, momenta (E, px, py, pz) in GeV, layout [nevt][npar][4]
float64.  The paper's own standalone application draws random momenta in the
same data-parallel way (Sec. 2.1-2.2, "check.exe"), but states no generator, energy
or seed; the choices here are this project's.
"""
from __future__ import annotations

import math

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ctr: uint32 array [..., 4]; key: uint32 array [..., 2] (broadcastable).
    Returns uint32 [..., 4].
    """
    c = [ctr[..., i].astype(np.uint64) for i in range(4)]
    k0 = np.broadcast_to(key[..., 0], ctr.shape[:-1]).astype(np.uint32)
    k1 = np.broadcast_to(key[..., 1], ctr.shape[:-1]).astype(np.uint32)
    for r in range(10):
        p0 = PHILOX_M0 * c[0]
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0.astype(np.uint64), lo1,
             hi0 ^ c[3] ^ k1.astype(np.uint64), lo0]
        if r < 9:
            k0 = ((k0.astype(np.uint64) + np.uint64(PHILOX_W0)) & _MASK32).astype(np.uint32)
            k1 = ((k1.astype(np.uint64) + np.uint64(PHILOX_W1)) & _MASK32).astype(np.uint32)
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def uniforms(seed: int, cand: np.ndarray, ndouble: int) -> np.ndarray:
    """``ndouble`` uniforms in (0, 1) per candidate index (uint64 array).

    Each Philox block yields two doubles of 53 bits: u = (k + 0.5) * 2^-53.
    """
    nblk = (ndouble + 1) // 2
    cand = cand.astype(np.uint64)
    ctr = np.zeros(cand.shape + (nblk, 4), dtype=np.uint32)
    ctr[..., 0] = (cand & _MASK32).astype(np.uint32)[..., None]
    ctr[..., 1] = (cand >> np.uint64(32)).astype(np.uint32)[..., None]
    ctr[..., 2] = np.arange(nblk, dtype=np.uint32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    x = philox4x32_10(ctr, key).astype(np.uint64)
    w = np.stack([(x[..., 0] << np.uint64(32)) | x[..., 1],
                  (x[..., 2] << np.uint64(32)) | x[..., 3]], axis=-1)
    w = (w >> np.uint64(11)).reshape(cand.shape + (2 * nblk,))[..., :ndouble]
    return (w.astype(np.float64) + 0.5) * (2.0 ** -53)


def rambo_massive(sqrts: float, masses, r: np.ndarray):
    """Final-state momenta for a batch: r has shape [nb, nfin, 4] uniforms.

    Returns (p [nb, nfin, 4], weight [nb]) where weight is the RAMBO phase-space
    weight including the massive correction (Kleiss-Stirling-Ellis eq. 4.11).
    """
    masses = np.asarray(masses, dtype=np.float64)
    nb, nfin, _ = r.shape
    c = 2.0 * r[..., 0] - 1.0
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    f = 2.0 * math.pi * r[..., 1]
    q0 = -np.log(r[..., 2] * r[..., 3])
    q = np.stack([q0, q0 * s * np.cos(f), q0 * s * np.sin(f), q0 * c], axis=-1)
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(axis=1))
    b = -Q[:, 1:] / M[:, None]
    g = Q[:, 0] / M
    a = 1.0 / (1.0 + g)
    x = sqrts / M
    bq = (b[:, None, :] * q[..., 1:]).sum(axis=2)
    p = np.empty_like(q)
    p[..., 0] = x[:, None] * (g[:, None] * q[..., 0] + bq)
    p[..., 1:] = x[:, None, None] * (q[..., 1:] + b[:, None, :] * q[..., 0:1]
                                     + a[:, None, None] * bq[..., None] * b[:, None, :])
    # massless weight (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)
    n = nfin
    lw = ((4 - 3 * n) * math.log(2 * math.pi) + (n - 1) * math.log(math.pi / 2)
          + (n - 2) * math.log(sqrts * sqrts) - math.lgamma(n) - math.lgamma(n - 1))
    wt = np.full(nb, math.exp(lw))
    if np.any(masses > 0):
        E = p[..., 0]
        xi = np.full(nb, math.sqrt(max(0.0, 1.0 - (masses.sum() / sqrts) ** 2)))
        for _ in range(60):
            e = np.sqrt(masses[None, :] ** 2 + (xi[:, None] * E) ** 2)
            fval = e.sum(axis=1) - sqrts
            dval = (xi[:, None] * E * E / e).sum(axis=1)
            step = fval / dval
            xi = xi - step
            if np.all(np.abs(step) <= 1e-15 * np.abs(xi)):
                break
        e = np.sqrt(masses[None, :] ** 2 + (xi[:, None] * E) ** 2)
        k = np.empty_like(p)
        k[..., 0] = e
        k[..., 1:] = xi[:, None, None] * p[..., 1:]
        kabs = np.sqrt((k[..., 1:] ** 2).sum(axis=2))
        wt = wt * (xi ** (2 * n - 3)
                   * np.prod(kabs / e, axis=1)
                   * sqrts / (kabs * kabs / e).sum(axis=1))
        p = k
    return p, wt


def _gluon_cuts(pg: np.ndarray, ptmin: float, drmin: float) -> np.ndarray:
    """Boolean mask [nb]: every final gluon has pT > ptmin and every pair Delta R > drmin."""
    nb, ng, _ = pg.shape
    ok = np.ones(nb, dtype=bool)
    if ng == 0:
        return ok
    pt = np.hypot(pg[..., 1], pg[..., 2])
    ok &= np.all(pt > ptmin, axis=1)
    pabs = np.sqrt(pt * pt + pg[..., 3] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        eta = 0.5 * np.log((pabs + pg[..., 3]) / (pabs - pg[..., 3]))
    phi = np.arctan2(pg[..., 2], pg[..., 1])
    for i in range(ng):
        for j in range(i + 1, ng):
            dphi = phi[:, i] - phi[:, j]
            dphi = dphi - 2 * math.pi * np.floor((dphi + math.pi) / (2 * math.pi))
            dphi = np.where(dphi <= -math.pi, dphi + 2 * math.pi, dphi)
            dr2 = (eta[:, i] - eta[:, j]) ** 2 + dphi ** 2
            ok &= dr2 > drmin * drmin
    return ok


def generate(nevt: int, ngluon_final: int, sqrts: float, seed: int, mt: float = 173.0,
             ptmin: float | None = None, drmin: float | None = None,
             batch: int = 1 << 18, return_weights: bool = False, first_candidate: int = 0):
    """``nevt`` phase-space points for g g -> t t~ + ``ngluon_final`` g.

    Returns momenta [nevt][2+2+ngluon_final][4] float64 (and the RAMBO weights
    and candidate indices when ``return_weights``).  Cuts apply only when
    ``ptmin``/``drmin`` are given.
    """
    npar = 4 + ngluon_final
    nfin = npar - 2
    masses = [mt, mt] + [0.0] * ngluon_final
    out = np.empty((nevt, npar, 4))
    wts = np.empty(nevt)
    cids = np.empty(nevt, dtype=np.int64)
    have = 0
    cand0 = first_candidate
    while have < nevt:
        nb = batch
        cand = np.arange(cand0, cand0 + nb, dtype=np.uint64)
        cand0 += nb
        r = uniforms(seed, cand, 4 * nfin).reshape(nb, nfin, 4)
        pf, wt = rambo_massive(sqrts, masses, r)
        ok = np.ones(nb, dtype=bool)
        if ngluon_final and (ptmin is not None or drmin is not None):
            ok = _gluon_cuts(pf[:, 2:, :], ptmin or 0.0, drmin or 0.0)
        idx = np.nonzero(ok)[0][: nevt - have]
        m = len(idx)
        e = 0.5 * sqrts
        out[have:have + m, 0] = (e, 0.0, 0.0, e)
        out[have:have + m, 1] = (e, 0.0, 0.0, -e)
        out[have:have + m, 2:] = pf[idx]
        wts[have:have + m] = wt[idx]
        cids[have:have + m] = cand[idx].astype(np.int64)
        have += m
    if return_weights:
        return out, wts, cids
    return out


# Workloads of the benchmark table: (process, nevt, sqrt(s), cuts, seed).
WORKLOADS = {
    "ggtt_16384": dict(ngluon_final=0, nevt=16384, sqrts=1000.0, cuts=False, seed=20251005 + 1),
    "ggttgg_524288": dict(ngluon_final=2, nevt=524288, sqrts=1500.0, cuts=True, seed=20251005 + 2),
    "ggttggg_262144": dict(ngluon_final=3, nevt=262144, sqrts=1500.0, cuts=True, seed=20251005 + 3),
    "ggttgggg_16384": dict(ngluon_final=4, nevt=16384, sqrts=2000.0, cuts=True, seed=20251005 + 5),
    "ggttggggg_512": dict(ngluon_final=5, nevt=512, sqrts=2000.0, cuts=True, seed=20251005 + 6),
}


def workload(name: str, nevt: int | None = None):
    """Momenta of a named workload (optionally only its first ``nevt`` events)."""
    w = WORKLOADS[name]
    n = w["nevt"] if nevt is None else nevt
    kw = dict(ptmin=20.0, drmin=0.4) if w["cuts"] else {}
    return generate(n, w["ngluon_final"], w["sqrts"], w["seed"], **kw)
