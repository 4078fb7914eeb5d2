"""Test helper: execute a compiled process program on the CPU with numpy.

Checks the process compiler's tables (op records, slots, jamp scatter,
colour matrix) and their Dirac conventions independently of CUDA.  It is a
separate restatement of the op semantics documented in
paper_2510_05392_gb300/compiler/program.py; the library never uses it.
"""
import math

import numpy as np

from paper_2510_05392_gb300.compiler import colour, program as P

METRIC = np.array([1.0, -1.0, -1.0, -1.0])


def _mdot(a, b):
    return (a * b * METRIC).sum(-1)


def _pol(p, lam, incoming):
    px, py, pz = p[:, 1], p[:, 2], p[:, 3]
    pt = np.hypot(px, py)
    pa = np.sqrt(pt * pt + pz * pz)
    with np.errstate(divide="ignore", invalid="ignore"):
        e1 = np.stack([0 * pt, px * pz / (pa * pt), py * pz / (pa * pt), -pt / pa], -1)
        e2 = np.stack([0 * pt, -py / pt, px / pt, 0 * pt], -1)
    z = pt == 0
    e1[z] = np.stack([0 * pt[z], np.where(pz[z] >= 0, 1.0, -1.0), 0 * pt[z], 0 * pt[z]], -1)
    e2[z] = np.array([0.0, 0.0, 1.0, 0.0])
    eps = (-lam * e1 - 1j * e2) / math.sqrt(2)
    return eps if incoming else eps.conj()


def _chi(p, h):
    px, py, pz = p[:, 1], p[:, 2], p[:, 3]
    pa = np.sqrt(px * px + py * py + pz * pz)
    a = np.sqrt(2 * pa * (pa + pz))
    if h > 0:
        return np.stack([(pa + pz) / a, (px + 1j * py) / a], -1)
    return np.stack([(-px + 1j * py) / a, (pa + pz) / a], -1)


def _ubar(p, h):
    pa = np.sqrt((p[:, 1:] ** 2).sum(-1))
    x = _chi(p, h)
    wm, wp = np.sqrt(np.maximum(p[:, 0] - h * pa, 0)), np.sqrt(np.maximum(p[:, 0] + h * pa, 0))
    u = np.concatenate([wm[:, None] * x, wp[:, None] * x], -1)
    return np.concatenate([u[:, 2:], u[:, :2]], -1).conj()


def _v(p, h):
    pa = np.sqrt((p[:, 1:] ** 2).sum(-1))
    x = _chi(p, -h)
    wp, wm = np.sqrt(np.maximum(p[:, 0] + h * pa, 0)), np.sqrt(np.maximum(p[:, 0] - h * pa, 0))
    return np.concatenate([wp[:, None] * x, -wm[:, None] * x], -1)


# chiral gamma matrices
_S = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1.0, -1.0])]
_G = []
for mu in range(4):
    g = np.zeros((4, 4), complex)
    g[:2, 2:] = _S[mu]
    g[2:, :2] = _S[mu] if mu == 0 else -_S[mu]
    _G.append(g)
_G = np.array(_G)


def _slash(a):  # a [..., 4] upper index -> [..., 4, 4]
    al = a * METRIC
    return np.einsum("...m,mij->...ij", al, _G)


def run(n, mom, mt=173.0, wt=1.4915, alphas=0.118, per_helicity=False):
    prog = P.build_program(n)
    Chat, D, _ = colour.colour_matrix(n)
    C = np.array(Chat, float)
    npar = n + 2
    nev = mom.shape[0]
    Kg = [mom[:, g] if g < 2 else -mom[:, g + 2] for g in range(n)]

    def K(mask):
        return sum(Kg[g] for g in range(n) if mask >> g & 1)

    p3, p4 = mom[:, 2], mom[:, 3]
    tot = np.zeros(nev)
    mh_all = np.zeros((nev, 1 << npar))
    for h in range(1 << npar):
        sg = lambda ip: 1 if (h >> (npar - 1 - ip)) & 1 else -1
        WG, WF, WB, WA = {}, {}, {}, {}   # slot pools: gluon, top-line, bilinear, accumulators
        J = np.zeros((nev, prog.ncolor), complex)
        for r in prog.ops:
            c = r[0]
            if c == P.OP_EXT_G:
                WG[r[1]] = _pol(mom[:, r[2]], sg(r[2]), r[3] == 1)
            elif c == P.OP_EXT_UB:
                WF[r[1]] = _ubar(p3, sg(2))
            elif c == P.OP_EXT_V:
                WF[r[1]] = _v(p4, sg(3))
            elif c == P.OP_V3:
                J1, J2, K1, K2 = WG[r[2]], WG[r[3]], K(r[4]), K(r[5])
                P_ = K1 + K2
                out = (_mdot(J1, J2)[:, None] * (K1 - K2) + J2 * _mdot(K1 + 2 * K2, J1)[:, None]
                       - J1 * _mdot(2 * K1 + K2, J2)[:, None])
                WG[r[1]] = out / _mdot(P_, P_)[:, None]
            elif c == P.OP_V4:
                X, Y, Z = WG[r[4]], WG[r[5]], WG[r[6]]
                Kt = K(r[7])
                inv = 1 / _mdot(Kt, Kt)[:, None]
                xy, xz, yz = _mdot(X, Y)[:, None], _mdot(X, Z)[:, None], _mdot(Y, Z)[:, None]
                WG[r[1]] = (xz * Y - yz * X) * inv
                WG[r[2]] = (xy * Z - yz * X) * inv
                WG[r[3]] = (xy * Z - xz * Y) * inv
            elif c in (P.OP_FPRE, P.OP_FSUF):
                Ks = K(r[4])
                q = (p3 - Ks) if c == P.OP_FPRE else (Ks - p4)
                den = 1 / (_mdot(q, q) - mt * mt + 1j * mt * wt)
                qm = _slash(q.astype(complex)) + mt * np.eye(4)
                if c == P.OP_FPRE:
                    t = np.einsum("ei,eij->ej", WF[r[2]], _slash(WG[r[3]]))
                    WF[r[1]] = np.einsum("ei,eij->ej", t, qm) * den[:, None]
                else:
                    t = np.einsum("eij,ej->ei", _slash(WG[r[3]]), WF[r[2]])
                    WF[r[1]] = np.einsum("eij,ej->ei", qm, t) * den[:, None]
            elif c == P.OP_XROW:
                WF[r[1]] = np.einsum("ei,eij->ej", WF[r[2]], _slash(WG[r[3]]))
            elif c == P.OP_YCOL:
                WF[r[1]] = np.einsum("eij,ej->ei", _slash(WG[r[2]]), WF[r[3]])
            elif c == P.OP_BIL:
                WB[r[1]] = np.einsum("ei,mij,ej->em", WF[r[2]], _G, WF[r[3]])
            elif c in (P.OP_AMP_SS, P.OP_AMP_VV):
                a = (WF[r[2]] * WF[r[3]]).sum(-1) if c == P.OP_AMP_SS else _mdot(WB[r[2]], WG[r[3]])
                if r[6] >= 0:   # colour-factor group: accumulate, last member scatters
                    ph = [1, -1, 1j, -1j][r[7] & 3]
                    WA[r[6]] = ph * a if r[7] & 4 else WA[r[6]] + ph * a
                    if not r[7] & 8:
                        continue
                    a = WA[r[6]]
                for e in prog.scatter[r[4]:r[4] + r[5]]:
                    J[:, e >> 2] += a * [1, -1, 1j, -1j][e & 3]
        mh = np.einsum("ei,ij,ej->e", J.conj(), C, J).real
        mh_all[:, h] = mh
        tot += mh
    fac = (4 * math.pi * alphas) ** n / (256 * math.factorial(n - 2) * D)
    return (tot * fac, mh_all * fac) if per_helicity else tot * fac
