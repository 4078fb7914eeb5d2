"""Lower a process's Feynman diagrams to a wavefunction/amplitude program.

The program is a flat list of operations over numbered wavefunction slots,
the form in which the CUDA diagram kernel executes it (one table entry per
HELAS-like call, Sec. 2.2 of the paper: external wavefunctions, internal
wavefunctions, amplitudes, jamp updates).  Diagram groups (Sec. 4.2, "dpg")
are contiguous ranges of the amplitude list.

Closing a diagram.  A diagram term with attachments B1..Bk along the top line
is closed at its "middle" block M (the block holding chain position
floor((n-1)/2)):  amp = U_L . Mslash . V_R, with U_L the top-line
wavefunction from ubar(p3) through the blocks left of M (each step
U' = U Bslash (qslash + m) / den) and V_R the one from v(p4) through the
blocks right of M.  One of X = U_L Mslash or Y = Mslash V_R is formed (the one
shared by more diagrams) and dotted with the other side.  Diagrams with a
single attachment (s-channel, k = 1) use amp = G0 . J_M with the bilinear
G0^mu = ubar gamma^mu v.  Every wavefunction is built once and shared.

Slots are assigned by linear-scan allocation over the emitted order, so the
per-thread working set is the maximum number of simultaneously live
wavefunctions.
"""
from __future__ import annotations

import heapq

from dataclasses import dataclass, field

from .diagrams import Process, process

# opcodes (must match the CUDA interpreter)
OP_EXT_G = 1    # out, ip(particle), incoming(1/0)
OP_EXT_UB = 2   # out
OP_EXT_V = 3    # out
OP_V3 = 4       # out, a, b, setX, setY          J = V3(a,b) / P^2
OP_V4 = 5       # out1, out2, out3, a, b, c, set  three 4-vertex structures / P^2
OP_FPRE = 6     # out, U, J, set                 U' = U Jslash (q+m) dP[set]
OP_FSUF = 7     # out, V, J, set                 V' = (q+m) Jslash V dS[set]
OP_XROW = 8     # out, U, J                      X = U Jslash
OP_YCOL = 9     # out, J, V                      Y = Jslash V
OP_BIL = 10     # out, U, V                      G^mu = U gamma^mu V
OP_AMP_SS = 11  # X, V, scatter offset, count, acc, mode   amp = X . V
OP_AMP_VV = 12  # G, J, scatter offset, count, acc, mode   amp = G . J (Minkowski)

OPNAMES = {v: k for k, v in dict(globals()).items() if k.startswith("OP_")}

# jamp coefficient codes: amp * {+1, -1, +i, -i}
COEF_CODE = {1: 0, -1: 1, 1j: 2, -1j: 3}
# channel colour-factor codes (0: flow absent)
CHANNEL_CODE = {1: 1, -1: 2, 1j: 3, -1j: 4}

# FP64 instruction counts per op (FMA = 1), used for the algorithmic flop
# count: see flops_per_op(); kept next to the opcode table.


@dataclass
class Program:
    n: int
    npar: int
    ncolor: int
    ops: list = field(default_factory=list)        # list of 8-int records
    scatter: list = field(default_factory=list)    # jamp*4 + coef
    nslot: int = 0                                 # gluon-wavefunction slots (1 variant)
    nslot_f: int = 0                               # top-line slots (2 variants)
    nslot_acc: int = 0                             # amplitude accumulators (4 variants)
    ncolour_groups: int = 0                        # distinct colour factors up to a phase
    channels: list = field(default_factory=list)   # per channel: [(flow, code)] sorted by flow
    ndiagrams: int = 0
    nterms: int = 0
    perms: list = field(default_factory=list)      # colour-flow orderings

    def counts(self):
        c = {}
        for op in self.ops:
            c[OPNAMES[op[0]]] = c.get(OPNAMES[op[0]], 0) + 1
        c["JAMP_UPDATES"] = len(self.scatter)
        return c


class _Builder:
    def __init__(self, P: Process):
        self.P = P
        self.n = P.n
        self.full = P.full
        self.ops = []          # (code, out_objs, in_objs, extra) with symbolic objects
        self.obj = {}          # key -> object id
        self.nobj = 0

    def _emit(self, code, outs, ins, extra):
        self.ops.append((code, outs, ins, extra))

    def _new(self, key):
        oid = self.nobj
        self.nobj += 1
        self.obj[key] = oid
        return oid

    # ---------------------------------------------------------- objects --
    def current(self, c):
        key = ("J", c.idx)
        if key in self.obj:
            return self.obj[key]
        if c.kind == "ext":
            g = min(c.gset)
            ip = g if g < 2 else g + 2
            o = self._new(key)
            self._emit(OP_EXT_G, [o], [], [ip, 1 if ip < 2 else 0])
            return o
        if c.kind == "v3":
            x, y = c.args
            a, b = self.current(x), self.current(y)
            o = self._new(key)
            self._emit(OP_V3, [o], [a, b], [_mask(x.gset), _mask(y.gset)])
            return o
        # v4: the three structures are produced together
        x, y, z = c.args
        a, b, cc = self.current(x), self.current(y), self.current(z)
        sibs = [s for s in self.P.currents_on(c.gset)
                if s.kind == "v4" and s.args == c.args]
        sibs.sort(key=lambda s: s.term)
        outs = [self._new(("J", s.idx)) for s in sibs]
        self._emit(OP_V4, outs, [a, b, cc], [_mask(c.gset)])
        return self.obj[key]

    def ubar(self):
        key = ("UB",)
        if key not in self.obj:
            o = self._new(key)
            self._emit(OP_EXT_UB, [o], [], [])
        return self.obj[key]

    def vsp(self):
        key = ("V",)
        if key not in self.obj:
            o = self._new(key)
            self._emit(OP_EXT_V, [o], [], [])
        return self.obj[key]

    def prefix(self, blocks):
        """U after absorbing blocks (left to right) from ubar(p3)."""
        if not blocks:
            return self.ubar()
        key = ("U",) + tuple(b.idx for b in blocks)
        if key in self.obj:
            return self.obj[key]
        u = self.prefix(blocks[:-1])
        j = self.current(blocks[-1])
        s = frozenset().union(*[b.gset for b in blocks])
        o = self._new(key)
        self._emit(OP_FPRE, [o], [u, j], [_mask(s)])
        return o

    def suffix(self, blocks):
        """V after absorbing blocks (right to left) from v(p4)."""
        if not blocks:
            return self.vsp()
        key = ("W",) + tuple(b.idx for b in blocks)
        if key in self.obj:
            return self.obj[key]
        v = self.suffix(blocks[1:])
        j = self.current(blocks[0])
        s = frozenset().union(*[b.gset for b in blocks])
        o = self._new(key)
        self._emit(OP_FSUF, [o], [v, j], [_mask(s)])
        return o

    def xrow(self, L, M):
        key = ("X",) + tuple(b.idx for b in L) + ("|", M.idx)
        if key not in self.obj:
            u = self.prefix(L)
            j = self.current(M)
            o = self._new(key)
            self._emit(OP_XROW, [o], [u, j], [])
        return self.obj[key]

    def ycol(self, M, R):
        key = ("Y", M.idx, "|") + tuple(b.idx for b in R)
        if key not in self.obj:
            j = self.current(M)
            v = self.suffix(R)
            o = self._new(key)
            self._emit(OP_YCOL, [o], [j, v], [])
        return self.obj[key]

    def g0(self):
        key = ("G0",)
        if key not in self.obj:
            u, v = self.ubar(), self.vsp()
            o = self._new(key)
            self._emit(OP_BIL, [o], [u, v], [])
        return self.obj[key]


def _has_v4(c) -> bool:
    """True when a gluon sub-tree contains a four-gluon vertex."""
    return c.kind == "v4" or any(_has_v4(a) for a in c.args)


def _mask(s) -> int:
    m = 0
    for g in s:
        m |= 1 << g
    return m


def _split(d, mpos):
    """(L, M, R) for a diagram term: M holds chain position mpos."""
    pos = 0
    for j, b in enumerate(d.blocks):
        if pos <= mpos < pos + len(b.gset):
            return d.blocks[:j], b, d.blocks[j + 1:]
        pos += len(b.gset)
    raise AssertionError


def build_program(n: int, order: str = "middle") -> Program:
    P = process(n)
    from itertools import permutations
    perms = list(permutations(range(n)))
    pidx = {p: i for i, p in enumerate(perms)}
    B = _Builder(P)
    mpos = (n - 1) // 2

    terms = []
    xcount, ycount = {}, {}
    for d in P.diagrams:
        if len(d.blocks) == 1:
            terms.append((d, None))
            continue
        L, M, R = _split(d, mpos)
        kx = (tuple(b.idx for b in L), M.idx)
        ky = (M.idx, tuple(b.idx for b in R))
        xcount[kx] = xcount.get(kx, 0) + 1
        ycount[ky] = ycount.get(ky, 0) + 1
        terms.append((d, (L, M, R, kx, ky)))

    # order: terms sharing their largest wavefunction are emitted together so
    # that big currents die soon after they are built
    def deps(t):
        d, s = t
        if s is None:
            return list(d.blocks[0].args)
        L, M, R, kx, ky = s
        return [M] + list(L) + list(R)

    def sort_key(t):
        ds = sorted(deps(t), key=lambda c: (-len(c.gset), c.idx))
        return tuple((-len(c.gset), c.idx) for c in ds)
    terms.sort(key=sort_key)

    # Diagram terms whose colour factors agree up to a unit phase share their
    # scatter: their amplitudes are summed (with that phase) into an
    # accumulator and the group's last member scatters the sum once.  (Each
    # group holds exactly one diagram made of three-point vertices, so there
    # are as many groups as single-diagram-enhancement channels below.)
    group_of, phase_of, rep = {}, {}, {}
    sorted_colour = {}     # a term's colour decomposition in flow order (used twice)
    for d, _ in terms:
        items = sorted(d.color.items(), key=lambda kv: pidx[kv[0]])
        sorted_colour[d.idx] = items
        c0 = complex(items[0][1])
        key = tuple((st, complex(c) / c0) for st, c in items)
        if key not in rep:
            rep[key] = (len(rep), items, c0)
        group_of[d.idx] = rep[key][0]
        phase_of[d.idx] = c0
    members = {}
    for d, _ in terms:
        members.setdefault(group_of[d.idx], []).append(d.idx)

    # Single-diagram-enhancement channels: the diagrams made of three-point
    # vertices only (the paper's channel counts 3 / 15 / 105 / 945, the
    # diagrams MadEvent's single diagram enhancement uses).  A channel is
    # identified by its colour factor: the flow coefficients divided by the
    # first one (flow order), coded 1: +1, 2: -1, 3: +i, 4: -i; channels are
    # numbered in the lexicographic order of these code vectors over all
    # flows (a zero entry, i.e. an absent flow, sorts lowest).  Terms with a
    # four-gluon vertex belong to no channel (-1).
    chan_code = {}
    for d, _ in terms:
        if any(_has_v4(b) for b in d.blocks):
            continue
        items = sorted_colour[d.idx]
        c0 = complex(items[0][1])
        chan_code[d.idx] = tuple((pidx[st], CHANNEL_CODE[complex(c) / c0]) for st, c in items)
    # lexicographic order of the dense code vectors, from the sparse lists:
    # at the first flow where two vectors differ the one with a coefficient
    # there (rather than none) or with the larger code is larger
    order = sorted(chan_code, key=lambda i: tuple((-f, c) for f, c in chan_code[i]))
    channel_of = {i: k for k, i in enumerate(order)}
    if len({chan_code[i] for i in order}) != len(order):
        raise AssertionError("two channels share a colour factor")
    rep_items = {g: (it, c0) for _, (g, it, c0) in rep.items()}

    scatter = []
    for d, s in terms:
        if s is None:
            g = B.g0()
            j = B.current(d.blocks[0])
            code, ins = OP_AMP_VV, [g, j]
        else:
            L, M, R, kx, ky = s
            if xcount[kx] >= ycount[ky]:
                x = B.xrow(L, M)
                v = B.suffix(R)
                code, ins = OP_AMP_SS, [x, v]
            else:
                u = B.prefix(L)
                y = B.ycol(M, R)
                code, ins = OP_AMP_SS, [u, y]
        g = group_of[d.idx]
        mem = members[g]
        if len(mem) == 1:
            off = len(scatter)
            for string, c in sorted_colour[d.idx]:
                scatter.append(pidx[string] * 4 + COEF_CODE[complex(c)])
            B._emit(code, [], ins, [off, len(scatter) - off, None, 0, channel_of.get(d.idx, -1)])
            continue
        first, last = mem[0] == d.idx, mem[-1] == d.idx
        acc_key = ("ACC", g)
        outs = [B._new(acc_key)] if first else []
        acc_in = [] if first else [B.obj[acc_key]]
        off = cnt = 0
        if last:
            items, c0 = rep_items[g]
            off = len(scatter)
            for string, c in items:
                scatter.append(pidx[string] * 4 + COEF_CODE[complex(c) / c0])
            cnt = len(scatter) - off
        mode = COEF_CODE[phase_of[d.idx]] | (4 if first else 0) | (8 if last else 0)
        B._emit(code, outs, ins + acc_in, [off, cnt, "acc", mode, channel_of.get(d.idx, -1)])

    # ------------------------------------------------ slot allocation ----
    # Three pools, by how many top-helicity variants an object carries:
    #   G: gluon wavefunctions (EXT_G, V3, V4)             1 variant
    #   F: top-line objects (ubar/v side, FPRE, FSUF, XROW, YCOL)  2 variants
    #      (the helicity of the top for ubar-side objects, of the antitop
    #      for v-side ones)
    #   the bilinear G0 = ubar gamma v                   4 variants, own storage
    #   A: amplitude accumulators of colour-factor groups  4 variants
    pool_of = {}
    for code, outs, ins, extra in B.ops:
        for o in outs:
            if code in (OP_EXT_G, OP_V3, OP_V4):
                pool_of[o] = "G"
            elif code == OP_BIL:
                pool_of[o] = "B"
            elif code in (OP_AMP_SS, OP_AMP_VV):
                pool_of[o] = "A"
            else:
                pool_of[o] = "F"
    last_use = {}
    for i, (code, outs, ins, extra) in enumerate(B.ops):
        for o in ins:
            last_use[o] = i
    slot_of = {}
    # free slots per pool: a min-heap (the lowest free slot is reused first)
    # and the same slots as a set for membership tests
    free = {"G": [], "F": [], "B": [], "A": []}
    free_set = {k: set() for k in free}
    nslot = {"G": 0, "F": 0, "B": 0, "A": 0}
    records = []
    for i, (code, outs, ins, extra) in enumerate(B.ops):
        in_slots = [slot_of[o] for o in ins]
        out_slots = []
        for o in outs:
            pl = pool_of[o]
            if o not in last_use and pl != "A":
                raise AssertionError("unused wavefunction")
            if free[pl]:
                s_ = heapq.heappop(free[pl])
                free_set[pl].discard(s_)
            else:
                s_ = nslot[pl]
                nslot[pl] += 1
            slot_of[o] = s_
            out_slots.append(s_)
        # release inputs whose last use is this op (outputs never alias inputs);
        # an accumulator dies at its group's final (scattering) member
        for o in set(ins) | set(outs):
            if last_use.get(o, i) == i and (o in ins or (extra and len(extra) == 5 and extra[3] & 8)):
                if o in slot_of and slot_of[o] not in free_set[pool_of[o]]:
                    heapq.heappush(free[pool_of[o]], slot_of[o])
                    free_set[pool_of[o]].add(slot_of[o])
        records.append(_record(code, out_slots, in_slots, extra))
    assert nslot["B"] <= 1
    prog = Program(n=n, npar=n + 2, ncolor=len(perms), ops=records, scatter=scatter,
                   nslot=nslot["G"], nslot_f=nslot["F"], nslot_acc=nslot["A"],
                   ndiagrams=P.ndiagrams, nterms=len(P.diagrams), perms=perms,
                   ncolour_groups=len(rep),
                   channels=[list(chan_code[i]) for i in order])
    return prog


def _record(code, outs, ins, extra):
    """8-int op record: [code, f1..f7] (layout documented per opcode)."""
    r = [code] + [0] * 7
    if code == OP_EXT_G:
        r[1], r[2], r[3] = outs[0], extra[0], extra[1]
    elif code in (OP_EXT_UB, OP_EXT_V):
        r[1] = outs[0]
    elif code == OP_V3:
        r[1], r[2], r[3], r[4], r[5] = outs[0], ins[0], ins[1], extra[0], extra[1]
    elif code == OP_V4:
        r[1], r[2], r[3] = outs
        r[4], r[5], r[6] = ins
        r[7] = extra[0]
    elif code in (OP_FPRE, OP_FSUF):
        r[1], r[2], r[3], r[4] = outs[0], ins[0], ins[1], extra[0]
    elif code in (OP_XROW, OP_YCOL, OP_BIL):
        r[1], r[2], r[3] = outs[0], ins[0], ins[1]
    elif code in (OP_AMP_SS, OP_AMP_VV):
        # [code, channel, X, V, scatter offset, scatter count, accumulator (-1: none), mode]
        # channel: the single-diagram-enhancement channel of a diagram made of
        # three-point vertices only, -1 for a term with a four-gluon vertex
        # mode: bits 0-1 phase code of this amplitude in its group's sum, bit 2
        # first member (initialises the accumulator), bit 3 last member (scatters)
        r[1] = extra[4]
        r[2], r[3], r[4], r[5] = ins[0], ins[1], extra[0], extra[1]
        if extra[2] is None:
            r[6], r[7] = -1, 0
        else:
            r[6] = outs[0] if outs else ins[2]
            r[7] = extra[3]
    else:
        raise ValueError(code)
    return r
