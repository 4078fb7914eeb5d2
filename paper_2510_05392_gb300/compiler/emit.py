"""Emit the process tables compiled into the CUDA library.

For every supported process the generated include file holds:
  OPS    int32[nops][8]   the wavefunction/amplitude program (program.py)
  SCAT   int32[nscat]     jamp scatter entries (flow * 4 + coefficient code)
  CHAT   int32[nc][nc]    integer colour matrix D * C (colour.py)
  CHO    int32[nch + 1]   single-diagram-enhancement channels: offsets into CHF
  CHF    int32[...]       per channel its colour factor, flow * 8 + code
                          (program.py: 1 +1, 2 -1, 3 +i, 4 -i; first entry +1)
and one registry row with the sizes, the common denominator D, the averaging
factor and the algorithmic FP64 operation counts per helicity.

Processes too large to compile in (g g > t t~ + 5 g: 810k ops, 5040 flows)
are written instead as a binary table file that the library loads at run
time (emit_blob; format below).

Usage: python -m paper_2510_05392_gb300.compiler.emit OUT.inc [maxgluons]
       python -m paper_2510_05392_gb300.compiler.emit --blob OUT.bin ngluons
"""
from __future__ import annotations

import math
import struct
import sys

from . import colour, program

PROCESSES = [
    ("ggtt", "g g > t t~"),
    ("ggttg", "g g > t t~ g"),
    ("ggttgg", "g g > t t~ g g"),
    ("ggttggg", "g g > t t~ g g g"),
    ("ggttgggg", "g g > t t~ g g g g"),
]

# Algorithmic FP64 operations (an FMA counts 2 flops, mul/add 1) of each op,
# from the arithmetic the operation must do, not from the instructions the
# compiler emits.  Complex a*b = 6 flops, a*b+c = 8.  Each entry is
# (flops shared by all top-helicity variants, flops per variant, variants):
# one evaluation of the program covers the four (top, antitop) helicity
# combinations of one gluon-helicity configuration.
_SLASH = 16            # Jslash blocks: 8 complex adds
_ROWJ = 56             # row spinor x Jslash: two 2x2 complex mat-vecs
_QM = 40 + 16          # (qslash + m): two 2x2 mat-vecs with real/imaginary entries + mass terms
_DEN = 24              # complex scaling by 1/den
FLOPS = {
    program.OP_EXT_G: (0, 0, 1),     # external states: per event, not counted
    program.OP_EXT_UB: (0, 0, 2),
    program.OP_EXT_V: (0, 0, 2),
    # V3: 3 complex Minkowski dots (30 + 2*14), 3 complex scalings by 1/P^2
    # (6), 4 components of j*d + s2*J2 - s1*J1 (4*(2 + 8 + 8))
    program.OP_V3: (30 + 28 + 6 + 72, 0, 1),
    # V4: 3 complex dots (90), 3 scalings (6), 3 x 4 components of a*X - b*Y (168)
    program.OP_V4: (90 + 6 + 168, 0, 1),
    program.OP_FPRE: (_SLASH, _ROWJ + _QM + _DEN, 2),
    program.OP_FSUF: (_SLASH, _ROWJ + _QM + _DEN, 2),
    program.OP_XROW: (_SLASH, _ROWJ, 2),
    program.OP_YCOL: (_SLASH, _ROWJ, 2),
    # bilinear: 8 complex products (48) + 12 complex adds (24), per variant
    program.OP_BIL: (0, 48 + 24, 4),
    # amplitudes: 4 complex products + 3 complex adds, per variant
    program.OP_AMP_SS: (0, 4 * 6 + 3 * 2, 4),
    program.OP_AMP_VV: (0, 4 * 6 + 3 * 2, 4),
}
JAMP_UPDATE_FLOPS = 2


def algorithmic_flops(prog: program.Program) -> dict:
    """FP64 flops per good helicity (all four top combinations good): the
    diagram program (ops + jamp updates) shared over four helicities, and the
    colour sum (symmetric quadratic form over A and B)."""
    unit = 0
    for op in prog.ops:
        sh, pv, nv = FLOPS[op[0]]
        unit += sh + pv * nv
    unit += JAMP_UPDATE_FLOPS * 4 * len(prog.scatter)
    # amplitudes added into their colour group's accumulator (all but the first)
    unit += JAMP_UPDATE_FLOPS * 4 * sum(
        1 for op in prog.ops if op[0] in (program.OP_AMP_SS, program.OP_AMP_VV)
        and op[6] >= 0 and not op[7] & 4)
    nc = prog.ncolor
    csum = 2 * (nc * (nc + 1) // 2) * 2 + 2 * nc
    return dict(diagram=unit / 4.0, colour=csum)


def channel_tables(prog: program.Program):
    """(offsets [nchannel + 1], entries flow * 8 + code) of the channels'
    colour factors."""
    off, ent = [0], []
    for ch in prog.channels:
        ent.extend(f * 8 + c for f, c in ch)
        off.append(len(ent))
    return off, ent


def _arr(name, vals, per_line=16):
    out = [f"static const int32_t {name}[{max(1, len(vals))}] = {{"]
    for i in range(0, len(vals), per_line):
        out.append("  " + ",".join(str(int(v)) for v in vals[i:i + per_line]) + ",")
    if not vals:
        out.append("  0")
    out.append("};")
    return "\n".join(out)


def emit(path: str, max_gluons: int = 6, list_path: str | None = None) -> None:
    """Write the table include file ``path`` and, next to it (or at
    ``list_path``), mg_proc_list.h with one X(index, ngluon, nslot_gluon,
    nslot_top, nslot_acc, ncolor) entry per process for the kernel
    instantiations."""
    lines = ["/* generated by paper_2510_05392_gb300.compiler.emit -- do not edit */",
             "#pragma once", "#include <stdint.h>", ""]
    rows = []
    xlist = []
    for name, proc in PROCESSES:
        n = 2 + len(proc.split()) - 5
        if n > max_gluons:
            continue
        prog = program.build_program(n)
        Chat, D, perms = colour.colour_matrix(n)
        assert [tuple(p) for p in perms] == [tuple(p) for p in prog.perms]
        flat_ops = [v for r in prog.ops for v in r]
        flat_c = [v for r in Chat for v in r]
        lines.append(_arr(f"OPS_{name}", flat_ops))
        lines.append(_arr(f"SCAT_{name}", prog.scatter))
        lines.append(_arr(f"CHAT_{name}", flat_c))
        cho, chf = channel_tables(prog)
        lines.append(_arr(f"CHO_{name}", cho))
        lines.append(_arr(f"CHF_{name}", chf))
        fl = algorithmic_flops(prog)
        iden = 256 * math.factorial(n - 2)
        rows.append(
            f'  {{"{name}", "{proc}", {n}, {n + 2}, {prog.ndiagrams}, {prog.nterms}, '
            f'{prog.ncolor}, {prog.nslot}, {prog.nslot_f}, {prog.nslot_acc}, {len(prog.ops)}, '
            f'{len(prog.scatter)}, '
            f'{D}LL, {iden}.0, {fl["diagram"]!r}, {fl["colour"]}.0, OPS_{name}, SCAT_{name}, '
            f'CHAT_{name}, NULL, NULL, {len(prog.channels)}, CHO_{name}, CHF_{name}}},')
        xlist.append(f"X({len(rows) - 1}, {n}, {prog.nslot}, {prog.nslot_f}, {max(1, prog.nslot_acc)}, "
                     f"{prog.ncolor})")
        lines.append("")
    lines.append("static const mg_proc_table MG_PROC_TABLES[] = {")
    lines.extend(rows)
    lines.append("};")
    lines.append(f"static const int MG_NPROC_TABLES = {len(rows)};")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    import os
    lp = list_path or os.path.join(os.path.dirname(path), "mg_proc_list.h")
    with open(lp, "w") as f:
        f.write("/* generated by paper_2510_05392_gb300.compiler.emit -- do not edit */\n"
                "#pragma once\n#define MG_PROC_LIST(X) " + " ".join(xlist) + "\n")


# Binary process table (little-endian), read by mg_process_create_from_tables:
#   char[8]  "MGPROC02"
#   int32[13] version (2), ngluon, npar, ncolor, nops, nscat, nslot (gluon),
#             nslot_top, nslot_acc, ncolour_groups, ndiagrams, nterms, nchannel
#   int64    D (common denominator);  float64 iden, flops_diagram, flops_colour
#   int32    ops[nops][8];  int32 scat[nscat]
#   int64    row[ncolor]    D * C_(id, r) by relative ordering r (colour.relative_row)
#   int8     perms[ncolor][ngluon]   the flow orderings, itertools order
#   int32    chan_off[nchannel + 1];  int32 chan_flows[chan_off[nchannel]]
BLOB_MAGIC = b"MGPROC02"


def emit_blob(n: int, path: str) -> None:
    prog = program.build_program(n)
    row, D = colour.relative_row(n)
    fl = algorithmic_flops(prog)
    iden = 256 * math.factorial(n - 2)
    with open(path + ".tmp", "wb") as f:
        f.write(BLOB_MAGIC)
        f.write(struct.pack("<13i", 2, n, n + 2, prog.ncolor, len(prog.ops), len(prog.scatter),
                            prog.nslot, prog.nslot_f, max(1, prog.nslot_acc), prog.ncolour_groups,
                            prog.ndiagrams, prog.nterms, len(prog.channels)))
        f.write(struct.pack("<q3d", D, float(iden), float(fl["diagram"]), float(fl["colour"])))
        f.write(struct.pack(f"<{8 * len(prog.ops)}i", *[v for r in prog.ops for v in r]))
        f.write(struct.pack(f"<{len(prog.scatter)}i", *prog.scatter))
        f.write(struct.pack(f"<{len(row)}q", *row))
        f.write(bytes(v for p in prog.perms for v in p))
        cho, chf = channel_tables(prog)
        f.write(struct.pack(f"<{len(cho)}i", *cho))
        f.write(struct.pack(f"<{len(chf)}i", *chf))
    import os
    os.replace(path + ".tmp", path)


if __name__ == "__main__":
    if sys.argv[1] == "--blob":
        emit_blob(int(sys.argv[3]), sys.argv[2])
    else:
        emit(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 6)
