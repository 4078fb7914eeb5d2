"""Process compiler and C-ABI library checks that need no GPU."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle
from oracle import color as ocolor
from paper_2510_05392_gb300 import phasespace as ps
from paper_2510_05392_gb300.compiler import colour, diagrams, program

import table_emulator

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "paper_table_complexity.json")


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_diagram_counts_match_paper(n):
    g = json.load(open(GOLDEN))["processes"]
    proc = "g g > t t~" + " g" * (n - 2)
    P = diagrams.Process(n)
    assert P.ndiagrams == g[proc]["diagrams"]
    # every colour coefficient of every diagram term is +-1 or +-i and every
    # string is a permutation of the gluons
    for d in P.diagrams:
        for s, c in d.color.items():
            assert sorted(s) == list(range(n))
            assert complex(c) in (1, -1, 1j, -1j)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_colour_matrix_bit_exact_vs_oracle(n):
    a = colour.colour_matrix(n)
    b = ocolor.color_matrix(n)
    assert a[1] == b[1]
    assert a[0] == b[0]
    assert [tuple(x) for x in a[2]] == [tuple(x) for x in b[2]]


# pool of every operand: G gluon wavefunctions, F top-line objects, B bilinear
_POOLS = {  # opcode: (output pools, [(field, pool) of inputs])
    program.OP_EXT_G: ("G", []), program.OP_EXT_UB: ("F", []), program.OP_EXT_V: ("F", []),
    program.OP_V3: ("G", [(2, "G"), (3, "G")]),
    program.OP_V4: ("GGG", [(4, "G"), (5, "G"), (6, "G")]),
    program.OP_FPRE: ("F", [(2, "F"), (3, "G")]), program.OP_FSUF: ("F", [(2, "F"), (3, "G")]),
    program.OP_XROW: ("F", [(2, "F"), (3, "G")]), program.OP_YCOL: ("F", [(2, "G"), (3, "F")]),
    program.OP_BIL: ("B", [(2, "F"), (3, "F")]),
    program.OP_AMP_SS: ("", [(2, "F"), (3, "F")]), program.OP_AMP_VV: ("", [(2, "B"), (3, "G")]),
}


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_program_slots_well_formed(n):
    """Every operand is read after it is written, in its own pool, and no
    output overwrites an input of the same operation."""
    prog = program.build_program(n)
    size = {"G": prog.nslot, "F": prog.nslot_f, "B": 1, "A": prog.nslot_acc}
    written = set()
    for r in prog.ops:
        outp, ins = _POOLS[r[0]]
        in_keys = [(pl, r[f]) for f, pl in ins]
        outs = [(pl, r[1 + i]) for i, pl in enumerate(outp)]
        if r[0] in (program.OP_AMP_SS, program.OP_AMP_VV) and r[6] >= 0:
            (outs if r[7] & 4 else in_keys).append(("A", r[6]))
        for key in in_keys:
            assert key in written, (r, key)
        for pl, s in outs:
            assert 0 <= s < size[pl]
            assert (pl, s) not in in_keys
        written.update(outs)
    assert all(0 <= (e >> 2) < prog.ncolor for e in prog.scatter)


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_compiled_tables_match_oracle_on_cpu(ng):
    """The op tables, executed by a numpy restatement of their semantics,
    reproduce the oracle per helicity (validates the compiler, not CUDA)."""
    p = ps.generate(5, ng, 1500.0, 900 + ng, ptmin=20.0, drmin=0.4) if ng else \
        ps.generate(5, 0, 1000.0, 900)
    a, ah = table_emulator.run(ng + 2, p, per_helicity=True)
    b, bh = oracle.me(p, per_helicity=True)
    assert np.abs(a / b - 1).max() < 1e-12
    assert np.abs(ah - bh).max() < 1e-12 * bh.max()


# ----------------------------------------------------------- C ABI -------

def _header_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2510_05392_gb300 import binding
    L = binding.lib()
    names = _header_functions()
    assert len(names) >= 37
    for name in names:
        assert hasattr(L, name), name


def test_status_strings_without_gpu():
    from paper_2510_05392_gb300 import binding
    L = binding.lib()
    assert L.mg_status_string(0) == b"ok"
    assert L.mg_status_string(-1) == b"unknown or unsupported process"
    assert L.mg_status_string(-3) == b"helicities not filtered"


def test_null_arguments_rejected_without_gpu():
    from paper_2510_05392_gb300 import binding
    L = binding.lib()
    h = ctypes.c_void_p()
    assert L.mg_process_create(None, None, ctypes.byref(h)) == binding.MG_ERR_BAD_ARG
    assert L.mg_sigmakin(None, None, 1, None, None) == binding.MG_ERR_BAD_ARG
    assert L.mg_process_info(None, None) == binding.MG_ERR_BAD_ARG


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_sde_channels_match_paper(n):
    """The single-diagram-enhancement channels (diagrams of three-point
    vertices only) are as many as the paper's table lists (2 to 5 gluons; it
    gives none beyond), and as many as the trees with trivalent vertices,
    (2n - 1)!!; the colour-factor groups of the program hold one channel each."""
    g = json.load(open(GOLDEN))["processes"]["g g > t t~" + " g" * (n - 2)]
    prog = program.build_program(n)
    if g["sde_channels"] is not None:
        assert len(prog.channels) == g["sde_channels"]
    assert len(prog.channels) == int(np.prod(np.arange(1, 2 * n, 2)))
    assert prog.ncolour_groups == len(prog.channels)
    amp = [op for op in prog.ops if op[0] in (program.OP_AMP_SS, program.OP_AMP_VV)]
    used = sorted(op[1] for op in amp if op[1] >= 0)
    assert used == list(range(len(prog.channels)))     # one diagram term per channel


@pytest.mark.parametrize("n", [2, 3, 4])
def test_sde_channels_match_oracle_diagrams(n):
    """The compiler's channels are, code for code and in the same order, the
    trivalent diagrams of the oracle's own diagram enumeration with colour
    factors from explicit Gell-Mann matrices (oracle/sde.py)."""
    from oracle import sde
    prog = program.build_program(n)
    dense = np.zeros((len(prog.channels), prog.ncolor), dtype=np.int8)
    for c, ch in enumerate(prog.channels):
        for f, code in ch:
            dense[c, f] = code
    assert np.array_equal(dense, sde.channels(n)[1])
