"""Host checks of the binary process-table loader (no GPU): a damaged or
foreign table file is rejected before anything reaches the device.

The files here are synthetic 7-gluon tables (5040 flows, a two-op program)
written with the layout documented in compiler/emit.py."""
import ctypes
import itertools
import struct

import pytest

from paper_2510_05392_gb300 import binding

BAD_PROCESS = -1


def _blob(ops=None, scat=(), perms=None, magic=b"MGPROC02", version=2, ncolor=5040, trailing=b"",
          nslot=(1, 1, 1), chan_off=(0, 1), chan_flows=(1,)):
    ops = ops if ops is not None else [[2, 0, 0, 0, 0, 0, 0, 0], [10, 0, 0, 0, 0, 0, 0, 0]]
    perms = perms if perms is not None else list(itertools.permutations(range(7)))
    out = magic
    out += struct.pack("<13i", version, 7, 9, ncolor, len(ops), len(scat), *nslot, 1, 1, 1,
                       len(chan_off) - 1)
    out += struct.pack("<q3d", 11664, 30720.0, 1.0, 1.0)
    out += struct.pack(f"<{8 * len(ops)}i", *[v for r in ops for v in r])
    out += struct.pack(f"<{len(scat)}i", *scat)
    out += struct.pack("<5040q", *([1] * 5040))
    out += bytes(v for p in perms for v in p)
    out += struct.pack(f"<{len(chan_off)}i", *chan_off)
    out += struct.pack(f"<{len(chan_flows)}i", *chan_flows)
    return out + trailing


def _create(path):
    lib = binding.lib()
    h = ctypes.c_void_p()
    par = binding.mg_params(173.0, 1.4915, 0.118, binding.MG_HEL_ALL, binding.MG_FP64)
    st = lib.mg_process_create_from_tables(str(path).encode(), ctypes.byref(par), ctypes.byref(h))
    if st == 0:
        lib.mg_process_destroy(h)
    return st


def test_well_formed_file_passes_the_host_checks(tmp_path):
    f = tmp_path / "ok.bin"
    f.write_bytes(_blob())
    # accepted by the parser; without a GPU the first CUDA call then fails
    assert _create(f) in (0, binding.MG_ERR_CUDA)


@pytest.mark.parametrize("case", [
    "magic", "version", "ncolor", "truncated", "trailing", "slot_out_of_range",
    "scatter_flow_out_of_range", "scatter_range_past_end", "not_a_permutation", "bad_opcode",
    "channel_out_of_range", "channel_flow_out_of_range", "channel_code", "channel_offsets"])
def test_damaged_file_is_rejected(tmp_path, case):
    perms = list(itertools.permutations(range(7)))
    amp = [11, 0, 0, 0, 0, 1, -1, 0]                      # AMP_SS scattering entry 0
    kw = {}
    if case == "magic":
        kw["magic"] = b"MGPROC01"                         # the previous layout
    elif case == "version":
        kw["version"] = 1
    elif case == "ncolor":
        kw["ncolor"] = 5039
    elif case == "trailing":
        kw["trailing"] = b"\0"
    elif case == "slot_out_of_range":
        kw["ops"] = [[4, 1, 0, 0, 1, 2, 0, 0]]            # V3 writes gluon slot 1 of 1
    elif case == "scatter_flow_out_of_range":
        kw["ops"] = [[2, 0, 0, 0, 0, 0, 0, 0], amp]
        kw["scat"] = (5040 * 4,)
    elif case == "scatter_range_past_end":
        kw["ops"] = [[2, 0, 0, 0, 0, 0, 0, 0], [11, 0, 0, 0, 0, 2, -1, 0]]
        kw["scat"] = (0,)
    elif case == "not_a_permutation":
        perms[17] = (0, 0, 1, 2, 3, 4, 5)
        kw["perms"] = perms
    elif case == "bad_opcode":
        kw["ops"] = [[13, 0, 0, 0, 0, 0, 0, 0]]
    elif case == "channel_out_of_range":
        kw["ops"] = [[2, 0, 0, 0, 0, 0, 0, 0], [11, 1, 0, 0, 0, 1, -1, 0]]   # channel 1 of 1
        kw["scat"] = (0,)
    elif case == "channel_flow_out_of_range":
        kw["chan_flows"] = (5040 * 8 + 1,)
    elif case == "channel_code":
        kw["chan_flows"] = (5,)
    elif case == "channel_offsets":
        kw["chan_off"] = (0, 1, 1)
        kw["chan_flows"] = (1,)
    data = _blob(**kw)
    if case == "truncated":
        data = data[:-100]
    f = tmp_path / f"{case}.bin"
    f.write_bytes(data)
    assert _create(f) == BAD_PROCESS


def test_missing_file(tmp_path):
    assert _create(tmp_path / "absent.bin") == BAD_PROCESS


def test_emitter_round_trip(tmp_path):
    """The process compiler's table file holds exactly its program, scatter
    list, colour row, flow orderings and channel colour factors (written for
    g g > t t~ g g here; the library itself only loads 7-gluon files)."""
    from paper_2510_05392_gb300.compiler import colour, emit, program
    f = tmp_path / "g4.bin"
    emit.emit_blob(4, str(f))
    data = f.read_bytes()
    assert data[:8] == b"MGPROC02"
    h = struct.unpack_from("<13i", data, 8)
    den, iden, fd, fc = struct.unpack_from("<q3d", data, 60)
    prog = program.build_program(4)
    assert h == (2, 4, 6, 24, len(prog.ops), len(prog.scatter), prog.nslot, prog.nslot_f,
                 prog.nslot_acc, prog.ncolour_groups, prog.ndiagrams, prog.nterms, 105)
    off = 60 + 32
    ops = struct.unpack_from(f"<{8 * h[4]}i", data, off)
    off += 32 * h[4]
    assert [list(ops[8 * i:8 * i + 8]) for i in range(h[4])] == [list(r) for r in prog.ops]
    scat = struct.unpack_from(f"<{h[5]}i", data, off)
    off += 4 * h[5]
    assert list(scat) == list(prog.scatter)
    row = struct.unpack_from("<24q", data, off)
    off += 8 * 24
    chat, d, perms = colour.colour_matrix(4)
    assert den == d and list(row) == list(chat[0])   # row of the identity ordering
    assert list(data[off:off + 24 * 4]) == [v for p in perms for v in p]
    off += 24 * 4
    cho = struct.unpack_from("<106i", data, off)
    off += 4 * 106
    chf = struct.unpack_from(f"<{cho[-1]}i", data, off)
    assert off + 4 * cho[-1] == len(data)
    assert [[(e >> 3, e & 7) for e in chf[cho[c]:cho[c + 1]]] for c in range(105)] == \
        [list(ch) for ch in prog.channels]
    assert iden == 512.0 and fd == emit.algorithmic_flops(prog)["diagram"]
