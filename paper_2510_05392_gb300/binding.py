"""Thin Python binding of the C ABI in include/mgpu.h (argument marshalling only).

Every computation runs in the CUDA library; this module only converts torch
tensors to device pointers and CUDA streams to handles.  Importing it loads
``_build/libmgpu.so`` and raises if the library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmgpu.so")

MG_OK = 0
MG_ERR_BAD_PROCESS = -1
MG_ERR_BAD_ARG = -2
MG_ERR_NOT_FILTERED = -3
MG_ERR_CUDA = -4
MG_ERR_DEVICE_TIMEOUT = -5
MG_ERR_NO_MEMORY = -6
MG_ERR_UNSUPPORTED = -7
MG_HEL_FILTERED, MG_HEL_ALL = 0, 1
MG_FP64, MG_MIXED_BF16 = 0, 1


class mg_params(ctypes.Structure):
    _fields_ = [("mt", ctypes.c_double), ("wt", ctypes.c_double), ("alphas", ctypes.c_double),
                ("hel_mode", ctypes.c_int), ("precision", ctypes.c_int)]


class mg_info(ctypes.Structure):
    _fields_ = [("npar", ctypes.c_int), ("ngluon", ctypes.c_int), ("ndiagrams", ctypes.c_int),
                ("nterms", ctypes.c_int), ("ncolor", ctypes.c_int), ("nhel", ctypes.c_int),
                ("ngood", ctypes.c_int), ("nslot", ctypes.c_int), ("nslot_top", ctypes.c_int),
                ("nops", ctypes.c_int),
                ("njamp_updates", ctypes.c_int), ("denom", ctypes.c_int64),
                ("iden", ctypes.c_double), ("flops_diagram", ctypes.c_double),
                ("flops_colour", ctypes.c_double), ("nchannel", ctypes.c_int)]


class mg_sigmakin_extras(ctypes.Structure):
    _fields_ = [("alphas_dev", ctypes.c_void_p), ("channel", ctypes.c_int),
                ("sde_weight_dev", ctypes.c_void_p), ("flow_weight_dev", ctypes.c_void_p),
                ("rnd_hel_dev", ctypes.c_void_p), ("hel_out_dev", ctypes.c_void_p),
                ("rnd_col_dev", ctypes.c_void_p), ("col_out_dev", ctypes.c_void_p),
                ("channel_ids_dev", ctypes.c_void_p)]


class MGError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().mg_status_string(status).decode()
        if status == MG_ERR_CUDA:
            msg += f" ({lib().mg_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg} [{status}]")
        self.status = status


_lib = None

_VP = ctypes.c_void_p
_SIGS = {
    "mg_process_create": ([ctypes.c_char_p, ctypes.POINTER(mg_params), ctypes.POINTER(_VP)], ctypes.c_int),
    "mg_process_create_from_tables": ([ctypes.c_char_p, ctypes.POINTER(mg_params), ctypes.POINTER(_VP)], ctypes.c_int),
    "mg_filter_helicities": ([_VP, _VP, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "mg_sigmakin": ([_VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "mg_sigmakin_hel": ([_VP, _VP, ctypes.c_int64, _VP, _VP, _VP], ctypes.c_int),
    "mg_set_launch": ([_VP, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "mg_process_info": ([_VP, ctypes.POINTER(mg_info)], ctypes.c_int),
    "mg_color_matrix": ([_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "mg_helicity_mask": ([_VP, ctypes.POINTER(ctypes.c_uint8)], ctypes.c_int),
    "mg_sde_channels": ([_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int8)], ctypes.c_int),
    "mg_process_destroy": ([_VP], None),
    "mg_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "mg_last_cuda_error": ([], ctypes.c_char_p),
    "mg_device_status": ([_VP, _VP], ctypes.c_int),
    "mg_sigmakin_ex": ([_VP, _VP, ctypes.c_int64, ctypes.POINTER(mg_sigmakin_extras), _VP, _VP], ctypes.c_int),
    "mg_debug_inject_stall": ([_VP, ctypes.c_uint], ctypes.c_int),
    "mg_debug_jamp_buffer": ([_VP, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
    "mg_filter_helicities_noalloc": ([_VP, _VP, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "mg_batch_create": ([ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_VP), ctypes.POINTER(_VP)], ctypes.c_int),
    "mg_batch_run": ([_VP, _VP], ctypes.c_int),
    "mg_batch_autotune": ([_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "mg_batch_config": ([_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "mg_batch_destroy": ([_VP], None),
    "mg_sigmakin_batch": ([ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_VP), _VP], ctypes.c_int),
    "mg_set_kernel_timing": ([_VP, ctypes.c_int], ctypes.c_int),
    "mg_kernel_times": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "mg_launch_count": ([ctypes.POINTER(ctypes.c_ulonglong)], ctypes.c_int),
    "mg_debug_colour_sum_rows": ([_VP, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "mg_probe_fp64_peak": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
}


def lib():
    """The loaded CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status, where):
    if status != MG_OK:
        raise MGError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


TABLE_FILE_PROCESS = "g g > t t~ g g g g g"


class Process:
    """Owner of one mg_process handle."""

    def __init__(self, process: str, mt=173.0, wt=1.4915, alphas=0.118,
                 hel_mode=MG_HEL_FILTERED, precision=MG_FP64):
        self._h = _VP()
        self.params = mg_params(mt, wt, alphas, hel_mode, precision)
        if " ".join(process.split()) == TABLE_FILE_PROCESS:
            # too large to compile into the library: tables from the process
            # compiler's binary file (generated once, a few minutes)
            from . import build
            path = build.process_tables(7)
            _check(lib().mg_process_create_from_tables(path.encode(), ctypes.byref(self.params),
                                                       ctypes.byref(self._h)),
                   "mg_process_create_from_tables")
        else:
            _check(lib().mg_process_create(process.encode(), ctypes.byref(self.params),
                                           ctypes.byref(self._h)), "mg_process_create")
        self.process = process

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().mg_process_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> mg_info:
        i = mg_info()
        _check(lib().mg_process_info(self._h, ctypes.byref(i)), "mg_process_info")
        return i

    def filter_helicities(self, momenta, stream=None) -> int:
        n = ctypes.c_int(0)
        _check(lib().mg_filter_helicities(self._h, _ptr(momenta), momenta.shape[0],
                                          _stream(stream), ctypes.byref(n)), "mg_filter_helicities")
        return n.value

    def sigmakin(self, momenta, out, stream=None):
        _check(lib().mg_sigmakin(self._h, _ptr(momenta), momenta.shape[0], _ptr(out),
                                 _stream(stream)), "mg_sigmakin")
        return out

    def sigmakin_hel(self, momenta, out, out_hel, stream=None):
        _check(lib().mg_sigmakin_hel(self._h, _ptr(momenta), momenta.shape[0], _ptr(out),
                                     _ptr(out_hel), _stream(stream)), "mg_sigmakin_hel")
        return out_hel

    def device_status(self, stream=None) -> int:
        """MG_OK or the status of the device-side work issued so far (syncs)."""
        return lib().mg_device_status(self._h, _stream(stream))

    def set_kernel_timing(self, max_launches: int):
        """Record CUDA events around each later kernel launch (0 = off)."""
        _check(lib().mg_set_kernel_timing(self._h, max_launches), "mg_set_kernel_timing")

    def kernel_times(self, reset=True):
        """{kind: (device ms summed, launches)} since the last reset for the
        kinds 'diagram', 'colour' (the colour-sum kernel of the mixed path
        or of a table-file process), 'event_sum' (waits for the events)."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int * 3)()
        _check(lib().mg_kernel_times(self._h, int(reset), ms, n), "mg_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(("diagram", "colour", "event_sum"))}

    def sigmakin_ex(self, momenta, out=None, alphas=None, channel=-1, sde=None, flow=None,
                    rnd_hel=None, hel_out=None, rnd_col=None, col_out=None, channel_ids=None,
                    stream=None):
        x = mg_sigmakin_extras(_ptr(alphas), channel, _ptr(sde), _ptr(flow), _ptr(rnd_hel),
                               _ptr(hel_out), _ptr(rnd_col), _ptr(col_out), _ptr(channel_ids))
        _check(lib().mg_sigmakin_ex(self._h, _ptr(momenta), momenta.shape[0], ctypes.byref(x),
                                    _ptr(out), _stream(stream)), "mg_sigmakin_ex")
        return out

    def set_launch(self, threads_per_event=0, block=0):
        _check(lib().mg_set_launch(self._h, threads_per_event, block), "mg_set_launch")

    def color_matrix(self):
        import numpy as np
        nc = self.info().ncolor
        a = np.zeros(nc * nc, dtype=np.int64)
        d = ctypes.c_int64(0)
        _check(lib().mg_color_matrix(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     ctypes.byref(d)), "mg_color_matrix")
        return a.reshape(nc, nc), d.value

    def sde_channels(self):
        """Colour-factor codes [nchannel][ncolor] (int8) of the channels."""
        import numpy as np
        n = ctypes.c_int(0)
        _check(lib().mg_sde_channels(self._h, ctypes.byref(n), None), "mg_sde_channels")
        codes = np.zeros((n.value, self.info().ncolor), dtype=np.int8)
        _check(lib().mg_sde_channels(self._h, None, codes.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))),
               "mg_sde_channels")
        return codes

    def helicity_mask(self):
        import numpy as np
        m = np.zeros(self.info().nhel, dtype=np.uint8)
        _check(lib().mg_helicity_mask(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
               "mg_helicity_mask")
        return m


def launch_count() -> int:
    """Kernel launches the library has issued so far (graph replays and the
    FP64 peak probe not included)."""
    n = ctypes.c_ulonglong(0)
    _check(lib().mg_launch_count(ctypes.byref(n)), "mg_launch_count")
    return n.value


class Batch:
    """Owner of one mg_batch plan over (Process, momenta tensor, output tensor)
    blocks; the tensors must stay alive while the plan is used."""

    def __init__(self, blocks):
        n = len(blocks)
        self._keep = blocks
        procs = (_VP * n)(*[p.handle for p, _, _ in blocks])
        moms = (_VP * n)(*[m.data_ptr() for _, m, _ in blocks])
        outs = (_VP * n)(*[o.data_ptr() for _, _, o in blocks])
        nev = (ctypes.c_int64 * n)(*[m.shape[0] for _, m, _ in blocks])
        self._h = _VP()
        _check(lib().mg_batch_create(n, procs, moms, nev, outs, ctypes.byref(self._h)),
               "mg_batch_create")
        self.n = n

    def run(self, stream=None):
        _check(lib().mg_batch_run(self._h, _stream(stream)), "mg_batch_run")

    def autotune(self, reps=2, stream=None) -> float:
        ms = ctypes.c_double(0.0)
        _check(lib().mg_batch_autotune(self._h, _stream(stream), reps, ctypes.byref(ms)),
               "mg_batch_autotune")
        return ms.value

    def config(self):
        t = (ctypes.c_int * self.n)()
        c = ctypes.c_int(0)
        _check(lib().mg_batch_config(self._h, t, ctypes.byref(c)), "mg_batch_config")
        return list(t), c.value

    def close(self):
        if self._h:
            lib().mg_batch_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
