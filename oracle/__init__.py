"""CPU oracle for g g -> t t~ + n g matrix elements.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library product
never does.  It shares no code with the CUDA path.

Pieces (each cites the passage it follows in its own module):
  bg.c            colour-ordered amplitudes by Berends-Giele recursion, helicity
                  sum and colour quadratic form, FP64 (-ffp-contract=off)
  color.py        exact rational colour matrix by recursive Fierz identities
  topology.py     brute-force diagram counter
  closed_form.py  Combridge's g g -> Q Qbar formula

Parity status: every function here is pinned by tests/test_oracle*.py
(closed form, the massless Parke-Taylor amplitudes, gauge, Lorentz and Bose
invariance, brute-force colour traces, diagram counts, paper table counts).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from functools import lru_cache

import numpy as np

from . import color as _color

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

DEFAULT_PARAMS = dict(mt=173.0, wt=1.4915, alphas=0.118)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile bg.c into _build/liboracle.so (OpenMP when available)."""
    src = os.path.join(HERE, "bg.c")
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_me.argtypes = [ctypes.c_int, dp, ctypes.c_int64, dp,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_uint8), dp, dp, ctypes.c_int]
            lib.oracle_me.restype = ctypes.c_int
            lib.oracle_amplitudes.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
            lib.oracle_amplitudes.restype = ctypes.c_int
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_externals.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_externals.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def ngluons(process: str) -> int:
    """Number of gluons n (incoming included) of 'g g > t t~ g ...'."""
    toks = process.replace(">", " > ").split()
    if toks[:5] != ["g", "g", ">", "t", "t~"] or any(t != "g" for t in toks[5:]):
        raise ValueError(f"unsupported process: {process!r}")
    return 2 + len(toks) - 5


def iden(n: int) -> int:
    """Averaging factor: 4 initial spins x 64 initial colours x (n-2)! identical final gluons."""
    return 256 * math.factorial(n - 2)


@lru_cache(maxsize=None)
def color_data(n: int):
    """(C_hat int64 [nc][nc], D, perms int32 [nc][n]) from the exact Fierz builder."""
    Chat, D, perms = _color.color_matrix(n)
    return (np.ascontiguousarray(np.array(Chat, dtype=np.int64)), int(D),
            np.ascontiguousarray(np.array(perms, dtype=np.int32)))


def threads() -> int:
    return _load().oracle_threads()


def me(momenta: np.ndarray, mt: float = DEFAULT_PARAMS["mt"], wt: float = DEFAULT_PARAMS["wt"],
       alphas: float = DEFAULT_PARAMS["alphas"], hel_mask=None, per_helicity: bool = False,
       nthreads: int = 0):
    """Averaged |M|^2 for momenta [nevt][npar][4] (FP64).

    Returns me [nevt], or (me, me_hel [nevt][2^npar]) when ``per_helicity``.
    """
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    nevt, npar, _ = mom.shape
    n = npar - 2
    Chat, D, perms = color_data(n)
    par = np.array([mt, wt, math.sqrt(4 * math.pi * alphas)], dtype=np.float64)
    out = np.zeros(nevt)
    hel = np.zeros((nevt, 1 << npar)) if per_helicity else None
    mask = None if hel_mask is None else np.ascontiguousarray(hel_mask, dtype=np.uint8)
    rc = _load().oracle_me(n, _ptr(mom, ctypes.c_double), nevt, _ptr(par, ctypes.c_double),
                           _ptr(Chat, ctypes.c_int64), D, len(perms), _ptr(perms, ctypes.c_int),
                           float(iden(n)), None if mask is None else _ptr(mask, ctypes.c_uint8),
                           _ptr(out, ctypes.c_double),
                           None if hel is None else _ptr(hel, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_me failed: {rc}")
    return (out, hel) if per_helicity else out


def amplitudes(p_event: np.ndarray, hel: int, gauge_leg: int = -1,
               mt: float = DEFAULT_PARAMS["mt"], wt: float = DEFAULT_PARAMS["wt"]):
    """Colour-ordered amplitudes A_s (no couplings) of one event [npar][4] and
    helicity index, in the ordering of ``color_data(n)[2]``.  ``gauge_leg``
    (0..n-1, gluon index in particle order) replaces that gluon's polarisation
    by its momentum."""
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    n = p.shape[0] - 2
    _, _, perms = color_data(n)
    par = np.array([mt, wt], dtype=np.float64)
    out = np.zeros(2 * len(perms))
    rc = _load().oracle_amplitudes(n, _ptr(p, ctypes.c_double), int(hel), int(gauge_leg),
                                   _ptr(par, ctypes.c_double), len(perms),
                                   _ptr(perms, ctypes.c_int), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("oracle_amplitudes failed")
    return out[0::2] + 1j * out[1::2]


def externals(p_event: np.ndarray, hel: int):
    """External states of one event [npar][4] and helicity index, in the
    conventions of the Berends-Giele amplitudes: (eps [n][4] complex, incoming
    eps and outgoing eps*; kin [n][4] incoming gluon momenta; ubar(p3) [4];
    v(p4) [4]), gluons in particle order."""
    p = np.ascontiguousarray(p_event, dtype=np.float64)
    n = p.shape[0] - 2
    eps = np.zeros(8 * n)
    kin = np.zeros(4 * n)
    ub = np.zeros(8)
    v = np.zeros(8)
    rc = _load().oracle_externals(n, _ptr(p, ctypes.c_double), int(hel), _ptr(eps, ctypes.c_double),
                                  _ptr(kin, ctypes.c_double), _ptr(ub, ctypes.c_double),
                                  _ptr(v, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("oracle_externals failed")
    c = lambda a: a[0::2] + 1j * a[1::2]
    return c(eps).reshape(n, 4), kin.reshape(n, 4), c(ub), c(v)


def good_helicity_mask(momenta_test: np.ndarray, rel: float = 1e-14, **kw) -> np.ndarray:
    """Helicity filter rule: h is good when |M_h|^2 > rel * max_h' |M_h'|^2 on
    any of the test events (the paper keeps the helicities with a non-zero
    contribution, Sec. 2.2 and Sec. 4.6, without stating a threshold)."""
    _, mh = me(momenta_test, per_helicity=True, **kw)
    mx = mh.max(axis=1, keepdims=True)
    return (mh > rel * mx).any(axis=0).astype(np.uint8)
