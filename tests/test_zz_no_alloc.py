"""GPU test of mg_filter_helicities_noalloc, the helicity filter that takes
its scratch from a fixed array inside the library instead of cudaMalloc.

It is meant for callers that cannot allocate device memory themselves or
through the library (memory owned by another allocator, or no device-wide
synchronisation from cudaFree allowed).  The test calls it through the C ABI
twice in a row and compares with mg_filter_helicities: the mask and count
must be identical (bit-exact, like every helicity-mask test here), and the
matrix elements computed after either filter must agree to 1e-9 relative.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(p, mom, n=None):
    L = binding.lib()
    f = L.mg_filter_helicities_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_int)]
    f.restype = ctypes.c_int
    ng = ctypes.c_int(-7)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(p.handle, ctypes.c_void_p(mom.data_ptr()), mom.shape[0] if n is None else n, stream,
           ctypes.byref(ng))
    return rc, ng.value


@pytest.mark.parametrize("ng_final,sqrts", [(0, 1000.0), (2, 1500.0), (3, 1500.0)])
def test_noalloc_filter_matches_allocating_filter(ng_final, sqrts):
    proc = "g g > t t~" + " g" * ng_final
    kw = dict(ptmin=20.0, drmin=0.4) if ng_final else {}
    test = torch.from_numpy(ps.generate(16, ng_final, sqrts, 12345, **kw)).cuda()
    mom = torch.from_numpy(ps.generate(101, ng_final, sqrts, 777, **kw)).cuda()

    ref = binding.Process(proc)
    nref = ref.filter_helicities(test)
    mref = ref.helicity_mask()
    out_ref = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    ref.sigmakin(mom, out_ref)

    p = binding.Process(proc)
    for _ in range(2):  # two calls in a row share (and reuse) the scratch array
        rc, n = _noalloc(p, test)
        assert rc == binding.MG_OK, binding.lib().mg_status_string(rc)
        assert n == nref
        assert np.array_equal(p.helicity_mask(), mref)
        out = torch.empty_like(out_ref)
        p.sigmakin(mom, out)
        torch.cuda.synchronize()
        rel = (out / out_ref - 1).abs().max().item()
        assert rel <= 1e-9


def test_noalloc_filter_full_array():
    """g g > t t~ g g: 64 test events x 64 helicities, the most events the
    fixed array takes, with the mask and count bit-exact against the
    allocating filter on the same events, twice in a row."""
    kw = dict(ptmin=20.0, drmin=0.4)
    test = torch.from_numpy(ps.generate(64, 2, 1500.0, 4321, **kw)).cuda()
    ref = binding.Process("g g > t t~ g g")
    nref = ref.filter_helicities(test)
    p = binding.Process("g g > t t~ g g")
    for _ in range(2):
        rc, n = _noalloc(p, test)
        assert rc == binding.MG_OK and n == nref == 64
        assert np.array_equal(p.helicity_mask(), ref.helicity_mask())


def test_noalloc_filter_rejects_too_many_events():
    test = torch.from_numpy(ps.generate(65, 1, 1500.0, 5, ptmin=20.0, drmin=0.4)).cuda()
    p = binding.Process("g g > t t~ g")
    rc, _ = _noalloc(p, test)
    assert rc == binding.MG_ERR_BAD_ARG
    rc, _ = _noalloc(p, test, n=0)
    assert rc == binding.MG_ERR_BAD_ARG
    rc, n = _noalloc(p, test, n=64)
    assert rc == binding.MG_OK and n == 32
