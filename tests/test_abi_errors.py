"""Host-side error paths of the C ABI that return before any CUDA call
(no GPU needed): every one gives its documented status."""
import ctypes

import pytest

from paper_2510_05392_gb300 import binding


def _create(process, **kw):
    par = dict(mt=173.0, wt=1.4915, alphas=0.118, hel_mode=binding.MG_HEL_FILTERED,
               precision=binding.MG_FP64)
    par.update(kw)
    h = ctypes.c_void_p()
    p = binding.mg_params(par["mt"], par["wt"], par["alphas"], par["hel_mode"], par["precision"])
    st = binding.lib().mg_process_create(process.encode() if process is not None else None,
                                         ctypes.byref(p), ctypes.byref(h))
    if st == binding.MG_OK:
        binding.lib().mg_process_destroy(h)
    return st


@pytest.mark.parametrize("process", ["g g > t t~ q", "u u~ > t t~", "g g > t t~ g g g g g g", "",
                                     "g g >", "g g > t t~ g g g g g"])
def test_unknown_process(process):
    # the 2 -> 7 process has no compiled-in tables: it is created from its table file
    assert _create(process) == binding.MG_ERR_BAD_PROCESS


@pytest.mark.parametrize("kw", [dict(mt=0.0), dict(mt=-1.0), dict(wt=-0.1), dict(alphas=0.0),
                                dict(hel_mode=7), dict(precision=3)])
def test_bad_parameters(kw):
    assert _create("g g > t t~ g", **kw) == binding.MG_ERR_BAD_ARG


def test_null_arguments():
    lib = binding.lib()
    h = ctypes.c_void_p()
    assert lib.mg_process_create(None, None, ctypes.byref(h)) == binding.MG_ERR_BAD_ARG
    assert lib.mg_process_create(b"g g > t t~", None, None) == binding.MG_ERR_BAD_ARG
    assert lib.mg_sigmakin(None, None, 1, None, None) == binding.MG_ERR_BAD_ARG
    assert lib.mg_filter_helicities(None, None, 1, None, None) == binding.MG_ERR_BAD_ARG
    assert lib.mg_set_launch(None, 1, 32) == binding.MG_ERR_BAD_ARG
    assert lib.mg_device_status(None, None) == binding.MG_ERR_BAD_ARG
    assert lib.mg_process_create_from_tables(None, None, ctypes.byref(h)) == binding.MG_ERR_BAD_ARG


def test_status_strings():
    lib = binding.lib()
    for s in (binding.MG_OK, binding.MG_ERR_BAD_PROCESS, binding.MG_ERR_BAD_ARG,
              binding.MG_ERR_NOT_FILTERED, binding.MG_ERR_CUDA, binding.MG_ERR_DEVICE_TIMEOUT,
              binding.MG_ERR_NO_MEMORY, binding.MG_ERR_UNSUPPORTED):
        assert lib.mg_status_string(s).decode() not in ("", "unknown status")
    assert lib.mg_status_string(-99).decode() == "unknown status"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library there is no fallback: the first call
    that needs it raises."""
    from paper_2510_05392_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libmgpu.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(ImportError):
        binding.lib()
    with pytest.raises(ImportError):
        binding.Process("g g > t t~ g g")
