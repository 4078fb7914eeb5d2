"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerance: per-event relative error <= 1e-9 on the FP64 path (the FP64
target for per-event matrix elements), max over every checked event.
"""
import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-9
PROCS = {  # ngluon_final: (process, sqrt(s), nevt for full parity)
    0: ("g g > t t~", 1000.0, 4096 + 37),
    1: ("g g > t t~ g", 1500.0, 1024 + 5),
    2: ("g g > t t~ g g", 1500.0, 384 + 3),
    3: ("g g > t t~ g g g", 1500.0, 96 + 1),
}


def _events(ng, n, seed, sqrts):
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    return ps.generate(n, ng, sqrts, seed, **kw)


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _process(proc, **kw):
    p = binding.Process(proc, **kw)
    return p


def _filtered(proc, ng, sqrts):
    p = _process(proc)
    p.filter_helicities(_gpu(_events(ng, 16, 12345, sqrts)))
    return p


@pytest.mark.parametrize("ng", sorted(PROCS))
def test_me_parity_fp64(ng):
    proc, sqrts, n = PROCS[ng]
    mom = _events(ng, n, 1000 + ng, sqrts)
    p = _filtered(proc, ng, sqrts)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin(_gpu(mom), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.me(mom)
    rel = np.abs(got / ref - 1)
    assert rel.max() <= RTOL, (rel.max(), np.median(rel))


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_per_helicity_parity(ng):
    proc, sqrts, _ = PROCS[ng]
    n = 33
    mom = _events(ng, n, 2000 + ng, sqrts)
    p = _filtered(proc, ng, sqrts)
    nhel = 1 << (ng + 4)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    outh = torch.empty((n, nhel), dtype=torch.float64, device="cuda")
    p.sigmakin_hel(_gpu(mom), out, outh)
    torch.cuda.synchronize()
    ref, refh = oracle.me(mom, per_helicity=True)
    gh = outh.cpu().numpy()
    assert np.abs(gh - refh).max() <= RTOL * refh.max()
    np.testing.assert_allclose(gh.sum(1), out.cpu().numpy(), rtol=1e-12)


@pytest.mark.parametrize("ng", [0, 1, 2, 3])
def test_helicity_mask_bit_exact(ng):
    proc, sqrts, _ = PROCS[ng]
    test_events = _events(ng, 16, 12345, sqrts)
    p = _process(proc)
    with pytest.raises(binding.MGError):
        p.helicity_mask()
    ngood = p.filter_helicities(_gpu(test_events))
    mask = p.helicity_mask()
    ref = oracle.good_helicity_mask(test_events)
    assert np.array_equal(mask, ref)
    assert ngood == int(ref.sum()) == 1 << (ng + 4)


@pytest.mark.parametrize("ng", [0, 1, 2, 3, 4])
def test_colour_matrix_through_abi_bit_exact(ng):
    proc = "g g > t t~" + " g" * ng
    p = _process(proc)
    C, D = p.color_matrix()
    Ch, Dh, _ = oracle.color_data(ng + 2)
    assert D == Dh
    assert np.array_equal(C, Ch)
    info = p.info()
    assert info.ncolor == len(Ch)


@pytest.mark.parametrize("tpe", [1, 2, 4, 8, 16, 32])
def test_launch_shapes_agree(tpe):
    proc, sqrts, _ = PROCS[2]
    mom = _gpu(_events(2, 301, 77, sqrts))
    p = _filtered(proc, 2, sqrts)
    ref = torch.empty(301, dtype=torch.float64, device="cuda")
    p.sigmakin(mom, ref)
    p.set_launch(threads_per_event=tpe, block=64 if tpe < 8 else 128)
    out = torch.empty_like(ref)
    p.sigmakin(mom, out)
    torch.cuda.synchronize()
    rel = (out / ref - 1).abs().max().item()
    assert rel < 1e-13


def test_edge_cases_and_errors():
    proc, sqrts, _ = PROCS[1]
    p = _process(proc)
    mom = _gpu(_events(1, 3, 5, sqrts))
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.MGError) as e:
        p.sigmakin(mom, out)
    assert e.value.status == binding.MG_ERR_NOT_FILTERED
    p.filter_helicities(_gpu(_events(1, 16, 12345, sqrts)))
    # nevt = 0 is a no-op
    empty = torch.empty((0, 5, 4), dtype=torch.float64, device="cuda")
    p.sigmakin(empty, torch.empty(0, dtype=torch.float64, device="cuda"))
    # host pointers are rejected
    with pytest.raises(binding.MGError) as e:
        p.sigmakin(torch.zeros((3, 5, 4), dtype=torch.float64), out)
    assert e.value.status == binding.MG_ERR_BAD_ARG
    # one event
    one = _events(1, 1, 6, sqrts)
    o1 = torch.empty(1, dtype=torch.float64, device="cuda")
    p.sigmakin(_gpu(one), o1)
    torch.cuda.synchronize()
    assert abs(o1.item() / oracle.me(one)[0] - 1) < RTOL
    with pytest.raises(binding.MGError) as e:
        binding.Process("g g > t t~ q")
    assert e.value.status == binding.MG_ERR_BAD_PROCESS


def test_hel_all_mode_matches_filtered():
    proc, sqrts, _ = PROCS[2]
    mom = _gpu(_events(2, 64, 8, sqrts))
    a = _filtered(proc, 2, sqrts)
    b = _process(proc, hel_mode=binding.MG_HEL_ALL)
    oa = torch.empty(64, dtype=torch.float64, device="cuda")
    ob = torch.empty_like(oa)
    a.sigmakin(mom, oa)
    b.sigmakin(mom, ob)
    torch.cuda.synchronize()
    assert torch.equal(oa, ob)


def test_full_size_workload_sampled():
    """The benchmark workload (g g > t t~ g g, 524288 events, sqrt(s) = 1500,
    cuts) in the benchmark's launch configuration, checked on a strided
    sample of events against the oracle."""
    mom = ps.workload("ggttgg_524288")
    p = _filtered("g g > t t~ g g", 2, 1500.0)
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    p.sigmakin(_gpu(mom), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(0, len(mom), 2053), [len(mom) - 1]]))
    ref = oracle.me(mom[idx])
    assert np.abs(got[idx] / ref - 1).max() <= RTOL
    assert np.all(np.isfinite(got)) and np.all(got > 0)


def test_ggttgggg_small():
    mom = _events(4, 4, 31, 2000.0)
    p = _process("g g > t t~ g g g g", hel_mode=binding.MG_HEL_ALL)
    p.set_launch(threads_per_event=32, block=128)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    p.sigmakin(_gpu(mom), out)
    torch.cuda.synchronize()
    ref = oracle.me(mom)
    assert np.abs(out.cpu().numpy() / ref - 1).max() <= RTOL


def test_pointer_and_size_errors():
    """Negative sizes, null, misaligned and host pointers, bad launch shapes:
    each returns its documented status and leaves the process usable."""
    proc, sqrts, _ = PROCS[1]
    p = _filtered(proc, 1, sqrts)
    L = binding.lib()
    mom = _gpu(_events(1, 4, 9, sqrts))
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    h = p.handle
    assert L.mg_sigmakin(h, mom.data_ptr(), -1, out.data_ptr(), None) == binding.MG_ERR_BAD_ARG
    assert L.mg_sigmakin(h, None, 4, out.data_ptr(), None) == binding.MG_ERR_BAD_ARG
    assert L.mg_sigmakin(h, mom.data_ptr(), 4, None, None) == binding.MG_ERR_BAD_ARG
    assert L.mg_sigmakin(h, mom.data_ptr() + 4, 4, out.data_ptr(), None) == binding.MG_ERR_BAD_ARG
    assert L.mg_sigmakin(h, mom.data_ptr(), 4, out.data_ptr() + 4, None) == binding.MG_ERR_BAD_ARG
    host = torch.zeros(4, dtype=torch.float64)
    assert L.mg_sigmakin(h, mom.data_ptr(), 4, host.data_ptr(), None) == binding.MG_ERR_BAD_ARG
    for tpe, block in [(3, 0), (64, 0), (0, 256), (0, 48), (0, 16)]:
        assert L.mg_set_launch(h, tpe, block) == binding.MG_ERR_BAD_ARG
    assert L.mg_filter_helicities(h, mom.data_ptr(), 0, None, None) == binding.MG_ERR_BAD_ARG
    assert L.mg_filter_helicities(h, mom.data_ptr(), 65537, None, None) == binding.MG_ERR_BAD_ARG
    # still usable, ragged sizes around a warp
    for n in (31, 33):
        m = _events(1, n, 100 + n, sqrts)
        o = torch.empty(n, dtype=torch.float64, device="cuda")
        p.sigmakin(_gpu(m), o)
        torch.cuda.synchronize()
        assert np.abs(o.cpu().numpy() / oracle.me(m) - 1).max() < RTOL
