"""GPU: the mixed-precision path (FP64 diagrams, tensor-core colour sum).

Bound: per-event relative error <= 1e-6 against the FP64 oracle, the bound
stated for the mixed colour sum (jamps in three BF16 pieces, colour matrix in
two, FP32 accumulation on the tensor cores, FP64 epilogue).
"""
import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_RTOL = 1e-6
# ng = 4 (720 flows) runs the block-triangular kernel (128-colour blocks)
CASES = {0: (1000.0, 515), 1: (1500.0, 301), 2: (1500.0, 257), 3: (1500.0, 65), 4: (2000.0, 24)}


def _events(ng, n, seed, sqrts):
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    return ps.generate(n, ng, sqrts, seed, **kw)


def _mixed(ng, sqrts):
    p = binding.Process("g g > t t~" + " g" * ng, precision=binding.MG_MIXED_BF16)
    p.filter_helicities(torch.from_numpy(_events(ng, 16, 12345, sqrts)).cuda())
    return p


@pytest.mark.parametrize("ng", sorted(CASES))
def test_mixed_colour_sum_within_bound(ng):
    sqrts, n = CASES[ng]
    mom = _events(ng, n, 3100 + ng, sqrts)
    p = _mixed(ng, sqrts)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin(torch.from_numpy(mom).cuda(), out)
    assert p.device_status() == binding.MG_OK
    got = out.cpu().numpy()
    ref = oracle.me(mom)
    rel = np.abs(got / ref - 1)
    print(f"ng={ng}: max rel {rel.max():.3e} median {np.median(rel):.3e}")
    assert rel.max() <= MIXED_RTOL


def test_mixed_matches_fp64_path_on_gpu():
    sqrts, n = 1500.0, 200
    mom = torch.from_numpy(_events(2, n, 3200, sqrts)).cuda()
    a = binding.Process("g g > t t~ g g")
    a.filter_helicities(torch.from_numpy(_events(2, 16, 12345, sqrts)).cuda())
    b = _mixed(2, sqrts)
    oa = torch.empty(n, dtype=torch.float64, device="cuda")
    ob = torch.empty_like(oa)
    a.sigmakin(mom, oa)
    b.sigmakin(mom, ob)
    torch.cuda.synchronize()
    assert ((ob / oa - 1).abs().max().item()) <= MIXED_RTOL


def test_mixed_rejects_per_helicity():
    p = _mixed(1, 1500.0)
    mom = torch.from_numpy(_events(1, 4, 1, 1500.0)).cuda()
    with pytest.raises(binding.MGError) as e:
        p.sigmakin_hel(mom, torch.empty(4, dtype=torch.float64, device="cuda"),
                       torch.empty((4, 32), dtype=torch.float64, device="cuda"))
    assert e.value.status == binding.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("ng", [2, 4])
def test_bounded_wait_reports_timeout_and_context_survives(ng):
    """A barrier that never completes (test hook) makes the tensor-core kernel
    (single-tile for 24 flows, block-triangular for 720) give up after its
    wait limit; the status is reported and the next call works."""
    sqrts = CASES[ng][0]
    p = _mixed(ng, sqrts)
    mom_np = _events(ng, 1, 3300, sqrts)          # one event: 128 or 512 rows
    mom = torch.from_numpy(mom_np).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    L = binding.lib()
    assert L.mg_debug_inject_stall(p.handle, 1024) == binding.MG_OK
    p.sigmakin(mom, out)
    assert p.device_status() == binding.MG_ERR_DEVICE_TIMEOUT
    assert L.mg_debug_inject_stall(p.handle, 0) == binding.MG_OK
    p.sigmakin(mom, out)
    assert p.device_status() == binding.MG_OK
    assert abs(out.item() / oracle.me(mom_np)[0] - 1) <= MIXED_RTOL


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_exact_inputs_bit_identical(ng):
    """Rows whose values are small integers (exact in one BF16 piece) and the
    integer matrix D*C: every product and partial sum of the tensor-core colour
    sum is an exactly representable integer (below 2^24 in the FP32
    accumulator, per 128-colour block for 720 flows), so the result must equal
    the exact integer quadratic form bit for bit."""
    sqrts = CASES[ng][0]
    p = _mixed(ng, sqrts)
    chat, _ = p.color_matrix()
    nc = chat.shape[0]
    amp = 4 if nc <= 128 else 1
    rng = np.random.default_rng(40 + ng)
    v = rng.integers(-amp, amp + 1, size=(256, nc)).astype(np.int64)
    exact = np.einsum("ri,ij,rj->r", v, chat, v).reshape(32, 8).sum(axis=1)
    q8 = torch.empty(32, dtype=torch.float64, device="cuda")
    rc = binding.lib().mg_debug_colour_sum_rows(
        p.handle, torch.from_numpy(v.astype(np.float64)).cuda().data_ptr(), 256,
        q8.data_ptr(), None)
    assert rc == binding.MG_OK
    got = q8.cpu().numpy()
    assert np.array_equal(got, exact.astype(np.float64)), np.abs(got - exact).max()
