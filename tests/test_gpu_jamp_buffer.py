"""The diagram kernel's two ways of forming the jamps give the same bits.

By default the jamp updates are FP64 reductions performed at L2 into a
per-thread buffer in global memory (zeroing stores, reductions and the final
read-back are relaxed operations of one thread, which stay in program order);
the test hook mg_debug_jamp_buffer(p, 0) switches to updates in place in local
memory.  Both add the same terms to every jamp in the same order, so every
output (|M|^2, per-helicity values, mixed-precision colour sums, channel and
flow weights) must agree bit for bit.  Parity of the default path with the
oracle is tested in test_gpu_parity.py and test_gpu_extras.py.
"""
import numpy as np
import pytest

from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {  # ngluon_final: (sqrt(s), events: several blocks and a ragged tail)
    1: (1500.0, 2048 + 13),
    2: (1500.0, 1024 + 7),
    3: (1500.0, 256 + 3),
}


def _events(ng, n, seed, sqrts):
    return ps.generate(n, ng, sqrts, seed, ptmin=20.0, drmin=0.4)


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _process(ng, sqrts, **kw):
    p = binding.Process("g g > t t~" + " g" * ng, **kw)
    p.filter_helicities(_gpu(_events(ng, 16, 12345, sqrts)))
    return p


def _both(p, run, first=(1, 0), second=(0, 0)):
    """run() under two settings (enable, max_bytes) of the jamp-buffer hook
    (default: buffer, then in-place updates); numpy copies of the outputs."""
    L = binding.lib()
    assert L.mg_debug_jamp_buffer(p.handle, *first) == binding.MG_OK
    a = [x.cpu().numpy().copy() for x in run()]
    assert L.mg_debug_jamp_buffer(p.handle, *second) == binding.MG_OK
    b = [x.cpu().numpy().copy() for x in run()]
    assert L.mg_debug_jamp_buffer(p.handle, 1, 0) == binding.MG_OK
    return a, b


@pytest.mark.parametrize("ng", sorted(CASES))
def test_fp64_me_and_per_helicity_bit_identical(ng):
    sqrts, n = CASES[ng]
    p = _process(ng, sqrts)
    mom = _gpu(_events(ng, n, 700 + ng, sqrts))
    nhel = 1 << (ng + 4)

    def run():
        me = torch.empty(n, dtype=torch.float64, device="cuda")
        mh = torch.empty(n * nhel, dtype=torch.float64, device="cuda")
        p.sigmakin(mom, me)
        me2 = torch.empty(n, dtype=torch.float64, device="cuda")
        p.sigmakin_hel(mom, me2, mh)
        torch.cuda.synchronize()
        return me, me2, mh

    a, b = _both(p, run)
    assert np.all(a[0] > 0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y), np.abs(x - y).max()


@pytest.mark.parametrize("ng", [2, 3])
def test_mixed_bit_identical(ng):
    sqrts, n = CASES[ng]
    p = _process(ng, sqrts, precision=binding.MG_MIXED_BF16)
    mom = _gpu(_events(ng, n, 710 + ng, sqrts))

    def run():
        me = torch.empty(n, dtype=torch.float64, device="cuda")
        p.sigmakin(mom, me)
        torch.cuda.synchronize()
        return (me,)

    a, b = _both(p, run)
    assert np.all(a[0] > 0)
    assert np.array_equal(a[0], b[0]), np.abs(a[0] - b[0]).max()


def test_extras_bit_identical():
    ng = 2
    sqrts, n = CASES[ng]
    p = _process(ng, sqrts)
    nc = p.info().ncolor
    mom = _gpu(_events(ng, n, 720, sqrts))
    chan = torch.from_numpy(np.arange(n, dtype=np.int32) % 15).cuda()

    def run():
        me = torch.empty(n, dtype=torch.float64, device="cuda")
        sde = torch.empty(n, dtype=torch.float64, device="cuda")
        flow = torch.empty(n * nc, dtype=torch.float64, device="cuda")
        p.sigmakin_ex(mom, out=me, sde=sde, flow=flow, channel_ids=chan)
        torch.cuda.synchronize()
        return me, sde, flow

    a, b = _both(p, run)
    for x, y in zip(a, b):
        assert np.array_equal(x, y), np.abs(x - y).max()


def test_large_calls_split_into_launches_bit_identical():
    """An FP64 call whose jamp buffer exceeds the limit runs as several
    launches over consecutive event ranges (here a 1 MB limit: 42 events of
    g g > t t~ g g per launch, 25 launches); |M|^2, the per-helicity values and the extras
    (alpha_s, channel weights, flow weights) of every event equal those of
    one launch over all events."""
    ng = 2
    sqrts, n = CASES[ng]
    p = _process(ng, sqrts)
    nc = p.info().ncolor
    nhel = 1 << (ng + 4)
    mom = _gpu(_events(ng, n, 730, sqrts))
    chan = torch.from_numpy(np.arange(n, dtype=np.int32) % 15).cuda()
    alphas = torch.from_numpy(0.118 * (1.0 + 0.1 * np.sin(np.arange(n)))).cuda()

    def run():
        me = torch.empty(n, dtype=torch.float64, device="cuda")
        me2 = torch.empty(n, dtype=torch.float64, device="cuda")
        mh = torch.empty(n * nhel, dtype=torch.float64, device="cuda")
        me3 = torch.empty(n, dtype=torch.float64, device="cuda")
        sde = torch.empty(n, dtype=torch.float64, device="cuda")
        flow = torch.empty(n * nc, dtype=torch.float64, device="cuda")
        p.sigmakin(mom, me)
        p.sigmakin_hel(mom, me2, mh)
        p.sigmakin_ex(mom, out=me3, alphas=alphas, sde=sde, flow=flow, channel_ids=chan)
        torch.cuda.synchronize()
        return me, me2, mh, me3, sde, flow

    a, b = _both(p, run, first=(1, 0), second=(1, 1 << 20))
    L = binding.lib()
    assert L.mg_debug_jamp_buffer(p.handle, 1, 1 << 20) == binding.MG_OK
    p.set_kernel_timing(64)
    p.sigmakin(mom, torch.empty(n, dtype=torch.float64, device="cuda"))
    launches = p.kernel_times(reset=True)["diagram"][1]
    p.set_kernel_timing(0)
    assert L.mg_debug_jamp_buffer(p.handle, 1, 0) == binding.MG_OK
    assert launches == 25, launches
    assert np.all(a[0] > 0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y), np.abs(x - y).max()


def test_hook_rejects_bad_arguments():
    L = binding.lib()
    assert L.mg_debug_jamp_buffer(None, 0, 0) == binding.MG_ERR_BAD_ARG
    p = binding.Process("g g > t t~")
    assert L.mg_debug_jamp_buffer(p.handle, 1, -1) == binding.MG_ERR_BAD_ARG
