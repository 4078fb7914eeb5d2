"""GPU: the kernel-timing hook of the C ABI (CUDA events recorded by the
library around each of its launches on the caller's stream)."""
import numpy as np
import pytest

from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [binding.MG_FP64, binding.MG_MIXED_BF16])
def test_kernel_times_count_every_launch(precision):
    mom = torch.from_numpy(ps.generate(300, 2, 1500.0, 7100, ptmin=20.0, drmin=0.4)).cuda()
    p = binding.Process("g g > t t~ g g", precision=precision)
    p.filter_helicities(mom[:16])
    out = torch.empty(300, dtype=torch.float64, device="cuda")
    p.set_kernel_timing(64)
    n0 = binding.launch_count()
    for _ in range(3):
        p.sigmakin(mom, out)
    launched = binding.launch_count() - n0
    kt = p.kernel_times(reset=True)
    assert launched == sum(n for _, n in kt.values())
    ms, n = kt["diagram"]
    assert n == 3 and ms > 0.0
    if precision == binding.MG_MIXED_BF16:
        assert kt["colour"][1] == 3 and kt["colour"][0] > 0.0
        assert kt["event_sum"][1] == 3
    else:
        assert kt["colour"][1] == 0 and kt["event_sum"][1] == 0
    # after a reset nothing is reported; timing off records nothing
    assert p.kernel_times()["diagram"][1] == 0
    p.set_kernel_timing(0)
    p.sigmakin(mom, out)
    assert p.kernel_times()["diagram"][1] == 0
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()


def test_kernel_times_overflow_is_reported():
    mom = torch.from_numpy(ps.generate(64, 1, 1500.0, 7101, ptmin=20.0, drmin=0.4)).cuda()
    p = binding.Process("g g > t t~ g")
    p.filter_helicities(mom[:16])
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    p.set_kernel_timing(2)
    for _ in range(3):
        p.sigmakin(mom, out)
    with pytest.raises(binding.MGError):
        p.kernel_times()
    p.set_kernel_timing(0)
