"""GPU: every benchmark workload at its full size, in the benchmark's launch
configuration (default threads per event and block, whole workload in one
call), FP64 and mixed precision, checked against the oracle on a strided
sample of events (the first and last event included)."""
import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = {"fp64": 1e-9, "mixed": 1e-6}
CASES = [  # workload, precision, number of sampled events
    ("ggtt_16384", "fp64", 16384),
    ("ggtt_16384", "mixed", 16384),
    ("ggttgg_524288", "mixed", 256),
    ("ggttggg_262144", "fp64", 64),
    ("ggttggg_262144", "mixed", 64),
    ("ggttgggg_16384", "fp64", 16),
    ("ggttgggg_16384", "mixed", 16),
    ("ggttggggg_512", "fp64", 2),
    ("ggttggggg_512", "mixed", 2),
]


@pytest.mark.parametrize("name,precision,nsample", CASES)
def test_full_size_sampled(name, precision, nsample):
    w = ps.WORKLOADS[name]
    ng, sqrts = w["ngluon_final"], w["sqrts"]
    mom = ps.workload(name)
    proc = "g g > t t~" + " g" * ng
    prec = binding.MG_MIXED_BF16 if precision == "mixed" else binding.MG_FP64
    p = binding.Process(proc, precision=prec)
    kw = dict(ptmin=20.0, drmin=0.4) if w["cuts"] else {}
    p.filter_helicities(torch.from_numpy(ps.generate(16, ng, sqrts, 12345, **kw)).cuda())
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    p.sigmakin(torch.from_numpy(mom).cuda(), out)
    assert p.device_status() == binding.MG_OK
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.unique(np.concatenate([np.linspace(0, len(mom) - 1, nsample).astype(np.int64),
                                    [len(mom) - 1]]))
    rel = np.abs(got[idx] / oracle.me(mom[idx]) - 1)
    assert rel.max() <= RTOL[precision], (name, precision, rel.max())


BATCH_BLOCKS = [(0, 1048576), (1, 262144), (2, 65536), (3, 16384)]   # the benchmark's uneven batch


def test_uneven_batch_full_size_sampled():
    """The benchmark's uneven four-process batch at full size, autotuned as
    the benchmark does, in one persistent launch; 24 sampled events per
    process against the oracle."""
    blocks, host = [], []
    for ng, n in BATCH_BLOCKS:
        kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
        p = binding.Process("g g > t t~" + " g" * ng)
        p.filter_helicities(torch.from_numpy(ps.generate(16, ng, 1500.0, 12345, **kw)).cuda())
        m = ps.generate(n, ng, 1500.0, 20251005 + 4, **kw)
        host.append(m)
        blocks.append((p, torch.from_numpy(m).cuda(),
                       torch.full((n,), -1.0, dtype=torch.float64, device="cuda")))
    b = binding.Batch(blocks)
    b.autotune(reps=1)
    b.run()
    torch.cuda.synchronize()
    for (p, _, o), m in zip(blocks, host):
        got = o.cpu().numpy()
        assert np.all(np.isfinite(got)) and np.all(got > 0)
        idx = np.unique(np.linspace(0, len(m) - 1, 24).astype(np.int64))
        assert np.abs(got[idx] / oracle.me(m[idx]) - 1).max() <= RTOL["fp64"]


@pytest.mark.parametrize("name", ["ggttgg_524288", "ggttggg_262144"])
def test_mixed_against_fp64_every_event(name):
    """The mixed-precision colour sum against the FP64 path (itself checked
    against the oracle above) on every event of the full workload: the
    per-process error bound of the mixed path is stated over the whole set,
    not a sample."""
    w = ps.WORKLOADS[name]
    ng, sqrts = w["ngluon_final"], w["sqrts"]
    md = torch.from_numpy(ps.workload(name)).cuda()
    test = torch.from_numpy(ps.generate(16, ng, sqrts, 12345, ptmin=20.0, drmin=0.4)).cuda()
    outs = []
    for prec in (binding.MG_FP64, binding.MG_MIXED_BF16):
        p = binding.Process("g g > t t~" + " g" * ng, precision=prec)
        p.filter_helicities(test)
        out = torch.empty(md.shape[0], dtype=torch.float64, device="cuda")
        p.sigmakin(md, out)
        assert p.device_status() == binding.MG_OK
        outs.append(out)
    rel = (outs[1] / outs[0] - 1).abs()
    print(f"{name}: mixed vs FP64 over {md.shape[0]} events: max {rel.max().item():.3e}, "
          f"median {rel.median().item():.3e}")
    assert rel.max().item() <= RTOL["mixed"]
