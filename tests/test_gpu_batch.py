"""GPU: uneven multi-process batch in one persistent launch (graph replay,
autotuner), checked against the single-process path and the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = {0: 4099, 1: 1030, 2: 260, 3: 33}   # ragged, uneven blocks


def _events(ng, n, seed):
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    return ps.generate(n, ng, 1500.0, seed, **kw)


def _blocks(sizes=SIZES):
    blocks, host = [], {}
    for ng, n in sizes.items():
        p = binding.Process("g g > t t~" + " g" * ng)
        p.filter_helicities(torch.from_numpy(_events(ng, 16, 12345)).cuda())
        m = _events(ng, n, 4000 + ng)
        host[ng] = m
        blocks.append((p, torch.from_numpy(m).cuda(),
                       torch.full((n,), -1.0, dtype=torch.float64, device="cuda")))
    return blocks, host


def test_batch_matches_single_process_path_and_oracle():
    blocks, host = _blocks()
    b = binding.Batch(blocks)
    b.run()
    torch.cuda.synchronize()
    for (p, m, o), ng in zip(blocks, SIZES):
        single = torch.empty_like(o)
        p.sigmakin(m, single)
        torch.cuda.synchronize()
        assert (o / single - 1).abs().max().item() < 1e-13
        idx = np.unique(np.linspace(0, len(host[ng]) - 1, 24).astype(int))
        ref = oracle.me(host[ng][idx])
        assert np.abs(o.cpu().numpy()[idx] / ref - 1).max() <= 1e-9


def test_graph_replay_and_autotune_keep_results():
    blocks, _ = _blocks()
    b = binding.Batch(blocks)
    b.run()
    torch.cuda.synchronize()
    first = [o.clone() for _, _, o in blocks]
    for _, _, o in blocks:
        o.fill_(-1.0)
    b.run()          # graph replay
    b.run()
    torch.cuda.synchronize()
    for a, (_, _, o) in zip(first, blocks):
        assert torch.equal(a, o)
    ms = b.autotune(reps=1)
    assert ms > 0
    tpe, ctas = b.config()
    assert all(t in (1, 2, 4, 8, 16) for t in tpe) and ctas >= 1
    for _, _, o in blocks:
        o.fill_(-1.0)
    b.run()
    torch.cuda.synchronize()
    for a, (_, _, o) in zip(first, blocks):
        assert (o / a - 1).abs().max().item() < 1e-13


def test_one_shot_batch_and_errors():
    blocks, _ = _blocks({1: 100, 2: 0, 3: 5})
    L = binding.lib()
    n = len(blocks)
    procs = (ctypes.c_void_p * n)(*[p.handle for p, _, _ in blocks])
    moms = (ctypes.c_void_p * n)(*[m.data_ptr() for _, m, _ in blocks])
    outs = (ctypes.c_void_p * n)(*[o.data_ptr() for _, _, o in blocks])
    nev = (ctypes.c_int64 * n)(*[m.shape[0] for _, m, _ in blocks])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mg_sigmakin_batch(n, procs, moms, nev, outs, stream) == binding.MG_OK
    torch.cuda.synchronize()
    for p, m, o in blocks:
        if m.shape[0]:
            single = torch.empty_like(o)
            p.sigmakin(m, single)
            torch.cuda.synchronize()
            assert (o / single - 1).abs().max().item() < 1e-13
    unfiltered = binding.Process("g g > t t~ g")
    big = binding.Process("g g > t t~ g g g g", hel_mode=binding.MG_HEL_ALL)
    for proc, status in ((unfiltered, binding.MG_ERR_NOT_FILTERED), (big, binding.MG_ERR_UNSUPPORTED)):
        m = blocks[0][1]
        with pytest.raises(binding.MGError) as e:
            binding.Batch([(proc, m, blocks[0][2])])
        assert e.value.status == status
