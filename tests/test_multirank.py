"""The multi-GPU path of bench.py on CPU: two gloo ranks (no GPU).

Events are independent, so ranks evaluate disjoint event sets with no
data-path collective (weak scaling); the only collective is the MAX of the
ranks' timings.  Checked here: disjoint, reproducible per-rank inputs and the
timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
from paper_2510_05392_gb300 import phasespace as ps


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mom = ps.generate(64, 2, 1500.0, 20251007, ptmin=20.0, drmin=0.4,
                      first_candidate=bench.shard_first_candidate(rank))
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slow one
    dist.barrier()
    q.put((rank, mom, t))
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps_ = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps_:
        p.start()
    out = dict((r, (m, t)) for r, m, t in (q.get(timeout=120) for _ in range(2)))
    for p in ps_:
        p.join(timeout=60)
        assert p.exitcode == 0
    m0, t0 = out[0]
    m1, t1 = out[1]
    assert t0 == t1 == 2.0
    # rank 0 holds the standard workload; rank 1 different (disjoint) events
    np.testing.assert_array_equal(m0, ps.generate(64, 2, 1500.0, 20251007, ptmin=20.0, drmin=0.4))
    assert not np.isclose(m0[:, 2:], m1[:, 2:]).all(axis=(1, 2)).any()


def test_single_process_timing_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5


def test_bench_gpus_flag_launches_the_ranks():
    """`bench.py --gpus 2` outside a launcher starts two ranks itself
    (torch.distributed.run, rendezvous on 127.0.0.1); --plan-only makes each
    rank report its shard over gloo and stop before any GPU work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--plan-only"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["n_gpus"] == 2
    ranks = sorted(d["plan"])
    assert [x[0] for x in ranks] == [0, 1]
    assert [x[1] for x in ranks] == [bench.shard_first_candidate(0), bench.shard_first_candidate(1)]
    assert ranks[0][2] != ranks[1][2]       # different events on the two ranks
