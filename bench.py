"""Throughput benchmark: g g -> t t~ g g matrix elements on GB300.

Workload (default): 524288 synthetic events of g g -> t t~ g g at sqrt(s) =
1500 GeV with gluon cuts (pT > 20 GeV, Delta R > 0.4), FP64 path, inputs
resident in HBM.  One step = one mg_sigmakin call over the whole batch
(momentum read, diagrams, colour sum, helicity sum).

Other workloads (--workload): ggtt_16384, ggttggg_262144, ggttgggg_16384,
ggttggggg_512 (2 -> 7, state in HBM), uneven_batch_4proc (one persistent
graph-replayed launch over four processes), ggttgggg_surrogate (exact ME,
MLP training, two-stage unweighting); --precision mixed puts the colour sum
on the tensor cores.

Prints one JSON line (rank 0).  Keys beyond the basic ones:
  e2e          the same metric through the public API with pinned host
               buffers: H2D of the step's momenta + mg_sigmakin + D2H of the
               matrix elements, every step
  roofline     the diagram kernel against the FP64 pipe ("alu"): algorithmic
               FP64 flops / the kernel's own CUDA-event time (recorded by the
               library around its launches) vs the FP64 FMA peak measured
               live by mg_probe_fp64_peak; traffic from the committed ncu
               summary when it matches the current kernel sources
  roofline_colour_tc   mixed precision: the tensor-core colour sum (HBM bound
               up to 128 flows, tensor bound above)
  roofline_colour_f64  the FP64 colour-sum kernel of the 2 -> 7 process
  gpu_launches the library's own kernel launches in the timed region
  cpu_baseline the CPU oracle on the host cores on a bounded sample, with its
               single-core rate, the CPU model and clock
  accuracy     the headline workload on strided events against the oracle
  sub_records  with the default workload: g g -> t t~ g g g (262144 events)
               in FP64 and in mixed precision, each with its own steps,
               rooflines, clocks and accuracy over 4096 strided events
               (max and median relative error), and their speed ratio
  clocks       nvidia-smi samples taken during the timed region
  me_log10_quantiles   quantiles of log10 |M|^2 of the workload

--impl reference times the CPU oracle (the only reference this workload
has) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ME events/s per process on 1 GB300: FP64 vs mixed vs surrogate; % of FP64 peak"
WORKLOADS = {
    # name: (process, ngluon_final, nevt, sqrt_s, cuts, seed)
    "ggttgg_524288": ("g g > t t~ g g", 2, 524288, 1500.0, True, 20251005 + 2),
    "ggtt_16384": ("g g > t t~", 0, 16384, 1000.0, False, 20251005 + 1),
    "ggttggg_262144": ("g g > t t~ g g g", 3, 262144, 1500.0, True, 20251005 + 3),
    "ggttgggg_16384": ("g g > t t~ g g g g", 4, 16384, 2000.0, True, 20251005 + 5),
    # 2 -> 7 (5040 flows): state in HBM, FP64 colour sum kernel of its own
    "ggttggggg_512": ("g g > t t~ g g g g g", 5, 512, 2000.0, True, 20251005 + 6),
}
# oracle events per CPU sample where one event takes seconds on the host
CPU_SAMPLE_CAP = {"ggttggggg_512": 4, "ggttgggg_16384": 256}
TEST_SEED = 12345  # helicity-filter test events


def shard_first_candidate(rank: int) -> int:
    """First generator candidate of a rank: ranks draw disjoint candidate
    ranges of the same seeded generator (rank 0 = the standard workload)."""
    return rank * (1 << 40)


def max_over_ranks(t: float, device=None) -> float:
    """Slowest rank's time (all ranks call it; identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return tt.item()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _events(name, nevt=None, first_candidate=0):
    from paper_2510_05392_gb300 import phasespace as ps
    proc, ng, n, sqrts, cuts, seed = WORKLOADS[name]
    kw = dict(ptmin=20.0, drmin=0.4) if cuts else {}
    return ps.generate(nevt or n, ng, sqrts, seed, first_candidate=first_candidate, **kw)


def _test_events(name):
    from paper_2510_05392_gb300 import phasespace as ps
    proc, ng, n, sqrts, cuts, seed = WORKLOADS[name]
    kw = dict(ptmin=20.0, drmin=0.4) if cuts else {}
    return ps.generate(16, ng, sqrts, TEST_SEED, **kw)


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


_FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def _fp64_peak():
    """FP64 FMA peak of this GPU in flops/s, measured live by the library's
    probe (16 independent FMA chains per thread), or None."""
    from paper_2510_05392_gb300 import binding
    L = binding.lib()
    L.mg_probe_fp64_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]
    peak = ctypes.c_double(0.0)
    return peak.value if L.mg_probe_fp64_peak(0, 20000, 5, ctypes.byref(peak)) == 0 else None


def _fp64_roofline(flops_per_step, seconds_per_step, kernel, peak):
    ach = flops_per_step / seconds_per_step
    return {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12 if peak else None,
            "unit": "TFLOP/s", "frac": ach / peak if peak else None, "traffic": None,
            "kernel": kernel + " (FP64 pipe; peak = FP64 FMA probe, measured live)",
            "flops_per_step": flops_per_step}


def _measured_peak(key):
    """Measured peak of this GPU pool (copy GB/s, cuBLAS bf16 TFLOP/s), else
    the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, ValueError, KeyError, TypeError):
        return _FALLBACK_PEAKS.get(key)


_KERNEL_SOURCES = {
    "k_sigmakin": ["mg_kernels.cu", "mg_kin.cuh", "mg_dirac.cuh", "mg_internal.h"],
    "k_colorsum_tc": ["mg_colorsum_tc.cu", "mg_tc.cuh", "mg_internal.h"],
}


def _kernel_hash(kernel="k_sigmakin"):
    h = hashlib.sha256()
    for f in _KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2510_05392_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload, events_per_launch=None):
    """DRAM bytes per launch from the committed ncu summary, when it was
    taken on the current kernel sources (else None); entries stored per event
    are scaled to events_per_launch."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = data.get(f"{kernel}:{workload}")
    if not e or e.get("kernel_hash") != _kernel_hash(kernel):
        return None
    if "dram_bytes_per_event" in e and events_per_launch:
        return e["dram_bytes_per_event"] * events_per_launch
    return e.get("dram_bytes_per_launch")


def cpu_baseline(name, nsample, steps=1, nthreads=0):
    """The oracle (as it stands) on the host cores over the first nsample
    events of the workload (nthreads 0: all cores); returns (events/s,
    threads, seconds)."""
    import oracle
    mom = _events(name, nsample)
    oracle.me(mom[:1])  # load/compile, warm
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.me(mom, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return steps * nsample / dt, (nthreads or oracle.threads()), dt


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    name = args.workload
    n = min(args.ref_sample, CPU_SAMPLE_CAP.get(name, args.ref_sample))
    import oracle
    mom = _events(name, n)
    oracle.me(mom[:min(8, n)])
    for _ in range(args.warmup):
        oracle.me(mom[: max(1, n // 8)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.me(mom)
    dt = time.perf_counter() - t0
    value = args.steps * n / dt
    proc = WORKLOADS[name][0]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "process": proc, "nevt_per_step": n,
                   "sample": f"first {n} events of {name}"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": oracle.threads(),
                         "kind": "oracle", "sample": f"first {n} events of {name} per step"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


BATCH_BLOCKS = [  # (process, ngluon_final, nevt): uneven blocks at sqrt(s) = 1500 GeV, cuts
    ("g g > t t~", 0, 1048576), ("g g > t t~ g", 1, 262144),
    ("g g > t t~ g g", 2, 65536), ("g g > t t~ g g g", 3, 16384)]


def run_batch(args):
    """Uneven multi-process batch in one persistent, graph-replayed launch
    (autotuned), against the same blocks launched process by process."""
    import torch
    from paper_2510_05392_gb300 import binding, build
    from paper_2510_05392_gb300 import phasespace as ps
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    blocks, total = [], 0
    for proc, ng, n in BATCH_BLOCKS:
        kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
        p = binding.Process(proc)
        p.filter_helicities(torch.from_numpy(ps.generate(16, ng, 1500.0, TEST_SEED, **kw)).to(dev))
        m = torch.from_numpy(ps.generate(n, ng, 1500.0, 20251005 + 4, **kw)).to(dev)
        blocks.append((p, m, torch.empty(n, dtype=torch.float64, device=dev)))
        total += n
    flops_step = 0.0
    for p, m, _ in blocks:
        i = p.info()
        flops_step += m.shape[0] * i.ngood * (i.flops_diagram + i.flops_colour)
    peak = _fp64_peak()
    b = binding.Batch(blocks)
    tuned_ms = b.autotune(reps=1)
    tpe, ctas = b.config()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        b.run(stream)
    torch.cuda.synchronize(dev)
    clocks = Clocks(dev.index) if not args.no_clocks else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.run(stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    t_batch = ev0.elapsed_time(ev1) / 1e3
    in_bytes = sum(m.numel() * m.element_size() for _, m, _ in blocks)
    # the same blocks, one launch per process
    ev0.record(stream)
    for _ in range(args.steps):
        for p, m, o in blocks:
            p.sigmakin(m, o, stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_seq = ev0.elapsed_time(ev1) / 1e3
    line = {
        "metric": METRIC, "value": total * args.steps / t_batch, "unit": "events/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Philox4x32-10 + massive RAMBO, gluon cuts)",
        "config": {"workload": "uneven_batch_4proc", "blocks": [[pr, n] for pr, _, n in BATCH_BLOCKS],
                   "launch": "one persistent kernel per step, CUDA-graph replay",
                   "autotuned": {"threads_per_event": tpe, "ctas_per_sm": ctas,
                                 "tuning_ms_per_step": tuned_ms},
                   "l2": f"not flushed: the steps' inputs ({in_bytes / 1e6:.0f} MB of momenta) exceed L2"},
        "per_process_launches_events_per_s": total * args.steps / t_seq,
        "roofline": _fp64_roofline(flops_step, t_batch / args.steps, "k_batch (whole step)", peak),
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def _sur_lib():
    from paper_2510_05392_gb300 import binding
    L = binding.lib()
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "mg_sur_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                          ctypes.POINTER(vp)],
        "mg_sur_fit_target": [vp, vp, ctypes.c_int64, vp],
        "mg_sur_train": [vp, vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                         ctypes.c_double, vp, dp],
        "mg_sur_predict": [vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp],
        "mg_unweight2": [vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                         vp, vp, ctypes.POINTER(ctypes.c_int64), vp],
        "mg_sur_destroy": [vp],
    }
    for k, a in sig.items():
        getattr(L, k).argtypes = a
    return L


def run_surrogate(args):
    """g g -> t t~ g g g g at sqrt(s) = 2000 GeV with cuts: exact FP64 matrix
    elements of the training events, MLP training on the GPU, two-stage
    unweighting of the candidates (exact FP64 matrix element only for the
    stage-1 survivors), against plain hit-or-miss unweighting run on a slice
    of the candidates (exact matrix element for every one); both measured by
    the Kish effective sample size of their output per second, over several
    seeds of the uniforms."""
    import numpy as np
    import torch
    from paper_2510_05392_gb300 import binding, build
    from paper_2510_05392_gb300 import phasespace as ps
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = _sur_lib()
    ntrain = args.nevt or 262144
    ncand = args.ncand
    sqrts, seed = 2000.0, 20251005 + 5
    kw = dict(ptmin=20.0, drmin=0.4)
    tr, phi_tr, _ = ps.generate(ntrain, 4, sqrts, seed, return_weights=True, **kw)
    ca, phi_ca, _ = ps.generate(ncand, 4, sqrts, seed + 1000, return_weights=True, **kw)
    p = binding.Process("g g > t t~ g g g g")
    p.filter_helicities(torch.from_numpy(ps.generate(16, 4, sqrts, TEST_SEED, **kw)).to(dev))
    p.set_launch(16, 128)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    trd = torch.from_numpy(tr).to(dev)
    me_tr = torch.empty(ntrain, dtype=torch.float64, device=dev)
    p.sigmakin(trd[:256], me_tr[:256], stream)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    p.sigmakin(trd, me_tr, stream)
    torch.cuda.synchronize(dev)
    t_exact = time.perf_counter() - t0
    rate_exact = ntrain / t_exact
    # surrogate training
    h = ctypes.c_void_p()
    assert L.mg_sur_create(32, 256, 3, 7, 4096, ctypes.byref(h)) == 0
    t0 = time.perf_counter()
    L.mg_sur_fit_target(h, ctypes.c_void_p(me_tr.data_ptr()), ntrain, sp)
    loss = ctypes.c_double()
    rc = L.mg_sur_train(h, ctypes.c_void_p(trd.data_ptr()), 8, ctypes.c_void_p(me_tr.data_ptr()), ntrain,
                        args.epochs, 4096, 1e-3, sp, ctypes.byref(loss))
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    assert rc == 0, rc
    # calibration on the training slice (timed with CUDA events: inference
    # throughput of the tensor-core MLP)
    pred_tr = torch.empty(ntrain, dtype=torch.float64, device=dev)
    ia, ib = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ia.record(stream)
    L.mg_sur_predict(h, ctypes.c_void_p(trd.data_ptr()), 8, ntrain, ctypes.c_void_p(pred_tr.data_ptr()), sp)
    ib.record(stream)
    torch.cuda.synchronize(dev)
    t_infer = ia.elapsed_time(ib) / 1e3
    # MLP work: tensor-core MMA flops as issued (K padded to 64-wide chunks,
    # widths to 16) per row: forward sum_l 2 Kpad_l Npad_l; a training row
    # adds the weight gradients (same) and the backward data GEMMs (l > 0)
    sizes = [(32, 256), (256, 256), (256, 256), (256, 16)]
    fwd_row = sum(2 * (-(-k // 64) * 64) * n for k, n in sizes)
    bwd_row = fwd_row + sum(2 * n * k for k, n in sizes[1:])
    train_flops = (ntrain // 4096) * 4096 * args.epochs * (fwd_row + bwd_row)
    bf16 = _measured_peak("bf16_tflops")
    mlp_roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": bf16,
                "kernel": "k_mlp_gemm (tcgen05; peak = measured cuBLAS bf16 burst)",
                "train_achieved": train_flops / t_train / 1e12,
                "train_frac": train_flops / t_train / 1e12 / bf16 if bf16 else None,
                "train_step_ms": 1e3 * t_train / ((ntrain // 4096) * args.epochs),
                "infer_achieved": ntrain * fwd_row / t_infer / 1e12,
                "infer_frac": ntrain * fwd_row / t_infer / 1e12 / bf16 if bf16 else None,
                "infer_events_per_s": ntrain / t_infer,
                "note": "4096-row batches of a 32-256-256-256-1 network: one CUDA-graph launch "
                        "of about 30 kernels per training step, latency bound"}
    w_tr = me_tr.cpu().numpy() * phi_tr
    what_tr = np.exp(pred_tr.cpu().numpy()) * phi_tr
    what_max = float(np.quantile(what_tr, 0.999))
    r_max = float(np.quantile(w_tr / what_tr, 0.999))
    lt = np.log(me_tr.cpu().numpy())
    r2 = 1 - np.mean((pred_tr.cpu().numpy() - lt) ** 2) / np.var(lt)
    cad = torch.from_numpy(ca).to(dev)
    phd = torch.from_numpy(phi_ca).to(dev)

    def ess(x):
        return float(x.sum() ** 2 / max((x ** 2).sum(), 1e-300))

    # plain hit-or-miss unweighting, run: exact FP64 matrix element for every
    # candidate of a slice, then accept with u < w / w_max; same convention
    # as the two-stage rule (w_max = 0.999 quantile of the calibration slice,
    # larger weights kept as overweights); output measured by its Kish
    # effective sample size per second
    npl = min(args.plain_cand, ncand)
    me_pl = torch.empty(npl, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    p.sigmakin(cad[:npl], me_pl, stream)
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    w_pl = me_pl.cpu().numpy() * phi_ca[:npl]
    w_q = float(np.quantile(w_tr, 0.999))
    plain_runs = []
    for k in range(args.seeds):
        u = np.random.default_rng(seed + 100 + k).uniform(size=npl)
        keep = u < w_pl / w_q
        wk = np.maximum(1.0, w_pl[keep] / w_q)
        plain_runs.append({"accepted": int(keep.sum()), "ess": ess(wk), "ess_per_s": ess(wk) / t_plain})
    # two-stage unweighting of all candidates, one run per uniform seed
    acc = torch.zeros(ncand, dtype=torch.uint8, device=dev)
    wt = torch.zeros(ncand, dtype=torch.float64, device=dev)
    nex = ctypes.c_int64()
    two_runs = []
    launches_two = 0
    clocks = Clocks(dev.index) if not args.no_clocks else None   # over the two-stage runs
    for k in range(args.seeds):
        rng = np.random.default_rng(seed + 200 + k)
        u1d, u2d = (torch.from_numpy(rng.uniform(size=ncand)).to(dev) for _ in range(2))
        torch.cuda.synchronize(dev)
        launches0 = binding.launch_count()
        t0 = time.perf_counter()
        rc = L.mg_unweight2(p.handle, h, ctypes.c_void_p(cad.data_ptr()), ctypes.c_void_p(phd.data_ptr()),
                            ctypes.c_void_p(u1d.data_ptr()), ctypes.c_void_p(u2d.data_ptr()), ncand,
                            what_max, r_max, ctypes.c_void_p(acc.data_ptr()),
                            ctypes.c_void_p(wt.data_ptr()), ctypes.byref(nex), sp)
        torch.cuda.synchronize(dev)
        t_two = time.perf_counter() - t0
        assert rc == 0, rc
        launches_two = binding.launch_count() - launches0
        wts = wt.cpu().numpy()
        a_ = acc.cpu().numpy() != 0
        two_runs.append({"seconds": t_two, "exact_evaluations": int(nex.value), "accepted": int(a_.sum()),
                         "ess": ess(wts[a_]), "ess_per_s": ess(wts[a_]) / t_two})

    clk = clocks.stop() if clocks else None

    def mean_err(xs):
        m = float(np.mean(xs))
        return m, (float(np.std(xs, ddof=1) / np.sqrt(len(xs))) if len(xs) > 1 else None)

    pl_m, pl_e = mean_err([r["ess_per_s"] for r in plain_runs])
    tw_m, tw_e = mean_err([r["ess_per_s"] for r in two_runs])
    gain = tw_m / pl_m
    gain_err = (gain * math.hypot(tw_e / tw_m, pl_e / pl_m)) if (tw_e is not None and pl_e is not None) else None
    t_two_mean = float(np.mean([r["seconds"] for r in two_runs]))
    line = {
        "metric": METRIC, "value": ncand / t_two_mean, "unit": "events/s", "n_gpus": 1,
        "steps": args.seeds, "warmup": 1, "ms_per_step": 1e3 * t_two_mean, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (exact ME) + bf16 (surrogate)", "data": "synthetic (Philox4x32-10 + massive RAMBO, gluon cuts)",
        "config": {"workload": "ggttgggg_surrogate", "process": "g g > t t~ g g g g", "sqrt_s_gev": sqrts,
                   "train_events": ntrain, "candidates": ncand, "plain_candidates": npl,
                   "epochs": args.epochs, "batch": 4096, "uniform_seeds": args.seeds,
                   "mlp": "32(28 log s_ij/s)-256-256-256-1 SiLU, BF16 weights/activations, FP32 master + Adam"},
        "exact_fp64": {"events_per_s": rate_exact, "seconds": t_exact,
                       "fp64_tflops": rate_exact * p.info().ngood * (p.info().flops_diagram + p.info().flops_colour) / 1e12},
        "roofline": _fp64_roofline(
            ntrain * p.info().ngood * (p.info().flops_diagram + p.info().flops_colour), t_exact,
            "k_sigmakin on the training events (wall time of the exact-ME pass)", _fp64_peak()),
        "training": {"seconds": t_train, "final_epoch_loss": loss.value, "r2_log_me_train": float(r2)},
        "roofline_mlp": mlp_roof,
        "two_stage": {"what_max": what_max, "r_max": r_max, "runs": two_runs,
                      "ess_per_s": tw_m, "ess_per_s_err": tw_e},
        "plain_hit_or_miss": {"w_max_quantile": w_q, "exact_seconds": t_plain, "runs": plain_runs,
                              "ess_per_s": pl_m, "ess_per_s_err": pl_e},
        "surrogate_gain_ess_per_s": gain, "surrogate_gain_err": gain_err,
        "gpu_launches": launches_two,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    L.mg_sur_destroy(h)


def _timed_steps(p, mom, out, stream, dev, steps, warmup, ws, flush, clocks_on):
    """Warm-up, then `steps` timed mg_sigmakin calls (L2 flushed before each,
    untimed; CUDA events on the launching stream) with the library's
    per-kernel timing; returns (device seconds per rank, max over ranks,
    wall seconds, per-kind kernel times, library launches, clocks)."""
    from paper_2510_05392_gb300 import binding
    import torch
    for _ in range(warmup):
        p.sigmakin(mom, out, stream)
    torch.cuda.synchronize(dev)
    clocks = Clocks(dev.index) if clocks_on else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    p.set_kernel_timing(steps * 3 * 256)
    p.kernel_times(reset=True)
    launches0 = binding.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(steps):
        flush.fill_(i & 0xFF)  # L2 flush between timed launches (not timed)
        ev[i][0].record(stream)
        p.sigmakin(mom, out, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    launches = binding.launch_count() - launches0
    kt = p.kernel_times(reset=True)
    p.set_kernel_timing(0)
    t_dev = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)
    # kernels launched in the timed region, counted by the library; the timed
    # regions (one per kind and chunk) cover one kernel each, or two for the
    # colour sum of a table-file process in mixed precision (BF16 pieces, then
    # the tensor cores)
    assert launches >= sum(n for _, n in kt.values()), (kt, launches)
    return t_dev, wall, kt, launches, clk


def _rooflines(name, precision, nevt, ngood, info, steps, kt, fp64_peak):
    """Roofline records of one measurement: the diagram kernel against the
    FP64 pipe, and the colour-sum kernel (tensor cores or FP64) when it runs
    in a kernel of its own."""
    colour_ms, colour_n = kt["colour"]
    separate_colour = colour_n > 0       # the colour sum runs in a kernel of its own
    # algorithmic FP64 work of the diagram kernel per step (mixed: the colour
    # sum runs on the tensor cores, so only the diagram work is FP64), over
    # the diagram kernel's own device time
    fp64_colour = info.flops_colour if (precision == "fp64" and not separate_colour) else 0.0
    flops_step = nevt * ngood * (info.flops_diagram + fp64_colour)
    diag_ms, diag_n = kt["diagram"]
    per_step = diag_n // steps
    achieved = flops_step * steps / (diag_ms / 1e3)
    roof = {"bound": "alu", "achieved": achieved / 1e12,
            "peak": fp64_peak / 1e12 if fp64_peak else None, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak if fp64_peak else None,
            "traffic": _traffic("k_sigmakin", name, nevt / per_step)
            if per_step == 1 or precision == "fp64" else None,
            "kernel": ("k_sigmakin_big" if separate_colour and precision == "fp64"
                       else "k_sigmakin") + " (FP64 pipe; peak = FP64 FMA probe, measured live)",
            "flops_per_event_and_helicity": info.flops_diagram + fp64_colour,
            "flops_per_launch": flops_step / per_step, "launches_per_step": per_step,
            "ms_per_step": diag_ms / steps}
    roof_tc = roof_colour = None
    if precision == "fp64" and separate_colour:
        # FP64 colour-sum kernel (table-file processes): algorithmic FP64
        # flops of the triangular quadratic form over its own device time
        c_flops = nevt * ngood * info.flops_colour
        c_ach = c_flops * steps / (colour_ms / 1e3)
        roof_colour = {"bound": "alu", "achieved": c_ach / 1e12,
                       "peak": fp64_peak / 1e12 if fp64_peak else None, "unit": "TFLOP/s",
                       "frac": c_ach / fp64_peak if fp64_peak else None, "traffic": None,
                       "kernel": "k_colour_big (FP64 pipe; peak = FP64 FMA probe, measured live)",
                       "launches_per_step": colour_n // steps,
                       "ms_per_step": colour_ms / steps, "flops_per_step": c_flops}
    if precision == "mixed":
        tc_ms, tc_n = kt["colour"]
        if info.ncolor > 128:
            # 5040 / 720 flows: a GEMM over the block upper triangle, tensor
            # bound.  MMA flops as issued: rows x (128-colour blocks J >= I)
            # x 128^2 x 2 flops x 5 BF16 piece products
            kb = -(-info.ncolor // 128)
            rows = nevt * ngood * 2
            mma_flops = rows * (kb * (kb + 1) // 2) * 128 * 128 * 2 * 5
            tc_ach = mma_flops * steps / (tc_ms / 1e3) / 1e12
            bf16 = _measured_peak("bf16_tflops")
            roof_tc = {"bound": "tensor", "achieved": tc_ach, "peak": bf16, "unit": "TFLOP/s",
                       "frac": tc_ach / bf16 if bf16 else None, "traffic": None,
                       "kernel": "k_colorsum_tc_big (with its BF16 row conversion; peak = "
                                 "measured cuBLAS bf16 burst)",
                       "launches_per_step": tc_n // steps,
                       "ms_per_step": tc_ms / steps, "flops_per_step": mma_flops}
        else:
            # bound by reading the BF16 jamp pieces once: 2 (re, im) x 3
            # pieces x ncolor x 2 bytes per event and good helicity
            bytes_step = nevt * ngood * 2 * 3 * info.ncolor * 2
            tc_ach = bytes_step * steps / (tc_ms / 1e3) / 1e9
            hbm = _measured_peak("hbm_gbs")
            roof_tc = {"bound": "hbm", "achieved": tc_ach, "peak": hbm, "unit": "GB/s",
                       "frac": tc_ach / hbm if hbm else None,
                       "traffic": _traffic("k_colorsum_tc", name, nevt * steps / tc_n),
                       "kernel": "k_colorsum_tc (peak = measured copy bandwidth)",
                       "launches_per_step": tc_n // steps,
                       "ms_per_step": tc_ms / steps, "bytes_per_step": bytes_step}
    return roof, roof_tc, roof_colour


def _accuracy(got, ref, idx, what):
    import numpy as np
    rel = np.abs(got[idx] / ref - 1)
    return {"events_checked": int(len(idx)), "max_rel_err": float(rel.max()),
            "median_rel_err": float(np.median(rel)), "against": what}


def _setup_process(name, precision, nevt, rank, dev):
    import torch
    from paper_2510_05392_gb300 import binding
    proc = WORKLOADS[name][0]
    mom_h = _events(name, nevt, first_candidate=shard_first_candidate(rank))
    mom = torch.from_numpy(mom_h).to(dev)
    out = torch.empty(nevt, dtype=torch.float64, device=dev)
    prec = binding.MG_MIXED_BF16 if precision == "mixed" else binding.MG_FP64
    p = binding.Process(proc, precision=prec)
    ngood = p.filter_helicities(torch.from_numpy(_test_events(name)).to(dev))
    return p, mom_h, mom, out, ngood


SUB_WORKLOAD = "ggttggg_262144"


def _sub_records(args, ws, rank, dev, stream, flush, fp64_peak):
    """g g -> t t~ g g g (262144 events per GPU) in FP64 and in mixed
    precision, each with its own steps, rooflines and clocks, and both
    checked on the same strided events against the oracle."""
    import numpy as np
    nevt = WORKLOADS[SUB_WORKLOAD][2]
    recs, outs, mom_h = {}, {}, None
    for prec in ("fp64", "mixed"):
        p, mom_h, mom, out, ngood = _setup_process(SUB_WORKLOAD, prec, nevt, rank, dev)
        info = p.info()
        t_dev, wall, kt, launches, clk = _timed_steps(
            p, mom, out, stream, dev, args.sub_steps, args.sub_warmup, ws, flush,
            rank == 0 and not args.no_clocks)
        roof, roof_tc, _ = _rooflines(SUB_WORKLOAD, prec, nevt, ngood, info, args.sub_steps, kt,
                                      fp64_peak)
        recs[prec] = {"workload": SUB_WORKLOAD, "precision": prec, "steps": args.sub_steps,
                      "warmup": args.sub_warmup, "value": ws * nevt * args.sub_steps / t_dev,
                      "unit": "events/s", "ms_per_step": 1e3 * t_dev / args.sub_steps,
                      "roofline": roof, "roofline_colour_tc": roof_tc, "gpu_launches": launches,
                      "clocks": clk, "wall_s_timed": wall}
        outs[prec] = out.cpu().numpy() if rank == 0 else None
        del p, mom, out
    res = {"ggttggg_262144_fp64": recs["fp64"], "ggttggg_262144_mixed": recs["mixed"],
           "mixed_over_fp64": recs["mixed"]["value"] / recs["fp64"]["value"]}
    if rank == 0:
        # the mixed path against the FP64 path (checked against the oracle)
        # on every event of the set: the per-process bound over the whole set
        rel = np.abs(outs["mixed"] / outs["fp64"] - 1)
        res["mixed_vs_fp64_all_events"] = {"events": int(len(rel)), "max_rel_err": float(rel.max()),
                                           "median_rel_err": float(np.median(rel))}
    if rank == 0 and args.sub_check > 0:
        import oracle
        idx = np.unique(np.linspace(0, nevt - 1, args.sub_check).astype(np.int64))
        ref = oracle.me(mom_h[idx])
        for prec in ("fp64", "mixed"):
            recs[prec]["accuracy"] = _accuracy(outs[prec], ref, idx,
                                               "CPU oracle (FP64), strided events")
    return res


def _cpu_info():
    """Host CPU model and maximum clock (lscpu, else the cpufreq files), for
    the CPU-baseline record."""
    fields = {}
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            k, _, v = line.partition(":")
            fields.setdefault(k.strip(), v.strip())
    except (OSError, subprocess.SubprocessError):
        pass
    model = " ".join(x for x in (fields.get("Vendor ID"), fields.get("Model name")) if x) or None
    mhz = None
    for k in ("CPU max MHz", "CPU MHz"):
        try:
            mhz = float(fields[k])
            break
        except (KeyError, ValueError):
            pass
    for path in ("/sys/devices/system/cpu/cpu0/cpufreq/cpuinfo_max_freq",
                 "/sys/devices/system/cpu/cpufreq/policy0/cpuinfo_max_freq",
                 "/sys/devices/system/cpu/cpu0/cpufreq/scaling_max_freq"):
        if mhz is not None:
            break
        try:
            with open(path) as fh:
                mhz = int(fh.read().strip()) / 1000.0
        except (OSError, ValueError):
            pass
    return model, mhz


def run_ours(args):
    import torch
    from paper_2510_05392_gb300 import build

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    name = args.workload
    proc, ng, n_default, sqrts, cuts, seed = WORKLOADS[name]
    nevt = args.nevt or n_default
    npar = ng + 4
    # each rank evaluates its own nevt events (weak scaling; rank 0 holds the
    # standard workload, rank r the next candidates of the same generator)
    p, mom_h, mom, out, ngood = _setup_process(name, args.precision, nevt, rank, dev)
    if args.tpe or args.block:
        p.set_launch(args.tpe, args.block)
    info = p.info()
    stream = torch.cuda.current_stream(dev)

    # FP64 peak measured live on this GPU (roofline denominator)
    fp64_peak = _fp64_peak()

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    t_dev, wall, kt, n_launches, clk = _timed_steps(
        p, mom, out, stream, dev, args.steps, args.warmup, ws, flush,
        rank == 0 and not args.no_clocks)
    value = ws * nevt * args.steps / t_dev
    ms_step = 1e3 * t_dev / args.steps
    roof, roof_tc, roof_colour = _rooflines(name, args.precision, nevt, ngood, info, args.steps,
                                            kt, fp64_peak)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(mom_h).pin_memory()
        host_out = torch.empty(nevt, dtype=torch.float64).pin_memory()
        for _ in range(1):
            mom.copy_(host_in, non_blocking=True)
            p.sigmakin(mom, out, stream)
            host_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            mom.copy_(host_in, non_blocking=True)
            p.sigmakin(mom, out, stream)
            host_out.copy_(out, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        te = max_over_ranks(a.elapsed_time(b) / 1e3, dev)
        e2e = {"value": ws * nevt * args.steps / te, "unit": "events/s",
               "h2d_bytes_per_step": nevt * npar * 4 * 8, "d2h_bytes_per_step": nevt * 8}
        assert torch.isfinite(host_out).all().item()

    # value distribution of |M|^2 (heavy tailed): quantiles of log10, untimed
    me_q = None
    accuracy = None
    if rank == 0:
        import numpy as np
        got = out.cpu().numpy()
        lg = np.log10(np.clip(got, 1e-300, None))
        me_q = {f"q{q:g}": float(np.quantile(lg, q / 100)) for q in (1, 10, 50, 90, 99)}
        if args.check > 0:
            import oracle
            idx = np.unique(np.linspace(0, nevt - 1, min(args.check, nevt)).astype(np.int64))
            accuracy = _accuracy(got, oracle.me(mom_h[idx]), idx, "CPU oracle (FP64), strided events")
    del p, mom, out

    sub = None
    if args.sub and name == "ggttgg_524288" and not args.nevt:
        sub = _sub_records(args, ws, rank, dev, stream, flush, fp64_peak)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ns = min(args.cpu_sample, CPU_SAMPLE_CAP.get(name, args.cpu_sample))
        v, cores, dt = cpu_baseline(name, ns)
        n1 = max(1, ns // 16)
        v1, _, dt1 = cpu_baseline(name, n1, nthreads=1)
        model, mhz = _cpu_info()
        cpu = {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"first {ns} events of {name}, {dt:.1f} s",
               "value_1core": v1, "sample_1core": f"first {n1} events of {name}, {dt1:.1f} s",
               "cpu_model": model, "cpu_max_mhz": mhz, "nproc": os.cpu_count()}
        if mhz is None:
            cpu["cpu_clock_note"] = "not exposed on this host (lscpu lists no MHz, no cpufreq files)"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+bf16x3",
            "data": "synthetic (Philox4x32-10 + massive RAMBO, gluon cuts)",
            "config": {"workload": name, "process": proc, "nevt_per_gpu": nevt,
                       "sqrt_s_gev": sqrts, "cuts": "pT>20 GeV, dR>0.4 (final gluons)" if cuts else "none",
                       "precision": args.precision, "ngood_helicities": ngood,
                       "l2": "flushed between timed launches (256 MiB write, untimed)",
                       "parallelism": f"dp{ws} (independent events per GPU)"},
            "roofline": roof,
            "roofline_colour_tc": roof_tc,
            "roofline_colour_f64": roof_colour,
            "e2e": e2e,
            "gpu_launches": n_launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "me_log10_quantiles": me_q,
            "wall_s_timed": wall,
            "sub_records": sub,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def plan_only(args):
    """Rank layout of a multi-rank run without touching a GPU: every rank
    reports its rank, the first generator candidate of its shard and a digest
    of its first events; rank 0 prints them as one JSON line."""
    import numpy as np
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("gloo")
    first = shard_first_candidate(rank)
    ev = _events(args.workload, 16, first_candidate=first)
    mine = torch.tensor([rank, first, int(hashlib.sha256(np.ascontiguousarray(ev).tobytes())
                                          .hexdigest()[:12], 16)], dtype=torch.int64)
    rows = [mine.clone() for _ in range(ws)]
    if ws > 1:
        dist.all_gather(rows, mine)
    if rank == 0:
        print(json.dumps({"plan": [[int(x) for x in r] for r in rows], "n_gpus": ws,
                          "workload": args.workload}), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def relaunch(args) -> int:
    """--gpus N > 1 outside a torch.distributed launcher: start N ranks of
    this script (one per GPU, rendezvous on 127.0.0.1) and return their exit
    status."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1", f"--master-port={port}",
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ggttgg_524288",
                    choices=sorted(WORKLOADS) + ["uneven_batch_4proc", "ggttgggg_surrogate"])
    ap.add_argument("--ncand", type=int, default=1048576, help="surrogate: candidates")
    ap.add_argument("--epochs", type=int, default=20, help="surrogate: training epochs")
    ap.add_argument("--plain-cand", type=int, default=32768,
                    help="surrogate: candidates of the plain hit-or-miss arm")
    ap.add_argument("--seeds", type=int, default=4, help="surrogate: uniform seeds per arm")
    ap.add_argument("--nevt", type=int, default=0, help="override events per GPU (profiling)")
    ap.add_argument("--tpe", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--cpu-sample", type=int, default=16384)
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--check", type=int, default=256, help="events checked against the oracle")
    ap.add_argument("--sub-steps", type=int, default=2, help="steps of the 2 -> 5 sub-records")
    ap.add_argument("--sub-warmup", type=int, default=3, help="warm-up of the 2 -> 5 sub-records")
    ap.add_argument("--sub-check", type=int, default=4096,
                    help="2 -> 5 events checked against the oracle (both precisions)")
    ap.add_argument("--no-sub", dest="sub", action="store_false",
                    help="no g g > t t~ g g g sub-records with the default workload")
    ap.add_argument("--plan-only", action="store_true",
                    help="print the rank layout (ranks, shards) and exit before any GPU work")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch(args))
    if args.warmup < 3 and args.impl == "ours" and not args.nevt:
        args.warmup = 3
    if args.plan_only:
        plan_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven_batch_4proc":
        run_batch(args)
    elif args.workload == "ggttgggg_surrogate":
        run_surrogate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
