"""GPU: the MLP surrogate's own forward/backward kernels against the CPU
oracle, its training, checkpointing, and the exact two-stage unweighting."""
import ctypes
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [32, 256, 256, 256, 1]


def _lib():
    L = binding.lib()
    vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    sig = {
        "mg_sur_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                           ctypes.POINTER(vp)], ctypes.c_int),
        "mg_sur_destroy": ([vp], None),
        "mg_sur_param_count": ([vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "mg_sur_get_params": ([vp, fp], ctypes.c_int),
        "mg_sur_set_params": ([vp, fp], ctypes.c_int),
        "mg_sur_get_grads": ([vp, fp], ctypes.c_int),
        "mg_sur_loss_grad": ([vp, vp, ctypes.c_int, vp, ctypes.c_int, dp, vp], ctypes.c_int),
        "mg_sur_fit_target": ([vp, vp, ctypes.c_int64, vp], ctypes.c_int),
        "mg_sur_adam": ([vp, ctypes.c_double, vp], ctypes.c_int),
        "mg_sur_get_target_stats": ([vp, dp], ctypes.c_int),
        "mg_sur_train": ([vp, vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                          ctypes.c_double, vp, dp], ctypes.c_int),
        "mg_sur_predict": ([vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp], ctypes.c_int),
        "mg_sur_save": ([vp, ctypes.c_char_p], ctypes.c_int),
        "mg_sur_load": ([vp, ctypes.c_char_p], ctypes.c_int),
        "mg_unweight2": ([vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                          vp, vp, ctypes.POINTER(ctypes.c_int64), vp], ctypes.c_int),
    }
    for k, (a, r) in sig.items():
        getattr(L, k).argtypes = a
        getattr(L, k).restype = r
    return L


def _new(L, bmax=4096, seed=3):
    h = ctypes.c_void_p()
    assert L.mg_sur_create(32, 256, 3, seed, bmax, ctypes.byref(h)) == 0
    return h


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _flat_to_params(flat):
    out, off = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = flat[off:off + a * b].reshape(b, a).astype(np.float64)
        off += a * b
        out.append([W, flat[off:off + b].astype(np.float64)])
        off += b
    return out


def _bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


@pytest.mark.parametrize("m", [512, 400])
def test_gradients_match_cpu_oracle(m):
    """Gradients of every layer against the CPU oracle (FP64 with the GPU's
    BF16 rounding points); m = 400 is padded to 512 rows inside the library
    (zero features, zero loss gradient), which must not change them."""
    L = _lib()
    h = _new(L)
    n = ctypes.c_int64()
    L.mg_sur_param_count(h, ctypes.byref(n))
    flat = np.zeros(n.value, dtype=np.float32)
    L.mg_sur_get_params(h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    mom = ps.generate(m, 2, 1500.0, 77, ptmin=20.0, drmin=0.4)
    y = np.random.default_rng(0).normal(size=m).astype(np.float32)
    loss = ctypes.c_double()
    md, yd = torch.from_numpy(mom).cuda(), torch.from_numpy(y).cuda()
    assert L.mg_sur_loss_grad(h, ctypes.c_void_p(md.data_ptr()), 6, ctypes.c_void_p(yd.data_ptr()), m,
                              ctypes.byref(loss), _stream()) == 0
    g = np.zeros_like(flat)
    L.mg_sur_get_grads(h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    # oracle on the same (BF16-rounded) weights and features, FP64 arithmetic,
    # rounding to BF16 where the BF16 training stores values
    params = _flat_to_params(flat)
    for p in params:
        p[0] = S.round_bf16(p[0])
    x = S.round_bf16(S.features(mom))
    lo, go = S.loss_and_grads(params, x, y.astype(np.float64), emulate_bf16=True)
    _, gx = S.loss_and_grads(params, x, y.astype(np.float64))
    assert abs(loss.value / lo - 1) < 1e-5
    gg = _flat_to_params(g)
    errs, errs_exact = {}, {}
    for l in range(4):
        for k in range(2):
            nrm = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            errs[(l, k)] = nrm(gg[l][k], go[l][k])
            errs_exact[(l, k)] = nrm(gg[l][k], gx[l][k])
    print("gradient errors vs BF16-emulating oracle:", errs)
    print("gradient errors vs exact FP64 oracle:", errs_exact)
    L.mg_sur_destroy(h)
    # residuals: values rounded to the other BF16 neighbour when FP32 and FP64
    # accumulation straddle a rounding boundary; bias sums cancel the most
    assert max(errs[(l, 0)] for l in range(4)) < 2e-3, errs
    assert max(errs[(l, 1)] for l in range(4)) < 5e-3, errs
    assert max(errs_exact[(l, 0)] for l in range(4)) < 3e-2


def test_forward_layers_on_tensor_cores():
    """Each layer's tensor-core GEMM against the same contraction in FP64 of
    the BF16 values it read (activations from the debug export, BF16-rounded
    weights): Z_l = A_l W_l^T + b_l to FP32 accumulation accuracy, and
    A_l+1 = silu(Z_l) rounded to BF16 (one BF16 step allowed for the fast
    exponential).  Pins the operand layouts, swizzle, descriptors, column
    tiles and the epilogue's row/column mapping."""
    L = _lib()
    L.mg_sur_debug_buffer.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_float)]
    h = _new(L, seed=11)
    n = ctypes.c_int64()
    L.mg_sur_param_count(h, ctypes.byref(n))
    flat = np.zeros(n.value, dtype=np.float32)
    L.mg_sur_get_params(h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    params = _flat_to_params(flat)
    m = 384
    mom = ps.generate(m, 2, 1500.0, 78, ptmin=20.0, drmin=0.4)
    y = np.zeros(m, dtype=np.float32)
    md, yd = torch.from_numpy(mom).cuda(), torch.from_numpy(y).cuda()
    assert L.mg_sur_loss_grad(h, ctypes.c_void_p(md.data_ptr()), 6, ctypes.c_void_p(yd.data_ptr()), m,
                              None, _stream()) == 0
    torch.cuda.synchronize()
    widths = [32, 256, 256, 256]
    outp = [256, 256, 256, 16]

    def buf(which, layer, cols):
        a = np.zeros(m * cols, dtype=np.float32)
        assert L.mg_sur_debug_buffer(h, which, layer, m, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))) == 0
        return a.reshape(m, cols).astype(np.float64)

    for l in range(4):
        A = buf(0, l, widths[l])
        Z = buf(1, l, outp[l])[:, :SIZES[l + 1]]
        W = S.round_bf16(params[l][0])
        ref = A @ W.T + params[l][1]
        scale = np.abs(A) @ np.abs(W).T + np.abs(params[l][1])
        assert (np.abs(Z - ref) <= 1e-5 * scale + 1e-30).all(), l
        if l < 3:
            An = buf(0, l + 1, widths[l + 1])
            sil = Z / (1 + np.exp(-Z))
            assert (np.abs(An - _bf16(sil)) <= 2 ** -7 * np.abs(sil) + 1e-30).all(), l
    L.mg_sur_destroy(h)


def _train_set(ng, n, seed, sqrts=1500.0):
    mom = ps.generate(n, ng, sqrts, seed, ptmin=20.0, drmin=0.4)
    p = binding.Process("g g > t t~" + " g" * ng)
    p.filter_helicities(torch.from_numpy(ps.generate(16, ng, sqrts, 12345, ptmin=20.0, drmin=0.4)).cuda())
    md = torch.from_numpy(mom).cuda()
    me = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin(md, me)
    return p, mom, md, me


def test_training_learns_log_me_and_checkpoint_roundtrip():
    L = _lib()
    p, mom, md, me = _train_set(2, 32768, 91)
    h = _new(L)
    s = _stream()
    assert L.mg_sur_fit_target(h, ctypes.c_void_p(me.data_ptr()), 32768, s) == 0
    first = ctypes.c_double()
    assert L.mg_sur_train(h, ctypes.c_void_p(md.data_ptr()), 6, ctypes.c_void_p(me.data_ptr()), 32768,
                          1, 4096, 1e-3, s, ctypes.byref(first)) == 0
    last = ctypes.c_double()
    assert L.mg_sur_train(h, ctypes.c_void_p(md.data_ptr()), 6, ctypes.c_void_p(me.data_ptr()), 32768,
                          30, 4096, 1e-3, s, ctypes.byref(last)) == 0
    assert last.value < 0.5 * first.value and last.value < 0.5   # standardised: 1 = no skill
    # held-out events: prediction explains most of the variance of log|M|^2
    _, mt, mtd, met = _train_set(2, 4096, 92)
    pred = torch.empty(4096, dtype=torch.float64, device="cuda")
    assert L.mg_sur_predict(h, ctypes.c_void_p(mtd.data_ptr()), 6, 4096, ctypes.c_void_p(pred.data_ptr()), s) == 0
    torch.cuda.synchronize()
    lt = torch.log(met)
    r2 = 1 - ((pred - lt) ** 2).mean() / lt.var()
    assert r2.item() > 0.5
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "sur.bin").encode()
        assert L.mg_sur_save(h, f) == 0
        h2 = _new(L, seed=99)
        assert L.mg_sur_load(h2, f) == 0
        pred2 = torch.empty_like(pred)
        L.mg_sur_predict(h2, ctypes.c_void_p(mtd.data_ptr()), 6, 4096, ctypes.c_void_p(pred2.data_ptr()), s)
        torch.cuda.synchronize()
        assert torch.equal(pred, pred2)
        L.mg_sur_destroy(h2)
    L.mg_sur_destroy(h)


def test_two_stage_unweighting_exact_and_gain():
    """Accept decisions match the oracle's rule on the same uniforms, and the
    trained surrogate needs far fewer exact matrix elements per unweighted
    event than plain hit-or-miss unweighting (exact matrix element on every
    candidate)."""
    L = _lib()
    ng = 1
    p, mom, md, me = _train_set(ng, 16384, 93)
    h = _new(L)
    s = _stream()
    L.mg_sur_fit_target(h, ctypes.c_void_p(me.data_ptr()), 16384, s)
    L.mg_sur_train(h, ctypes.c_void_p(md.data_ptr()), 5, ctypes.c_void_p(me.data_ptr()), 16384, 40, 4096,
                   1e-3, s, None)
    n = 65536
    cand, phi, _ = ps.generate(n, ng, 1500.0, 94, ptmin=20.0, drmin=0.4, return_weights=True)
    rng = np.random.default_rng(5)
    u1, u2 = rng.uniform(size=n), rng.uniform(size=n)
    cd = torch.from_numpy(cand).cuda()
    pd, u1d, u2d = (torch.from_numpy(a).cuda() for a in (phi, u1, u2))
    # calibration: maxima from the training slice (quantiles against outliers)
    pred_tr = torch.empty(16384, dtype=torch.float64, device="cuda")
    L.mg_sur_predict(h, ctypes.c_void_p(md.data_ptr()), 5, 16384, ctypes.c_void_p(pred_tr.data_ptr()), s)
    _, phi_tr, _ = ps.generate(16384, ng, 1500.0, 93, ptmin=20.0, drmin=0.4, return_weights=True)
    what_tr = np.exp(pred_tr.cpu().numpy()) * phi_tr
    w_tr = me.cpu().numpy() * phi_tr
    what_max = float(np.quantile(what_tr, 0.999))
    r_max = float(np.quantile(w_tr / what_tr, 0.999))
    acc = torch.zeros(n, dtype=torch.uint8, device="cuda")
    wt = torch.zeros(n, dtype=torch.float64, device="cuda")
    nex = ctypes.c_int64()
    assert L.mg_unweight2(p.handle, h, ctypes.c_void_p(cd.data_ptr()), ctypes.c_void_p(pd.data_ptr()),
                          ctypes.c_void_p(u1d.data_ptr()), ctypes.c_void_p(u2d.data_ptr()), n, what_max,
                          r_max, ctypes.c_void_p(acc.data_ptr()), ctypes.c_void_p(wt.data_ptr()),
                          ctypes.byref(nex), s) == 0
    acc_g, wt_g = acc.cpu().numpy().astype(bool), wt.cpu().numpy()
    # oracle rule with the oracle's exact |M|^2 and the GPU surrogate's w_hat
    pred = torch.empty(n, dtype=torch.float64, device="cuda")
    L.mg_sur_predict(h, ctypes.c_void_p(cd.data_ptr()), 5, n, ctypes.c_void_p(pred.data_ptr()), s)
    what = np.exp(pred.cpu().numpy()) * phi
    s1 = u1 < what / what_max
    w = np.zeros(n)
    w[s1] = oracle.me(cand[s1]) * phi[s1]
    acc_o, wt_o, s1_o = S.unweight_two_stage(w, what, u1, u2, what_max, r_max)
    assert nex.value == int(s1_o.sum())
    near = np.abs((w / what) / r_max - u2) < 1e-8
    assert np.array_equal(acc_g[~near], acc_o[~near])
    np.testing.assert_allclose(wt_g[acc_g & acc_o], wt_o[acc_g & acc_o], rtol=1e-9)
    # gain, like for like: plain hit-or-miss unweighting of the same
    # candidates (exact matrix element for every one) with the same rule as
    # the two-stage path -- the maximum is the 0.999 quantile of the
    # calibration slice and larger weights stay as overweights -- and both
    # paths measured by the Kish effective sample size of their weighted
    # output per exact matrix element evaluated
    me_all = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin(cd, me_all)
    torch.cuda.synchronize()
    w_all = me_all.cpu().numpy() * phi
    w_q = float(np.quantile(w_tr, 0.999))
    u3 = np.random.default_rng(6).uniform(size=n)
    keep = u3 < w_all / w_q
    wt_plain = np.maximum(1.0, w_all[keep] / w_q)

    def ess(x):
        return x.sum() ** 2 / (x ** 2).sum()

    plain = ess(wt_plain) / n
    two = ess(wt_g[acc_g]) / nex.value
    print(f"effective unweighted events per exact ME: plain {plain:.4f}, two-stage {two:.4f}, "
          f"gain {two / plain:.2f} (accepted {keep.sum()} / {acc_g.sum()})")
    assert two > 2 * plain


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    """The tensor-core GEMMs' mbarrier waits are bounded: with the test hook
    making the operand barrier expect more bytes than its TMA copies deliver,
    every GEMM gives up after about a second, records the timeout and returns;
    mg_sur_device_status reports it once, and the next prediction on the same
    context is bit-identical to one made before the stall."""
    L = _lib()
    L.mg_sur_debug_inject_stall.argtypes = [ctypes.c_void_p, ctypes.c_uint]
    L.mg_sur_device_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    h = _new(L, bmax=256)
    s = _stream()
    md = torch.from_numpy(ps.generate(128, 2, 1500.0, 81, ptmin=20.0, drmin=0.4)).cuda()
    ref = torch.empty(128, dtype=torch.float64, device="cuda")
    assert L.mg_sur_predict(h, ctypes.c_void_p(md.data_ptr()), 6, 128, ctypes.c_void_p(ref.data_ptr()), s) == 0
    assert L.mg_sur_device_status(h, s) == binding.MG_OK
    assert L.mg_sur_debug_inject_stall(h, 16) == 0
    out = torch.empty_like(ref)
    assert L.mg_sur_predict(h, ctypes.c_void_p(md.data_ptr()), 6, 128, ctypes.c_void_p(out.data_ptr()), s) == 0
    assert L.mg_sur_device_status(h, s) == binding.MG_ERR_DEVICE_TIMEOUT
    assert L.mg_sur_device_status(h, s) == binding.MG_OK        # reported once
    assert L.mg_sur_debug_inject_stall(h, 0) == 0
    assert L.mg_sur_predict(h, ctypes.c_void_p(md.data_ptr()), 6, 128, ctypes.c_void_p(out.data_ptr()), s) == 0
    assert L.mg_sur_device_status(h, s) == binding.MG_OK
    assert torch.equal(out, ref)
    L.mg_sur_destroy(h)


def test_graph_replayed_training_matches_plain_steps():
    """mg_sur_train replays one captured training step as a CUDA graph (device-
    side batch index and Adam step count); the same batches run as explicit
    mg_sur_loss_grad + mg_sur_adam calls on an identical network give the
    same parameters and last-epoch loss (the bias corrections are computed on
    the device in one path and on the host in the other, hence a tolerance)."""
    L = _lib()
    p, mom, md, me = _train_set(1, 8192, 95)
    s = _stream()
    ha, hb = _new(L, seed=21), _new(L, seed=21)
    for h in (ha, hb):
        assert L.mg_sur_fit_target(h, ctypes.c_void_p(me.data_ptr()), 8192, s) == 0
    la = ctypes.c_double()
    assert L.mg_sur_train(ha, ctypes.c_void_p(md.data_ptr()), 5, ctypes.c_void_p(me.data_ptr()), 8192, 3,
                          4096, 1e-3, s, ctypes.byref(la)) == 0
    ms = (ctypes.c_double * 2)()
    L.mg_sur_get_target_stats(hb, ms)
    y = ((torch.log(me) - ms[0]) / ms[1]).float()
    lb = []
    for ep in range(3):
        for b in range(2):
            l = ctypes.c_double()
            assert L.mg_sur_loss_grad(hb, ctypes.c_void_p(md[4096 * b:].data_ptr()), 5,
                                      ctypes.c_void_p(y[4096 * b:].data_ptr()), 4096, ctypes.byref(l), s) == 0
            assert L.mg_sur_adam(hb, 1e-3, s) == 0
            if ep == 2:
                lb.append(l.value)
    torch.cuda.synchronize()
    n = ctypes.c_int64()
    L.mg_sur_param_count(ha, ctypes.byref(n))
    pa, pb = np.zeros(n.value, np.float32), np.zeros(n.value, np.float32)
    L.mg_sur_get_params(ha, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    L.mg_sur_get_params(hb, pb.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    print(f"graph vs plain steps: max |dp| {np.abs(pa - pb).max():.2e}, loss {la.value:.6f} / {np.mean(lb):.6f}")
    assert np.abs(pa - pb).max() <= 1e-4 * np.abs(pb).max()
    assert abs(la.value / np.mean(lb) - 1) < 1e-4
    L.mg_sur_destroy(ha)
    L.mg_sur_destroy(hb)
