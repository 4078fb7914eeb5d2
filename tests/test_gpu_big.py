"""GPU: g g -> t t~ + 5 g (2 -> 7, 5040 colour flows), run with its state in
HBM from the process compiler's table file, against the CPU oracle
(Berends-Giele colour-ordered amplitudes and the exact colour matrix).

The table file is generated on first use (a few minutes); the oracle takes a
few seconds per event on the host cores."""
import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROC = "g g > t t~ g g g g g"
RTOL = 1e-9


def _events(n, seed):
    return ps.generate(n, 5, 2000.0, seed, ptmin=20.0, drmin=0.4)


@pytest.fixture(scope="module")
def big():
    return binding.Process(PROC, hel_mode=binding.MG_HEL_ALL)


@pytest.fixture(scope="module")
def events():
    mom = _events(3, 424242)
    return mom, oracle.me(mom, per_helicity=True)


def test_info(big):
    i = big.info()
    assert (i.npar, i.ngluon, i.ncolor, i.nhel, i.ngood) == (9, 7, 5040, 512, 512)


def test_me_and_per_helicity_match_oracle(big, events):
    mom, (ref, ref_h) = events
    md = torch.from_numpy(mom).cuda()
    out = torch.empty(len(mom), dtype=torch.float64, device="cuda")
    out_h = torch.empty((len(mom), 512), dtype=torch.float64, device="cuda")
    big.sigmakin(md, out)
    single = out.clone()
    big.sigmakin_hel(md, out, out_h)
    torch.cuda.synchronize()
    got, got_h = out.cpu().numpy(), out_h.cpu().numpy()
    assert np.abs(got / ref - 1).max() <= RTOL
    assert np.array_equal(single.cpu().numpy(), got)       # deterministic
    scale = ref_h.max(axis=1, keepdims=True)
    assert np.abs(got_h - ref_h).max() <= RTOL * scale.min()
    np.testing.assert_allclose(got_h.sum(axis=1), got, rtol=1e-13)


def test_chunks_and_ragged_sizes(big, events):
    """One event, then the three events again: same values whatever the
    batch (the items of a launch are independent)."""
    mom, (ref, _) = events
    md = torch.from_numpy(mom).cuda()
    one = torch.empty(1, dtype=torch.float64, device="cuda")
    big.sigmakin(md[1:2], one)
    torch.cuda.synchronize()
    assert abs(one.item() / ref[1] - 1) <= RTOL


def test_filter_keeps_every_helicity(events):
    mom, (_, ref_h) = events
    p = binding.Process(PROC)
    n = p.filter_helicities(torch.from_numpy(mom[:2]).cuda())
    expect = oracle.good_helicity_mask(mom[:2])
    assert n == int(expect.sum())
    assert np.array_equal(p.helicity_mask().astype(bool), expect.astype(bool))


def test_colour_matrix_matches_oracle(big):
    got, d = big.color_matrix()
    ref, D, _ = oracle.color_data(7)
    assert d == D
    assert np.array_equal(got, ref)


# the stated bound of the mixed-precision colour sum (BF16 pieces, FP32
# accumulation): relative 1e-6 per event
MIXED_RTOL = 1e-6


def test_mixed_colour_sum_on_tensor_cores(events):
    """Colour sum of the 5040 flows on the tensor cores (BF16 pieces, FP32
    accumulation per 128-colour block, blocks added in FP64) against the
    oracle; per-helicity values against the FP64 path."""
    mom, (ref, ref_h) = events
    p = binding.Process(PROC, hel_mode=binding.MG_HEL_ALL, precision=binding.MG_MIXED_BF16)
    md = torch.from_numpy(mom).cuda()
    out = torch.empty(len(mom), dtype=torch.float64, device="cuda")
    out_h = torch.empty((len(mom), 512), dtype=torch.float64, device="cuda")
    p.sigmakin_hel(md, out, out_h)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    rel = np.abs(out.cpu().numpy() / ref - 1)
    print(f"2->7 mixed: max rel {rel.max():.3e}")
    assert rel.max() <= MIXED_RTOL
    got_h = out_h.cpu().numpy()
    scale = ref_h.max(axis=1, keepdims=True)            # per event
    assert (np.abs(got_h - ref_h) <= MIXED_RTOL * scale).all()


def test_unsupported_paths(big):
    mom = torch.from_numpy(_events(1, 5)).cuda()
    with pytest.raises(binding.MGError):       # the fixed-scratch filter holds 256 helicities
        binding.lib()
        n = binding.ctypes.c_int(0)
        binding._check(binding.lib().mg_filter_helicities_noalloc(
            big.handle, binding._ptr(mom), 1, None, binding.ctypes.byref(n)), "noalloc")


def test_extras_flow_weights_alphas_sde_and_choices(big, events):
    """Per-event extras of the 2 -> 7 process: flow weights against the
    oracle's Berends-Giele colour-ordered amplitudes (sum_h |J_s,h|^2 =
    sum_h |A_s,h|^2 for every one of the 5040 flows), alpha_s rescaling,
    channel weights, and the helicity and colour choices."""
    mom, (ref, _) = events
    n = len(mom)
    md = torch.from_numpy(mom).cuda()
    nc = 5040
    flow = torch.empty((n, nc), dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    a = np.array([0.10, 0.118, 0.13])[:n]
    sde = torch.empty(n, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(11)
    rh, rc = rng.uniform(size=n), rng.uniform(size=n)
    hel = torch.empty(n, dtype=torch.int32, device="cuda")
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    big.sigmakin_ex(md, out, alphas=torch.from_numpy(a).cuda(), channel=17, sde=sde, flow=flow,
                    rnd_hel=torch.from_numpy(rh).cuda(), hel_out=hel,
                    rnd_col=torch.from_numpy(rc).cuda(), col_out=col)
    outh = torch.empty((n, 512), dtype=torch.float64, device="cuda")
    big.sigmakin_hel(md, torch.empty(n, dtype=torch.float64, device="cuda"), outh)
    torch.cuda.synchronize()
    got, fw, mh = out.cpu().numpy(), flow.cpu().numpy(), outh.cpu().numpy()
    assert np.abs(got / (ref * (a / 0.118) ** 7) - 1).max() <= RTOL
    w = sde.cpu().numpy()
    assert np.all(w >= 0) and np.all(w <= 1)
    assert big.info().nchannel == 135135               # (2 * 7 - 1)!! trivalent diagrams
    ids = torch.tensor([17, 135134, 135135][:n], dtype=torch.int32, device="cuda")
    w2 = torch.empty(n, dtype=torch.float64, device="cuda")
    big.sigmakin_ex(md, None, channel_ids=ids, sde=w2)
    torch.cuda.synchronize()
    w2 = w2.cpu().numpy()
    assert w2[0] == w[0] and (n < 3 or w2[2] == 0.0) and (n < 2 or 0.0 <= w2[1] <= 1.0)
    ref_flow = sum(np.abs(oracle.amplitudes(mom[0], h)) ** 2 for h in range(512))
    assert np.abs(fw[0] - ref_flow).max() <= RTOL * ref_flow.max()

    def pick(wts, r):
        c = np.cumsum(wts)
        return int(np.searchsorted(c, r * c[-1], side="right"))

    got_h, got_c = hel.cpu().numpy(), col.cpu().numpy()
    for e in range(n):
        assert got_c[e] == pick(fw[e], rc[e])
        cum = np.cumsum(mh[e]) / mh[e].sum()
        if np.min(np.abs(cum - rh[e])) > 1e-12:
            assert got_h[e] == pick(mh[e], rh[e])


def test_two_chunks_with_extras():
    """640 events: more than one chunk of jamp rows (622 events fit 24 GiB),
    so the second chunk's offsets into momenta, outputs and per-event inputs
    are used; events on both sides of the boundary against the oracle."""
    mom = _events(640, 777)
    idx = [0, 621, 622, 639]
    ref = oracle.me(mom[idx])
    p = binding.Process(PROC, hel_mode=binding.MG_HEL_ALL, precision=binding.MG_MIXED_BF16)
    a = np.full(640, 0.118)
    a[idx] = [0.11, 0.12, 0.125, 0.13]
    out = torch.empty(640, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(torch.from_numpy(mom).cuda(), out, alphas=torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    assert p.device_status() == 0
    got = out.cpu().numpy()[idx]
    assert np.abs(got / (ref * (a[idx] / 0.118) ** 7) - 1).max() <= MIXED_RTOL
