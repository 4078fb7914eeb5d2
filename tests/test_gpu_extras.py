"""GPU: per-event extras of sigmaKin -- running alpha_s, flow weights
(jamp-level parity with the oracle), single-diagram-enhancement weights,
helicity and colour choice."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_05392_gb300 import binding
from paper_2510_05392_gb300 import phasespace as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(ng, n, seed, sqrts=1500.0):
    kw = dict(ptmin=20.0, drmin=0.4) if ng else {}
    mom = ps.generate(n, ng, sqrts, seed, **kw)
    p = binding.Process("g g > t t~" + " g" * ng)
    p.filter_helicities(torch.from_numpy(ps.generate(16, ng, sqrts, 12345, **kw)).cuda())
    return p, mom, torch.from_numpy(mom).cuda()


def test_per_event_alphas():
    p, mom, md = _setup(1, 24, 5100)
    a = np.random.default_rng(1).uniform(0.10, 0.13, 24)
    out = torch.empty(24, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(md, out, alphas=torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.array([oracle.me(mom[i:i + 1], alphas=a[i])[0] for i in range(24)])
    assert np.abs(got / ref - 1).max() <= 1e-9


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_flow_weights_match_oracle_colour_ordered_amplitudes(ng):
    """sum_h |J_s,h|^2 equals sum_h |A_s,h|^2 of the oracle's Berends-Giele
    colour-ordered amplitudes for every flow s (jamps and colour-ordered
    amplitudes agree up to a phase per helicity)."""
    n = 5
    p, mom, md = _setup(ng, n, 5200 + ng)
    nc = math.factorial(ng + 2)
    flow = torch.empty((n, nc), dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(md, out, flow=flow)
    single = torch.empty_like(out)
    p.sigmakin(md, single)
    torch.cuda.synchronize()
    assert torch.allclose(out, single, rtol=1e-13, atol=0)
    got = flow.cpu().numpy()
    nhel = 1 << (ng + 4)
    for e in range(n):
        ref = sum(np.abs(oracle.amplitudes(mom[e], h)) ** 2 for h in range(nhel))
        assert np.abs(got[e] - ref).max() <= 1e-9 * ref.max()


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_sde_channels_match_oracle(ng):
    """The library's channels are the oracle's trivalent diagrams, colour
    code for colour code and in the same order (3 / 15 / 105 channels)."""
    from oracle import sde
    p = binding.Process("g g > t t~" + " g" * ng)
    codes = p.sde_channels()
    assert p.info().nchannel == len(codes) == [3, 15, 105][ng]
    assert np.array_equal(codes, sde.channels(ng + 2)[1])


@pytest.mark.parametrize("ng", [0, 1, 2])
def test_sde_weights_match_oracle_every_channel(ng):
    """Single-diagram-enhancement weight of every channel for every event,
    element by element against the oracle's diagram-by-diagram evaluation
    (textbook Feynman rules, colour from Gell-Mann matrices), through
    per-event channel ids: every (event, channel) pair in one call."""
    from oracle import sde
    n = 4
    p, mom, _ = _setup(ng, n, 5300 + ng)
    ref = sde.sde_weights(mom)                       # [n][nchannel]
    nch = ref.shape[1]
    rep = torch.from_numpy(np.repeat(mom, nch, axis=0)).cuda()
    ids = torch.from_numpy(np.tile(np.arange(nch, dtype=np.int32), n)).cuda()
    w = torch.empty(n * nch, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(rep, None, channel_ids=ids, sde=w)
    # the whole-call channel gives the same numbers as the per-event ids
    one = torch.empty(n, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(torch.from_numpy(mom).cuda(), None, channel=nch - 1, sde=one)
    torch.cuda.synchronize()
    got = w.cpu().numpy().reshape(n, nch)
    err = np.abs(got - ref)
    print(f"ng={ng}: max |dw| {err.max():.2e}, max rel {(err / np.maximum(ref, 1e-300)).max():.2e}")
    assert (err <= 1e-9 * ref + 1e-15).all()
    assert np.array_equal(one.cpu().numpy(), got[:, nch - 1])
    np.testing.assert_allclose(got.sum(axis=1), 1.0, rtol=1e-12)


def test_sde_argument_errors_and_out_of_range_ids():
    p, mom, md = _setup(1, 4, 5350)
    ids = torch.tensor([0, 15, -1, 14], dtype=torch.int32, device="cuda")
    w = torch.empty(4, dtype=torch.float64, device="cuda")
    p.sigmakin_ex(md, None, channel_ids=ids, sde=w)
    torch.cuda.synchronize()
    got = w.cpu().numpy()
    assert got[1] == 0.0 and got[2] == 0.0 and got[0] > 0.0 and got[3] > 0.0
    with pytest.raises(binding.MGError):
        p.sigmakin_ex(md, None, channel=0)           # weight output missing
    with pytest.raises(binding.MGError):
        p.sigmakin_ex(md, None, channel_ids=ids)     # weight output missing
    with pytest.raises(binding.MGError):
        p.sigmakin_ex(md, None, channel=15, sde=w)   # 15 channels: 0..14


def test_helicity_and_colour_choice():
    n = 257
    p, mom, md = _setup(2, n, 5400)
    rng = np.random.default_rng(3)
    rh, rc = rng.uniform(size=n), rng.uniform(size=n)
    hel = torch.empty(n, dtype=torch.int32, device="cuda")
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    flow = torch.empty((n, 24), dtype=torch.float64, device="cuda")
    p.sigmakin_ex(md, None, flow=flow, rnd_hel=torch.from_numpy(rh).cuda(), hel_out=hel,
                  rnd_col=torch.from_numpy(rc).cuda(), col_out=col)
    outh = torch.empty((n, 64), dtype=torch.float64, device="cuda")
    p.sigmakin_hel(md, torch.empty(n, dtype=torch.float64, device="cuda"), outh)
    torch.cuda.synchronize()
    mh, fw = outh.cpu().numpy(), flow.cpu().numpy()

    def pick(w, r):
        c = np.cumsum(w)
        return int(np.searchsorted(c, r * c[-1], side="right"))

    exp_h = np.array([pick(mh[e], rh[e]) for e in range(n)])
    exp_c = np.array([pick(fw[e], rc[e]) for e in range(n)])
    got_h, got_c = hel.cpu().numpy(), col.cpu().numpy()
    near_h = np.array([np.min(np.abs(np.cumsum(mh[e]) / mh[e].sum() - rh[e])) < 1e-12 for e in range(n)])
    assert np.array_equal(got_h[~near_h], exp_h[~near_h])
    assert np.array_equal(got_c, exp_c)
    assert got_h.min() >= 0 and got_h.max() < 64 and got_c.min() >= 0 and got_c.max() < 24
