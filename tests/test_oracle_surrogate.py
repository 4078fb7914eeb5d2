"""Pins of the surrogate oracle (no GPU)."""
import numpy as np

from oracle import surrogate as S
from paper_2510_05392_gb300 import phasespace as ps


def test_features_are_pair_invariants():
    mom = ps.generate(50, 4, 2000.0, 3, ptmin=20.0, drmin=0.4)
    x = S.features(mom)
    assert x.shape == (50, 32)
    np.testing.assert_allclose(x[:, 0], 0.0, atol=1e-12)         # log(s_12 / s)
    assert np.all(x[:, 28:] == 0.0)
    # massive pair (t, t~): s_34 >= 4 m^2
    k34 = [(i, j) for i in range(8) for j in range(i + 1, 8)].index((2, 3))
    assert np.all(np.exp(x[:, k34]) * 2000.0 ** 2 >= 4 * 173.0 ** 2 * (1 - 1e-12))
    # an explicit pair: log((p_4 + p_6)^2 / s) from the four-vectors
    k46 = [(i, j) for i in range(8) for j in range(i + 1, 8)].index((4, 6))
    q = mom[:, 4] + mom[:, 6]
    np.testing.assert_allclose(x[:, k46], np.log((q[:, 0] ** 2 - (q[:, 1:] ** 2).sum(1)) / 2000.0 ** 2),
                               rtol=1e-9)
    # momentum conservation: sum over j != i of s_ij relates to masses, and
    # Lorentz invariance: a boost leaves the features unchanged
    b = np.array([0.3, -0.1, 0.4]); g = 1 / np.sqrt(1 - b @ b)
    L = np.eye(4); L[0, 0] = g; L[0, 1:] = L[1:, 0] = g * b
    L[1:, 1:] += (g - 1) * np.outer(b, b) / (b @ b)
    np.testing.assert_allclose(S.features(mom @ L.T), x, rtol=1e-9, atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = S.init_params([32, 16, 16, 16, 1], seed=2)
    x = rng.uniform(0, 1, (7, 32))
    y = rng.normal(size=7)
    loss, grads = S.loss_and_grads(params, x, y)
    h = 1e-6
    for l in range(len(params)):
        for k in range(2):
            P = params[l][k]
            flat = P.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = S.loss_and_grads(params, x, y)
                flat[idx] = old - h
                lm, _ = S.loss_and_grads(params, x, y)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[l][k].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-7 * max(1e-3, abs(an)) + 1e-10


def test_linear_model_reaches_normal_equations():
    """One linear layer trained by the oracle's Adam converges to the
    least-squares solution of the normal equations."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(256, 4))
    y = x @ np.array([0.5, -1.0, 2.0, 0.25]) + 0.3 + 0.01 * rng.normal(size=256)
    params = S.init_params([4, 1], seed=0)
    st = {}
    for _ in range(3000):
        _, g = S.loss_and_grads(params, x, y)
        S.adam_step(params, g, st, lr=1e-2)
    A = np.hstack([x, np.ones((256, 1))])
    sol = np.linalg.lstsq(A, y, rcond=None)[0]
    np.testing.assert_allclose(params[0][0][0], sol[:4], atol=2e-3)
    np.testing.assert_allclose(params[0][1][0], sol[4], atol=2e-3)


def test_unweighting_special_cases_and_unbiasedness():
    rng = np.random.default_rng(7)
    n = 200000
    w = rng.lognormal(0.0, 1.0, n)
    u1, u2 = rng.uniform(size=n), rng.uniform(size=n)
    # perfect surrogate: stage 2 always accepts, plain unweighting
    acc, wt, s1 = S.unweight_two_stage(w, w, u1, u2, w.max(), 1.0)
    assert np.array_equal(acc, u1 < w / w.max())
    # constant surrogate: stage 1 keeps everything, stage 2 is hit-or-miss on w
    c = np.full(n, 1.0)
    acc, wt, s1 = S.unweight_two_stage(w, c, u1, u2, 1.0, w.max())
    assert s1.all() and np.array_equal(acc, u2 < w / w.max())
    # any surrogate: the weighted accepted sum estimates sum(w) / max-normaliser
    what = w * rng.lognormal(0.0, 0.3, n)
    wmax, rmax = np.quantile(what, 0.99), np.quantile(w / what, 0.99)
    acc, wt, s1 = S.unweight_two_stage(w, what, u1, u2, wmax, rmax)
    est = wt.sum() * wmax * rmax
    assert abs(est / w.sum() - 1) < 0.02


def test_bf16_rounding_reference_values():
    r = S.round_bf16
    assert r(np.array([1.0]))[0] == 1.0
    assert r(np.array([1.0 + 2.0 ** -9]))[0] == 1.0              # tie -> even
    assert r(np.array([1.0 + 3 * 2.0 ** -9]))[0] == 1.0 + 2.0 ** -7
    assert r(np.array([-3.0 - 2.0 ** -8]))[0] == -3.0
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(r(x) / x - 1) <= 2.0 ** -8)
    y = r(x)
    np.testing.assert_array_equal(r(y), y)


def test_emulated_bf16_gradients_close_to_exact():
    rng = np.random.default_rng(2)
    params = S.init_params([32, 64, 64, 1], seed=1)
    x = rng.uniform(0, 1, (128, 32))
    y = rng.normal(size=128)
    _, g = S.loss_and_grads(params, x, y)
    _, ge = S.loss_and_grads(params, x, y, emulate_bf16=True)
    for l in range(3):
        assert np.linalg.norm(ge[l][0] - g[l][0]) < 0.05 * np.linalg.norm(g[l][0])
