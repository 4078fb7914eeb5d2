"""The seeded input generator (no GPU)."""
import numpy as np

from paper_2510_05392_gb300 import phasespace as ps


def test_philox_known_answers():
    # Known-answer vectors published with the Random123 reference implementation
    f = ps.philox4x32_10
    z = f(np.zeros(4, np.uint32), np.zeros(2, np.uint32))
    assert [int(x) for x in z] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    o = f(np.full(4, 0xFFFFFFFF, np.uint32), np.full(2, 0xFFFFFFFF, np.uint32))
    assert [int(x) for x in o] == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    pi = f(np.array([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], np.uint32),
           np.array([0xA4093822, 0x299F31D0], np.uint32))
    assert [int(x) for x in pi] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_momenta_conserve_and_are_on_shell():
    p = ps.generate(2000, 3, 1500.0, 1, ptmin=20.0, drmin=0.4)
    tot = p[:, 0] + p[:, 1] - p[:, 2:].sum(1)
    assert np.abs(tot).max() < 1e-9
    m2 = p[..., 0] ** 2 - (p[..., 1:] ** 2).sum(-1)
    np.testing.assert_allclose(np.sqrt(m2[:, 2:4]), 173.0, rtol=1e-10)
    assert np.abs(m2[:, 4:]).max() < 1e-6
    pt = np.hypot(p[:, 4:, 1], p[:, 4:, 2])
    assert pt.min() > 20.0


def test_candidate_counter_is_batch_independent():
    a = ps.generate(300, 2, 1500.0, 3, ptmin=20.0, drmin=0.4, batch=1 << 12)
    b = ps.generate(300, 2, 1500.0, 3, ptmin=20.0, drmin=0.4, batch=97)
    assert np.array_equal(a, b)


def test_weights_positive_and_massless_volume():
    # massless 2-body: flat weight = (2 pi)^-2 (pi/2) / 1 = 1/(8 pi)
    p, w, _ = ps.generate(10, 0, 1000.0, 4, mt=0.0, return_weights=True)
    np.testing.assert_allclose(w, 1 / (8 * np.pi), rtol=1e-12)
    p, w, _ = ps.generate(10, 2, 1500.0, 4, return_weights=True)
    assert np.all(w > 0)
