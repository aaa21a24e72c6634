"""The seeded input generator: counter-based RNG, scan, data model."""
import math

import numpy as np
import pytest

import synth
from conftest import read_golden


def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = synth.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_are_counter_based_and_standard():
    a = synth.normal(7, 3, 200_000)
    b = synth.normal(7, 3, 1000, start=123_456)
    assert np.array_equal(a[123_456:124_456], b)
    assert abs(a.mean()) < 5 / math.sqrt(a.size)
    assert abs(a.var() - 1.0) < 5 * math.sqrt(2.0 / a.size)
    assert not np.array_equal(a[:100], synth.normal(8, 3, 100))


def test_scan_is_deterministic_and_in_range():
    e = synth.make_experiment(16, 4, 8192, 1000)
    p1 = synth.pointing(e, with_angles=True)
    p2 = synth.pointing(e, with_angles=True)
    assert np.array_equal(p1["pix"], p2["pix"]) and np.array_equal(p1["psi"], p2["psi"])
    assert p1["pix"].min() >= 0 and p1["pix"].max() < e.npix
    assert p1["psi"].min() >= 0 and p1["psi"].max() < math.pi
    assert np.all(np.abs(p1["z"]) <= 1) and np.all((p1["phi"] >= 0) & (p1["phi"] < 2 * math.pi))
    # The pixel of a sample is the simulator's HEALPix pixel of its direction.
    assert np.array_equal(synth.ang2pix_ring(16, p1["z"], p1["phi"]), p1["pix"])


def test_scan_geometry_covers_the_expected_cap():
    # Boresight within beta +- alpha = [5, 95] deg of the precession axis (+x):
    # about (1 - cos 95deg) / 2 = 54% of the sky is ever observed.
    e = synth.make_experiment(16, 4, 72_000, 1000)  # one precession period
    pt = synth.pointing(e, with_angles=True)
    x = np.sqrt(1 - pt["z"] ** 2) * np.cos(pt["phi"])
    ang = np.degrees(np.arccos(np.clip(x, -1, 1)))
    assert ang.min() > 5 - 1.01 and ang.max() < 95 + 1.01
    h = np.bincount(pt["pix"], minlength=e.npix)
    assert 0.45 < (h > 0).mean() < 0.65


def test_flagging_fraction():
    e = synth.make_experiment(16, 4, 50_000, 3)
    pt = synth.pointing(e, flag_frac=0.1)
    frac = (pt["pix"] < 0).mean()
    assert abs(frac - 0.1) < 0.01


def test_tod_data_model_noiseless():
    e = synth.make_experiment(8, 4, 1000, 5)
    pt = synth.pointing(e)
    sky = synth.sky_map(e.npix, 5)
    d = synth.tod(e, pt["pix"], pt["psi"], sky, white=False)
    p, a = pt["pix"], 2 * pt["psi"]
    expect = sky[p, 0] + sky[p, 1] * np.cos(a) + sky[p, 2] * np.sin(a)
    np.testing.assert_allclose(d, expect, rtol=0, atol=1e-12)
    d32 = synth.tod(e, pt["pix"], pt["psi"], sky, white=False, dtype=np.float32)
    assert d32.dtype == np.float32 and np.array_equal(d32, d.astype(np.float32))


def test_tod_white_noise_level():
    e = synth.make_experiment(8, 4, 50_000, 9)
    pt = synth.pointing(e)
    sky = np.zeros((e.npix, 3))
    d = synth.tod(e, pt["pix"], pt["psi"], sky).reshape(e.ndet, e.ns)
    np.testing.assert_allclose(d.std(axis=1), e.sigma, rtol=0.02)


def test_toeplitz_band_symbol_nonnegative():
    sig = np.array([1.0, 1.7])
    c = synth.toeplitz_band(sig, 0.1, 1.0, 20.0, 2 ** 16, 512)
    assert c.shape == (2, 512)
    np.testing.assert_allclose(c[1], c[0] / 1.7 ** 2)
    # Symbol c0 + 2 sum_k c_k cos(k w) on a fine grid.
    w = np.linspace(0, math.pi, 8193)
    k = np.arange(1, 512)
    sym = c[0, 0] + 2 * np.cos(np.outer(w, k)) @ c[0, 1:]
    assert sym.min() > 0
    assert abs(sym[-1] - 1.0) < 0.05  # far above fknee the inverse spectrum is ~1/sigma^2


def test_one_over_f_spectrum_shape():
    e = synth.make_experiment(8, 1, 2 ** 16, 11)
    n = synth.one_over_f_noise(e, 2 ** 16, 0.1, 1.0)
    f = np.fft.rfftfreq(n.size, 1 / 20.0)
    p = np.abs(np.fft.rfft(n)) ** 2 / n.size
    lo = p[(f > 0.005) & (f < 0.02)].mean()
    hi = p[(f > 5) & (f < 10)].mean()
    # expected ratio (1 + 0.1/0.0125)/(1 + 0.1/7.5) ~ 8.9
    assert 5 < lo / hi < 14
    assert abs(hi / e.sigma[0] ** 2 - 1.0) < 0.1
