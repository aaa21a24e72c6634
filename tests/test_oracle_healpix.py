"""Pins of the oracle's HEALPix RING pixelisation (Gorski et al. 2005)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import healpix


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64, 256, 512])
def test_round_trip_every_pixel(nside):
    p = np.arange(healpix.nside2npix(nside))
    z, phi = healpix.pix2ang_ring(nside, p)
    assert np.array_equal(healpix.ang2pix_ring(nside, z, phi), p)


def test_base_pixel_centres_textbook():
    for pix, zs, ps in read_golden("healpix_nside1_centres.txt"):
        z, phi = healpix.pix2ang_ring(1, np.array([int(pix)]))
        assert z[0] == pytest.approx(float(Fraction(zs)), abs=1e-15)
        assert phi[0] == pytest.approx(float(Fraction(ps)) * math.pi, abs=1e-15)
        assert healpix.ang2pix_ring(1, z, phi)[0] == int(pix)


@pytest.mark.parametrize("nside", [1, 4, 16, 128])
def test_ring_structure(nside):
    # 4i pixels on ring i of the polar caps, 4 nside on every belt ring,
    # rings numbered 1 .. 4 nside - 1, pixels of a ring contiguous.
    p = np.arange(healpix.nside2npix(nside))
    ring = healpix.ring_of_pixel(nside, p)
    assert ring.min() == 1 and ring.max() == 4 * nside - 1
    assert np.all(np.diff(ring) >= 0)
    counts = np.bincount(ring)[1:]
    i = np.arange(1, 4 * nside)
    expect = np.minimum(np.minimum(4 * i, 4 * nside), 4 * (4 * nside - i))
    assert np.array_equal(counts, expect)
    # centres of a ring share z; z decreases ring by ring
    z, _ = healpix.pix2ang_ring(nside, p)
    zr = np.array([z[ring == r][0] for r in i])
    assert np.all(np.diff(zr) < 0)


@pytest.mark.parametrize("nside", [1, 8, 32])
def test_poles(nside):
    assert healpix.ang2pix_ring(nside, np.array([1.0]), np.array([0.3]))[0] == 0
    s = healpix.ang2pix_ring(nside, np.array([-1.0]), np.array([5.0]))[0]
    assert healpix.nside2npix(nside) - 4 <= s < healpix.nside2npix(nside)


def test_equal_area():
    # Uniform points on the sphere fill every pixel equally (chi-square).
    rng = np.random.default_rng(0)
    n, nside = 2_000_000, 8
    z = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    h = np.bincount(healpix.ang2pix_ring(nside, z, phi), minlength=768)
    e = n / 768
    chi2 = np.sum((h - e) ** 2 / e)
    assert abs(chi2 - 767) < 6 * math.sqrt(2 * 767)


def test_points_near_centres_stay():
    nside = 32
    p = np.arange(healpix.nside2npix(nside))
    z, phi = healpix.pix2ang_ring(nside, p)
    rng = np.random.default_rng(1)
    dz = rng.uniform(-1, 1, p.size) * 0.05 / nside ** 2
    dphi = rng.uniform(-1, 1, p.size) * 0.05 / nside
    z2 = np.clip(z + dz, -1, 1)
    assert np.array_equal(healpix.ang2pix_ring(nside, z2, (phi + dphi) % (2 * math.pi)), p)


def test_phi_wraps():
    nside = 16
    z = np.linspace(-0.99, 0.99, 101)
    a = healpix.ang2pix_ring(nside, z, np.full(z.size, 1e-12))
    b = healpix.ang2pix_ring(nside, z, np.full(z.size, 2 * math.pi - 1e-12))
    r = healpix.ring_of_pixel(nside, a)
    assert np.array_equal(r, healpix.ring_of_pixel(nside, b))


def test_simulated_pointing_agrees():
    # The simulator's pixelisation and the oracle's agree on a real scan.
    e = synth.make_experiment(64, 16, 20_000, 1234)
    pt = synth.pointing(e, with_angles=True)
    assert np.array_equal(healpix.ang2pix_ring(64, pt["z"], pt["phi"]), pt["pix"])


def test_planted_mistake_is_caught(monkeypatch):
    # A wrong shift rule in the belt (a plausible slip) breaks the round trip.
    orig = healpix.ang2pix_ring

    def wrong(nside, z, phi):
        out = orig(nside, z, phi)
        z = np.asarray(z)
        belt = np.abs(z) <= 2 / 3
        n = nside
        ncap = 2 * n * (n - 1)
        ring = (out - ncap) // (4 * n) + n
        shifted = belt & ((ring - n) % 2 == 0)
        out = out.copy()
        out[shifted] = ncap + (ring[shifted] - n) * 4 * n + ((out[shifted] - ncap) % (4 * n) + 1) % (4 * n)
        return out

    p = np.arange(healpix.nside2npix(4))
    z, phi = healpix.pix2ang_ring(4, p)
    assert not np.array_equal(wrong(4, z, phi), p)
