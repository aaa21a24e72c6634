"""HEALPix RING pixelisation, plain FP64 numpy (Gorski et al. 2005, ApJ 622:759,
Sec. 4 and the RING-scheme pixel-centre formulas).

The paper only speaks of "the sky pixel" a sample falls in (Sec. II, Eq. 3
and the pointing matrix of Eq. 8); the pixelisation of the workloads is
HEALPix RING.  This is the oracle for the library's device ``ang2pix``.
Operation order is fixed (one IEEE operation per step, no fused
multiply-add) so that any other implementation that follows the same steps
in correctly rounded FP64 gets the same integer for every input:

    za = |z|;  tt = phi * (2/pi)  (wrapped into [0, 4))
    equatorial belt (za <= 2/3):
        t1 = nside * (0.5 + tt);  t2 = nside * (z * 0.75)
        jp = floor(t1 - t2);  jm = floor(t1 + t2)
        ir = nside + 1 + jp - jm;  kshift = 1 - (ir mod 2)
        ip = ((jp + jm - nside + kshift + 1) div 2) mod 4 nside
        pix = 2 nside (nside - 1) + (ir - 1) 4 nside + ip
    polar caps (za > 2/3):
        tp = tt - floor(tt);  tmp = nside * sqrt(3 * (1 - za))
        jp = floor(tp * tmp);  jm = floor((1 - tp) * tmp)
        ir = jp + jm + 1;  ip = floor(tt * ir) mod 4 ir
        pix = 2 ir (ir - 1) + ip                    (z > 0)
        pix = 12 nside^2 - 2 ir (ir + 1) + ip       (z <= 0)
"""
from __future__ import annotations

import numpy as np

TWO_OVER_PI = 2.0 / np.pi


def nside2npix(nside: int) -> int:
    return 12 * nside * nside


def ang2pix_ring(nside: int, z, phi) -> np.ndarray:
    """RING index of the pixel containing the direction (z = cos theta, phi)."""
    z = np.asarray(z, np.float64)
    phi = np.asarray(phi, np.float64)
    n = np.int64(nside)
    nsd = np.float64(nside)
    za = np.abs(z)
    tt = phi * TWO_OVER_PI
    tt = np.where(tt >= 4.0, tt - 4.0, tt)
    tt = np.where(tt < 0.0, tt + 4.0, tt)
    out = np.empty(z.shape, np.int64)

    eq = za <= 2.0 / 3.0
    if np.any(eq):
        ze, te = z[eq], tt[eq]
        t1 = nsd * (0.5 + te)
        t2 = nsd * (ze * 0.75)
        jp = np.floor(t1 - t2).astype(np.int64)
        jm = np.floor(t1 + t2).astype(np.int64)
        ir = n + 1 + jp - jm
        kshift = 1 - (ir & 1)
        ip = (jp + jm - n + kshift + 1) // 2
        ip = ip % (4 * n)
        out[eq] = 2 * n * (n - 1) + (ir - 1) * 4 * n + ip

    pol = ~eq
    if np.any(pol):
        zp, zap, tp_ = z[pol], za[pol], tt[pol]
        tp = tp_ - np.floor(tp_)
        tmp = nsd * np.sqrt(3.0 * (1.0 - zap))
        jp = np.floor(tp * tmp).astype(np.int64)
        jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
        ir = jp + jm + 1
        ip = np.floor(tp_ * ir.astype(np.float64)).astype(np.int64)
        ip = ip % (4 * ir)
        north = 2 * ir * (ir - 1) + ip
        south = 12 * n * n - 2 * ir * (ir + 1) + ip
        out[pol] = np.where(zp > 0.0, north, south)
    return out


def _isqrt(a: np.ndarray) -> np.ndarray:
    """Exact integer square root floor(sqrt(a)) for a >= 0 (int64)."""
    r = np.floor(np.sqrt(a.astype(np.float64))).astype(np.int64)
    r = np.where(r * r > a, r - 1, r)
    r = np.where((r + 1) * (r + 1) <= a, r + 1, r)
    return r


def pix2ang_ring(nside: int, pix) -> tuple[np.ndarray, np.ndarray]:
    """Centre (z, phi) of RING pixels.

    North cap (pix < 2 nside (nside-1)): ring i = floor((1 + sqrt(1 + 2 pix)) / 2)
    from the pole, j = pix - 2 i (i-1) + 1, z = 1 - i^2 / (3 nside^2),
    phi = (j - 1/2) pi / (2 i).  Equatorial belt: ring i = (pix - ncap) div 4nside
    + nside, j = (pix - ncap) mod 4nside + 1, s = (i - nside) mod 2,
    z = (2 nside - i) 2 / (3 nside), phi = (j - (1 + s)/2) pi / (2 nside).
    South cap: the mirror of the north cap counted from the last pixel."""
    p = np.asarray(pix, np.int64)
    n = np.int64(nside)
    npix = 12 * n * n
    ncap = 2 * n * (n - 1)
    z = np.empty(p.shape, np.float64)
    phi = np.empty(p.shape, np.float64)

    north = p < ncap
    if np.any(north):
        pn = p[north]
        i = (1 + _isqrt(1 + 2 * pn)) // 2
        j = pn - 2 * i * (i - 1) + 1
        fi = i.astype(np.float64)
        z[north] = 1.0 - fi * fi / (3.0 * float(n) * float(n))
        phi[north] = (j.astype(np.float64) - 0.5) * np.pi / (2.0 * fi)

    south = p >= npix - ncap
    if np.any(south):
        ps = npix - p[south]
        i = (1 + _isqrt(2 * ps - 1)) // 2
        j = 4 * i + 1 - (ps - 2 * i * (i - 1))
        fi = i.astype(np.float64)
        z[south] = -1.0 + fi * fi / (3.0 * float(n) * float(n))
        phi[south] = (j.astype(np.float64) - 0.5) * np.pi / (2.0 * fi)

    eq = ~(north | south)
    if np.any(eq):
        pe = p[eq] - ncap
        i = pe // (4 * n) + n
        j = pe % (4 * n) + 1
        s = (i - n) % 2
        z[eq] = (2.0 * float(n) - i.astype(np.float64)) * 2.0 / (3.0 * float(n))
        phi[eq] = (j.astype(np.float64) - (1.0 + s.astype(np.float64)) / 2.0) * np.pi / (2.0 * float(n))
    return z, phi


def ring_of_pixel(nside: int, pix) -> np.ndarray:
    """Ring index 1 .. 4 nside - 1 (counted from the north pole) of RING pixels."""
    p = np.asarray(pix, np.int64)
    n = np.int64(nside)
    npix = 12 * n * n
    ncap = 2 * n * (n - 1)
    ring = np.empty(p.shape, np.int64)
    north = p < ncap
    south = p >= npix - ncap
    eq = ~(north | south)
    ring[north] = (1 + _isqrt(1 + 2 * p[north])) // 2
    ring[south] = 4 * n - (1 + _isqrt(2 * (npix - p[south]) - 1)) // 2
    ring[eq] = (p[eq] - ncap) // (4 * n) + n
    return ring
