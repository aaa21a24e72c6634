"""Seeded synthetic inputs shared by the oracle's tests and by the CUDA library's
tests and benchmark.

This module simulates the *experiment*, not the map-maker: a spinning and
precessing scan, the HEALPix pixel that each simulated sample falls in, the
polarisation angle with a rotating half-wave plate, a Gaussian sky, white and
1/f noise, and the time-ordered data of the paper's data model (Eq. 1-2).
It also turns a noise power spectrum into the banded inverse-noise filter
coefficients that a caller hands to the library (the 512-lag band with a
Bartlett taper).  None of the GLS solve (pointing operator, noise weighting,
preconditioner, PCG) lives here.

Everything is deterministic given the seed: per-detector parameters come from
numpy's PCG64, per-sample random numbers from a counter-based Philox4x32-10
generator in ``synth.c`` (so any subset of samples can be regenerated alone).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libbmsynth.so")
_lib = None

# Solver types (number of Stokes components per pixel).
SOLVER_I, SOLVER_QU, SOLVER_IQU = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``libbmsynth.so`` next to this file with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _ScanParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "fsamp", "spin_hz", "prec_period_s", "alpha_rad", "beta_rad",
        "hwp_hz", "hwp_phase0", "spin_phase0", "prec_phase0")]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, u64, u32, f64 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        lib.synth_philox4x32_10.argtypes = [P, P, P]
        lib.synth_normal.argtypes = [u64, u32, i64, i64, f64, P]
        lib.synth_uniform.argtypes = [u64, u32, i64, P]
        lib.synth_ang2pix_ring.argtypes = [i64, i64, P, P, P]
        lib.synth_scan.argtypes = [ctypes.POINTER(_ScanParams), i64, ctypes.c_int32, i64, i64,
                                   P, P, P, f64, u64, P, P, P, P]
        lib.synth_tod.argtypes = [i64, i64, P, P, P, f64, f64, P, u64, P, P, P, P, P]
        lib.synth_trig32.argtypes = [i64, P, P, P]
        for f in ("synth_philox4x32_10", "synth_normal", "synth_uniform", "synth_ang2pix_ring",
                  "synth_scan", "synth_tod", "synth_trig32"):
            getattr(lib, f).restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Counter-based random numbers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al. 2011) — exposed for its known-answer test."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    _load().synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normal(seed: int, stream: int, n: int, scale: float = 1.0, start: int = 0) -> np.ndarray:
    """Standard normals start .. start+n-1 of a Philox stream, times scale."""
    out = np.empty(int(n), np.float64)
    _load().synth_normal(seed, stream, int(start), int(n), float(scale), _ptr(out))
    return out


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(int(n), np.float64)
    _load().synth_uniform(seed, stream, int(n), _ptr(out))
    return out


def ang2pix_ring(nside: int, z: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """The simulator's own HEALPix RING pixelisation (used to build pointing)."""
    z = np.ascontiguousarray(z, np.float64)
    phi = np.ascontiguousarray(phi, np.float64)
    pix = np.empty(z.shape, np.int32)
    _load().synth_ang2pix_ring(int(nside), z.size, _ptr(z), _ptr(phi), _ptr(pix))
    return pix


# --------------------------------------------------------------------------
# Experiment description
# --------------------------------------------------------------------------
@dataclass
class ScanSpec:
    """Scan law: spin 0.05 Hz, precession period 1 h, 20 Hz sampling, HWP 1 Hz,
    precession opening 45 deg, spin angle 50 deg."""
    fsamp: float = 20.0
    spin_hz: float = 0.05
    prec_period_s: float = 3600.0
    alpha_deg: float = 45.0
    beta_deg: float = 50.0
    hwp_hz: float = 1.0
    det_span_deg: float = 1.0  # detector offsets within +-span of the boresight


@dataclass
class Experiment:
    """Per-detector parameters of one simulated run (seeded)."""
    nside: int
    ndet: int
    ns: int                      # samples per detector
    seed: int
    scan: ScanSpec = field(default_factory=ScanSpec)
    ox: np.ndarray = None        # focal-plane offsets [rad]
    oy: np.ndarray = None
    psi_det: np.ndarray = None   # detector polarisation angle, U[0, pi)
    sigma: np.ndarray = None     # white-noise rms per sample [uK], U[1, 2]
    hwp_phase0: float = 0.0
    spin_phase0: float = 0.0
    prec_phase0: float = 0.0

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside

    @property
    def nsamples(self) -> int:
        return self.ndet * self.ns

    @property
    def det_offsets(self) -> np.ndarray:
        return np.arange(self.ndet + 1, dtype=np.int64) * self.ns


def detector_offsets(ndet: int, span_deg: float):
    """Focal-plane offsets: four detectors on a cross at (+-span, 0), (0, +-span);
    otherwise a k x k square grid spanning +-span (row-major, first ndet)."""
    s = math.radians(span_deg)
    if ndet == 4:
        ox = np.array([s, -s, 0.0, 0.0])
        oy = np.array([0.0, 0.0, s, -s])
        return ox, oy
    k = max(1, math.ceil(math.sqrt(ndet)))
    g = np.linspace(-s, s, k) if k > 1 else np.zeros(1)
    gx, gy = np.meshgrid(g, g, indexing="xy")
    return gx.ravel()[:ndet].copy(), gy.ravel()[:ndet].copy()


def make_experiment(nside: int, ndet: int, ns: int, seed: int, scan: ScanSpec | None = None) -> Experiment:
    scan = scan or ScanSpec()
    rng = np.random.default_rng(seed)
    ox, oy = detector_offsets(ndet, scan.det_span_deg)
    psi_det = rng.uniform(0.0, math.pi, ndet)
    sigma = rng.uniform(1.0, 2.0, ndet)
    hwp0, spin0, prec0 = rng.uniform(0.0, 2 * math.pi, 3)
    return Experiment(nside=nside, ndet=ndet, ns=ns, seed=seed, scan=scan, ox=ox, oy=oy,
                      psi_det=psi_det, sigma=sigma, hwp_phase0=float(hwp0),
                      spin_phase0=float(spin0), prec_phase0=float(prec0))


def _scan_params(e: Experiment) -> _ScanParams:
    s = e.scan
    return _ScanParams(s.fsamp, s.spin_hz, s.prec_period_s, math.radians(s.alpha_deg),
                       math.radians(s.beta_deg), s.hwp_hz, e.hwp_phase0, e.spin_phase0,
                       e.prec_phase0)


def pointing(e: Experiment, flag_frac: float = 0.0, with_angles: bool = False,
             psi_dtype=np.float64):
    """Simulated pointing, laid out [ndet][ns]: pix (int32, -1 = flagged), psi,
    and optionally the direction (z = cos theta, phi)."""
    n = e.nsamples
    pix = np.empty(n, np.int32)
    psi = np.empty(n, np.float64)
    z = np.empty(n, np.float64) if with_angles else None
    phi = np.empty(n, np.float64) if with_angles else None
    sp = _scan_params(e)
    ox = np.ascontiguousarray(e.ox, np.float64)
    oy = np.ascontiguousarray(e.oy, np.float64)
    pd = np.ascontiguousarray(e.psi_det, np.float64)
    _load().synth_scan(ctypes.byref(sp), e.nside, e.ndet, 0, e.ns, _ptr(ox), _ptr(oy), _ptr(pd),
                       float(flag_frac), (e.seed * 7919 + 17) & 0xFFFFFFFFFFFFFFFF,
                       _ptr(pix), _ptr(psi), _ptr(z), _ptr(phi))
    out = {"pix": pix, "psi": psi.astype(psi_dtype) if psi_dtype != np.float64 else psi}
    if with_angles:
        out["z"], out["phi"] = z, phi
    return out


def sky_map(npix: int, seed: int, sigma_i: float = 100.0, sigma_qu: float = 10.0,
            realisation: int = 0) -> np.ndarray:
    """Gaussian sky [npix][3] (I, Q, U): iid per pixel, I ~ N(0, sigma_i^2),
    Q, U ~ N(0, sigma_qu^2) in uK."""
    m = normal(seed, 100 + realisation, 3 * npix).reshape(npix, 3)
    m[:, 0] *= sigma_i
    m[:, 1:] *= sigma_qu
    return m


def stokes_weights(solver: int):
    """Which Stokes parameters the simulated sky contributes for a solver type."""
    return {SOLVER_IQU: (1.0, 1.0), SOLVER_QU: (0.0, 1.0), SOLVER_I: (1.0, 0.0)}[solver]


def trig32(psi):
    """(cos 2psi, sin 2psi) rounded to FP32: precomputed pointing entries."""
    psi = np.ascontiguousarray(psi, np.float64)
    c = np.empty(psi.size, np.float32)
    s = np.empty(psi.size, np.float32)
    _load().synth_trig32(psi.size, _ptr(psi), _ptr(c), _ptr(s))
    return c, s


def tod(e: Experiment, pix, psi, sky, solver: int = SOLVER_IQU, white: bool = True,
        noise_seed: int | None = None, extra=None, dtype=np.float64, noise_scale: float = 1.0,
        trig=None):
    """Time-ordered data [ndet][ns] of the data model d = s + n (Eq. 1-2).
    ``white``: add sigma_det * N(0,1); ``extra``: an additional noise stream
    (e.g. 1/f) added sample by sample; ``trig``: FP32 (cos 2psi, sin 2psi) to
    use as the pointing entries instead of the angle."""
    aI, aP = stokes_weights(solver)
    pix = np.ascontiguousarray(pix, np.int32)
    psi = np.ascontiguousarray(psi, np.float64)
    sky = np.ascontiguousarray(sky, np.float64)
    sig = np.ascontiguousarray(e.sigma * noise_scale, np.float64) if white else None
    ext = None if extra is None else np.ascontiguousarray(extra, np.float64)
    seed = e.seed if noise_seed is None else noise_seed
    n = e.nsamples
    out64 = np.empty(n, np.float64) if dtype == np.float64 else None
    out32 = np.empty(n, np.float32) if dtype == np.float32 else None
    c32 = s32 = None
    if trig is not None:
        c32 = np.ascontiguousarray(trig[0], np.float32)
        s32 = np.ascontiguousarray(trig[1], np.float32)
    _load().synth_tod(e.ndet, e.ns, _ptr(pix), _ptr(psi), _ptr(sky), aI, aP, _ptr(sig),
                      seed, _ptr(ext), _ptr(out64), _ptr(out32), _ptr(c32), _ptr(s32))
    return out64 if out64 is not None else out32


# --------------------------------------------------------------------------
# 1/f noise and the banded inverse-noise filter handed to the library
# --------------------------------------------------------------------------
def psd(f, sigma: float, fknee: float, alpha: float):
    """Noise power spectrum sigma^2 (1 + (fknee/f)^alpha) (per-sample variance units)."""
    f = np.asarray(f, np.float64)
    with np.errstate(divide="ignore"):
        return sigma * sigma * (1.0 + (fknee / f) ** alpha)


def toeplitz_band(sigma: np.ndarray, fknee: float, alpha: float, fsamp: float,
                  grid_len: int, nlags: int) -> np.ndarray:
    """Inverse-noise band c[d][k], k = 0..nlags-1, for each detector.

    The inverse spectrum 1/P(f_j) is sampled on the frequency grid of length
    ``grid_len`` (f_j = j fsamp / grid_len, the zero-frequency term set to 0
    since a 1/f spectrum diverges there), transformed back to lags by the real
    inverse DFT, truncated to |k| < nlags and multiplied by the Bartlett taper
    (1 - k/nlags).  The taper's transform is the non-negative Fejer kernel, so
    the band's symbol stays >= 0 and every finite section is positive
    semi-definite.  Per detector the band scales as 1/sigma_d^2."""
    j = np.arange(grid_len // 2 + 1)
    f = j * (fsamp / grid_len)
    ip = np.zeros_like(f)
    ip[1:] = 1.0 / psd(f[1:], 1.0, fknee, alpha)
    lag = np.fft.irfft(ip, n=grid_len)[:nlags]
    lag = lag * (1.0 - np.arange(nlags) / nlags)
    sig = np.asarray(sigma, np.float64)
    return lag[None, :] / (sig[:, None] ** 2)


def one_over_f_noise(e: Experiment, chunk_len: int, fknee: float, alpha: float,
                     seed: int | None = None) -> np.ndarray:
    """Noise with spectrum sigma_d^2 (1 + (fknee/f)^alpha), generated chunk by
    chunk by shaping Philox white noise in the Fourier domain (the zero
    frequency takes the gain of the first non-zero frequency).  [ndet][ns] FP64."""
    seed = e.seed if seed is None else seed
    out = np.empty(e.nsamples, np.float64)
    for d in range(e.ndet):
        w = normal(seed, 200, e.ns, scale=float(e.sigma[d]), start=d * e.ns)
        for c0 in range(0, e.ns, chunk_len):
            seg = w[c0:c0 + chunk_len]
            L = seg.size
            fr = np.fft.rfftfreq(L, 1.0 / e.scan.fsamp)
            g = np.empty_like(fr)
            g[1:] = np.sqrt(1.0 + (fknee / fr[1:]) ** alpha)
            g[0] = g[1] if L > 1 else 1.0
            out[d * e.ns + c0: d * e.ns + c0 + L] = np.fft.irfft(np.fft.rfft(seg) * g, n=L)
    return out
