"""Plain FP64 generalized-least-squares map-making (the paper's Sec. II), written
for a reader to check against the equations, not for speed.

Notation follows the paper: d = P s + n (Eq. 3), the pointing matrix P has one
row per time sample with the non-zeros [1, cos 2psi_t, sin 2psi_t] in the
columns (I_p, Q_p, U_p) of the pixel p_t hit at time t (Eq. 8; the angle is
called theta in the paper, psi here), the GLS estimate solves
A x = b with A = P^T N^-1 P and b = P^T N^-1 d (Eq. 5-6), and the
block-diagonal preconditioner is M = (P^T diag(N)^-1 P)^-1 (Eq. 7).

Readings where the paper is silent (each is listed with its reason in the
design notes):
  * QU solves use the rows [cos 2psi, sin 2psi]; I solves the row [1].
  * A pixel is masked when it has fewer than ``min_hits`` samples, or (for
    QU and IQU) when its block is not positive definite or its condition
    number lambda_max / lambda_min exceeds ``max_cond`` (strictly).
  * Masked pixels leave the unknowns: the rows of P for samples in masked
    pixels, and for flagged samples (pixel index -1), are zero, and those
    samples of d are set to zero before N^-1 is applied.
  * The banded Toeplitz N^-1 acts on each detector's samples chunk by chunk
    (chunks of ``chunk_len`` samples, the last one possibly shorter), with
    nothing coupled across chunk edges.
  * diag(N)^-1 in Eq. 7 is the per-detector white level 1/sigma_d^2.
  * PCG starts from x = 0 and stops when ||r||_2 <= tol ||b||_2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

I_ONLY, QU, IQU = 1, 2, 3


# ----------------------------------------------------------------------------
# Pointing matrix (Eq. 8)
# ----------------------------------------------------------------------------
def pointing_weights(psi, ncomp: int) -> np.ndarray:
    """Non-zeros of each row of P (Eq. 2 and 8): [1, cos 2psi, sin 2psi] for IQU,
    [cos 2psi, sin 2psi] for QU, [1] for I.  Shape [Nt, ncomp], FP64."""
    psi = np.asarray(psi, np.float64)
    if ncomp == IQU:
        return np.stack([np.ones_like(psi), np.cos(2.0 * psi), np.sin(2.0 * psi)], axis=1)
    if ncomp == QU:
        return np.stack([np.cos(2.0 * psi), np.sin(2.0 * psi)], axis=1)
    if ncomp == I_ONLY:
        return np.ones((psi.size, 1))
    raise ValueError("ncomp must be 1, 2 or 3")


def pointing_weights_trig(c, s, ncomp: int) -> np.ndarray:
    """Rows of P from precomputed c = cos 2psi and s = sin 2psi (e.g. FP32
    values delivered with the data): the given numbers are the entries."""
    c = np.asarray(c, np.float64)
    s = np.asarray(s, np.float64)
    if ncomp == IQU:
        return np.stack([np.ones_like(c), c, s], axis=1)
    if ncomp == QU:
        return np.stack([c, s], axis=1)
    if ncomp == I_ONLY:
        return np.ones((c.size, 1))
    raise ValueError("ncomp must be 1, 2 or 3")


def hwp_angles(det_offsets, psi_det, nu, phi0) -> np.ndarray:
    """Polarisation angle of every sample under a rotating half-wave plate
    (Eq. 2: theta includes the optics; the build's reading of the HWP is
    theta = psi_d + 2 phi_hwp): sample k of detector d (k counted from the
    detector's first sample, which is taken at k = 0) has
        theta = psi_d + 2 phi_hwp(k),   phi_hwp(k) = 2 pi nu k + phi0,
    nu the plate's turns per sample (f_hwp / f_samp).  2 pi nu k is a multiple
    of 2 pi plus 2 pi frac(nu k); frac(nu k) is formed exactly from the
    rational value of nu (a binary FP64 number) with Python integers, so the
    angle keeps FP64 accuracy however long the detector.  Samples laid out
    detector by detector; FP64 [nsamples]."""
    from fractions import Fraction
    off = np.asarray(det_offsets, np.int64)
    psi_det = np.asarray(psi_det, np.float64)
    fr = Fraction(float(nu))
    num, den = fr.numerator, fr.denominator
    out = np.empty(int(off[-1]))
    for d in range(off.size - 1):
        n = int(off[d + 1] - off[d])
        # frac(nu k) = ((num k) mod den) / den, exactly, then rounded once
        turns = np.array([((num * k) % den) / den for k in range(n)], np.float64)
        out[off[d]:off[d + 1]] = psi_det[d] + 2.0 * (2.0 * np.pi * turns + phi0)
    return out


def hits(pix, npix: int) -> np.ndarray:
    """Number of samples in each pixel (flagged samples, pix = -1, not counted)."""
    pix = np.asarray(pix)
    return np.bincount(pix[pix >= 0], minlength=npix).astype(np.int64)


def effective_pixels(pix, mask) -> np.ndarray:
    """Pixel index of each sample, with -1 for flagged samples and for samples
    whose pixel is masked (their row of P is zero)."""
    pix = np.asarray(pix, np.int64)
    pe = pix.copy()
    valid = pe >= 0
    pe[valid & mask[np.where(valid, pe, 0)].astype(bool)] = -1
    return pe


def apply_P(pe, v, x) -> np.ndarray:
    """y = P x: y_t = sum_k v[t, k] x[p_t, k]; zero rows where pe = -1."""
    x = np.asarray(x, np.float64)
    ok = pe >= 0
    y = np.zeros(pe.size)
    y[ok] = np.sum(v[ok] * x[pe[ok]], axis=1)
    return y


def apply_PT(pe, v, y, npix: int) -> np.ndarray:
    """q = P^T y: q[p, k] = sum over samples t in pixel p of v[t, k] y_t."""
    ok = pe >= 0
    ncomp = v.shape[1]
    q = np.zeros((npix, ncomp))
    for k in range(ncomp):
        q[:, k] = np.bincount(pe[ok], weights=v[ok, k] * y[ok], minlength=npix)
    return q


# ----------------------------------------------------------------------------
# Inverse noise covariance
# ----------------------------------------------------------------------------
def sample_detector(det_offsets) -> np.ndarray:
    """Detector index of each sample for samples laid out detector by detector."""
    off = np.asarray(det_offsets, np.int64)
    return np.repeat(np.arange(off.size - 1), np.diff(off))


@dataclass
class WhiteNoise:
    """Diagonal N^-1 with weight 1/sigma_d^2 for every sample of detector d."""
    inv_var: np.ndarray      # [ndet]
    det_offsets: np.ndarray  # [ndet + 1]

    def sample_weights(self) -> np.ndarray:
        return np.asarray(self.inv_var, np.float64)[sample_detector(self.det_offsets)]

    def apply(self, y) -> np.ndarray:
        return self.sample_weights() * y

    def white_level(self) -> np.ndarray:
        return self.sample_weights()


@dataclass
class SampleWeightNoise:
    """Diagonal N^-1 = W with its own weight w_t >= 0 for every sample: the
    general weighting of Eq. 4 with a diagonal W.  A weight of 0 takes the
    sample out of every sum (gap treatment)."""
    weights: np.ndarray  # [nsamples]

    def sample_weights(self) -> np.ndarray:
        return np.asarray(self.weights, np.float64)

    def apply(self, y) -> np.ndarray:
        return self.sample_weights() * y

    def white_level(self) -> np.ndarray:
        return self.sample_weights()


@dataclass
class OffsetFilterNoise:
    """White N^-1 (weight 1/sigma_d^2) with a baseline offset per interval
    marginalised out (a filtering template): W = Nk - Nk F (F^T Nk F)^+ F^T Nk,
    where F is the indicator matrix of the baseline intervals (each detector's
    samples cut into intervals of ``baseline_len``, the last one possibly
    shorter) and Nk is N^-1 restricted to the kept samples (``kept``, set by
    the System: flagged samples and samples of masked pixels do not enter the
    offset fit).  Written out: on a kept sample, (W y)_t = w_t (y_t - mean of
    y over the kept samples of its interval); 0 elsewhere."""
    inv_var: np.ndarray
    det_offsets: np.ndarray
    baseline_len: int
    kept: np.ndarray = None  # [nsamples] bool

    def with_kept(self, kept) -> "OffsetFilterNoise":
        return OffsetFilterNoise(self.inv_var, self.det_offsets, self.baseline_len, np.asarray(kept, bool))

    def white_level(self) -> np.ndarray:
        return np.asarray(self.inv_var, np.float64)[sample_detector(self.det_offsets)]

    def intervals(self):
        off = np.asarray(self.det_offsets, np.int64)
        for d in range(off.size - 1):
            for a in range(off[d], off[d + 1], self.baseline_len):
                yield a, min(a + self.baseline_len, off[d + 1])

    def apply(self, y) -> np.ndarray:
        y = np.asarray(y, np.float64)
        k = np.ones(y.size, bool) if self.kept is None else self.kept
        w = self.white_level()
        z = np.zeros_like(y)
        for a, e in self.intervals():
            kk = k[a:e]
            n = int(kk.sum())
            if n == 0:
                continue
            m = y[a:e][kk].sum() / n
            z[a:e] = np.where(kk, w[a:e] * (y[a:e] - m), 0.0)
        return z


@dataclass
class ToeplitzNoise:
    """Banded symmetric Toeplitz N^-1 per chunk of each detector's samples:
    z_t = c_0 y_t + sum_{k=1}^{L-1} c_k (y_{t-k} + y_{t+k}), with y taken as
    zero outside the chunk.  ``coeffs`` is [ndet][L]; ``white_inv_var`` is the
    per-detector diagonal used by the preconditioner (Eq. 7)."""
    coeffs: np.ndarray
    det_offsets: np.ndarray
    chunk_len: int
    white_inv_var: np.ndarray

    def apply(self, y) -> np.ndarray:
        y = np.asarray(y, np.float64)
        z = np.zeros_like(y)
        off = np.asarray(self.det_offsets, np.int64)
        for d in range(off.size - 1):
            c = np.asarray(self.coeffs[d], np.float64)
            kernel = np.concatenate([c[:0:-1], c])  # c_{L-1} .. c_1, c_0, c_1 .. c_{L-1}
            for a in range(off[d], off[d + 1], self.chunk_len):
                e = min(a + self.chunk_len, off[d + 1])
                z[a:e] = toeplitz_band_apply(y[a:e], kernel)
        return z

    def white_level(self) -> np.ndarray:
        return np.asarray(self.white_inv_var, np.float64)[sample_detector(self.det_offsets)]


def toeplitz_band_apply(y, kernel) -> np.ndarray:
    """Finite section of the band: np.convolve with the symmetric kernel of odd
    length 2L-1, keeping the outputs aligned with y (zero beyond the ends)."""
    L = (kernel.size + 1) // 2
    full = np.convolve(y, kernel)              # length n + 2L - 2
    return full[L - 1: L - 1 + y.size]


# ----------------------------------------------------------------------------
# Block-diagonal preconditioner (Eq. 7) and the pixel mask
# ----------------------------------------------------------------------------
def block_matrices(pix, v, w, npix: int) -> np.ndarray:
    """B_p = sum over samples t in p of w_t v_t v_t^T  (P^T diag(N)^-1 P, Eq. 7),
    over every non-flagged sample.  Shape [npix, ncomp, ncomp]."""
    pix = np.asarray(pix, np.int64)
    ok = pix >= 0
    ncomp = v.shape[1]
    B = np.zeros((npix, ncomp, ncomp))
    for i in range(ncomp):
        for j in range(ncomp):
            B[:, i, j] = np.bincount(pix[ok], weights=w[ok] * v[ok, i] * v[ok, j], minlength=npix)
    return B


def block_condition(B) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Eigenvalue extremes and condition number lambda_max / lambda_min of each
    symmetric block (inf where lambda_min <= 0)."""
    ev = np.linalg.eigvalsh(B)
    lmin, lmax = ev[:, 0], ev[:, -1]
    with np.errstate(divide="ignore", invalid="ignore"):
        cond = np.where(lmin > 0, lmax / np.where(lmin > 0, lmin, 1.0), np.inf)
    return lmin, lmax, cond


def pixel_mask(hit_count, B, min_hits: int, max_cond: float) -> np.ndarray:
    """True where a pixel is left out of the solve (see the module notes)."""
    ncomp = B.shape[1]
    lmin, _, cond = block_condition(B)
    bad = hit_count < min_hits
    if ncomp > 1:
        bad |= (lmin <= 0) | (cond > max_cond)
    else:
        bad |= B[:, 0, 0] <= 0
    return bad


def block_inverse(B, mask) -> np.ndarray:
    """M_p = B_p^-1 for kept pixels, 0 for masked ones."""
    M = np.zeros_like(B)
    keep = ~mask
    if np.any(keep):
        M[keep] = np.linalg.inv(B[keep])
    return M


def precond_apply(M, r) -> np.ndarray:
    """z_p = M_p r_p."""
    return np.einsum("pij,pj->pi", M, r)


# ----------------------------------------------------------------------------
# The GLS system (Eq. 5-6)
# ----------------------------------------------------------------------------
class System:
    """A = P^T N^-1 P on the kept pixels, with the preconditioner of Eq. 7."""

    def __init__(self, pix, psi, ncomp: int, npix: int, noise, min_hits: int = 3,
                 max_cond: float = 1e3, trig=None):
        """psi: polarisation angles; or trig = (cos 2psi, sin 2psi) given directly."""
        self.npix, self.ncomp, self.noise = npix, ncomp, noise
        self.pix = np.asarray(pix, np.int64)
        self.v = pointing_weights(psi, ncomp) if trig is None else pointing_weights_trig(*trig, ncomp)
        self.hits = hits(self.pix, npix)
        self.B = block_matrices(self.pix, self.v, noise.white_level(), npix)
        self.mask = pixel_mask(self.hits, self.B, min_hits, max_cond)
        self.M = block_inverse(self.B, self.mask)
        self.pe = effective_pixels(self.pix, self.mask)
        if hasattr(noise, "with_kept"):  # a weighting that depends on which samples enter the system
            self.noise = noise.with_kept(self.pe >= 0)

    def masked_tod(self, d) -> np.ndarray:
        """d with the samples of flagged or masked pixels set to zero."""
        d = np.asarray(d, np.float64).copy()
        d[self.pe < 0] = 0.0
        return d

    def rhs(self, d) -> np.ndarray:
        """b = P^T N^-1 d (Eq. 6)."""
        return apply_PT(self.pe, self.v, self.noise.apply(self.masked_tod(d)), self.npix)

    def matvec(self, x) -> np.ndarray:
        """A x = P^T N^-1 P x (Eq. 6)."""
        return apply_PT(self.pe, self.v, self.noise.apply(apply_P(self.pe, self.v, x)), self.npix)

    def precond(self, r) -> np.ndarray:
        return precond_apply(self.M, r)


@dataclass
class SolveInfo:
    iterations: int
    rel_residual: float       # ||b - A x|| / ||b||, recomputed at the end
    converged: bool


def pcg(system: System, b, tol: float, maxiter: int, x0=None) -> tuple[np.ndarray, SolveInfo]:
    """Preconditioned conjugate gradient for A x = b with M of Eq. 7.

    x0 = 0 (or given); r = b - A x0; z = M r; p = z; rho = r.z; then per
    iteration q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q, stop if
    ||r|| <= tol ||b||, z = M r, rho' = r.z, beta = rho'/rho, p = z + beta p."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    r = b - system.matvec(x) if x0 is not None else b.copy()
    bnorm = np.sqrt(np.sum(b * b))
    if bnorm == 0.0:
        return x, SolveInfo(0, 0.0, True)
    z = system.precond(r)
    p = z.copy()
    rho = np.sum(r * z)
    it = 0
    converged = np.sqrt(np.sum(r * r)) <= tol * bnorm
    while not converged and it < maxiter:
        q = system.matvec(p)
        alpha = rho / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if np.sqrt(np.sum(r * r)) <= tol * bnorm:
            converged = True
            break
        z = system.precond(r)
        rho_new = np.sum(r * z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    res = b - system.matvec(x)
    return x, SolveInfo(it, float(np.sqrt(np.sum(res * res)) / bnorm), converged)


def gls_map(system: System, d, tol: float = 1e-13, maxiter: int = 1000):
    """GLS map (Eq. 5) by PCG; masked pixels set to NaN."""
    x, info = pcg(system, system.rhs(d), tol, maxiter)
    out = x.copy()
    out[system.mask] = np.nan
    return out, info


# ----------------------------------------------------------------------------
# Dense forms for tiny problems
# ----------------------------------------------------------------------------
def dense_pointing(pe, v, npix: int) -> np.ndarray:
    """P as a dense Nt x (npix * ncomp) matrix, written row by row from Eq. 8."""
    nt, ncomp = v.shape
    P = np.zeros((nt, npix * ncomp))
    for t in range(nt):
        if pe[t] >= 0:
            for k in range(ncomp):
                P[t, pe[t] * ncomp + k] = v[t, k]
    return P


def dense_inv_noise(noise, nt: int) -> np.ndarray:
    """N^-1 as a dense Nt x Nt matrix (diagonal, or block-diagonal Toeplitz bands)."""
    if isinstance(noise, (WhiteNoise, SampleWeightNoise)):
        return np.diag(noise.sample_weights())
    Ni = np.zeros((nt, nt))
    off = np.asarray(noise.det_offsets, np.int64)
    for d in range(off.size - 1):
        c = noise.coeffs[d]
        L = c.size
        for a in range(off[d], off[d + 1], noise.chunk_len):
            e = min(a + noise.chunk_len, off[d + 1])
            for i in range(a, e):
                for j in range(max(a, i - L + 1), min(e, i + L)):
                    Ni[i, j] = c[abs(i - j)]
    return Ni


def dense_gls(system: System, d) -> np.ndarray:
    """(P^T N^-1 P)^-1 P^T N^-1 d on the kept pixels (Eq. 5) by a Cholesky
    factorisation of the dense A; masked pixels NaN."""
    nt = system.pix.size
    P = dense_pointing(system.pe, system.v, system.npix)
    Ni = dense_inv_noise(system.noise, nt)
    keep = np.repeat(~system.mask, system.ncomp)
    Pk = P[:, keep]
    A = Pk.T @ Ni @ Pk
    b = Pk.T @ (Ni @ system.masked_tod(d))
    L = np.linalg.cholesky(A)
    y = _forward_sub(L, b)
    xk = _backward_sub(L.T, y)
    x = np.full(system.npix * system.ncomp, np.nan)
    x[keep] = xk
    return x.reshape(system.npix, system.ncomp)


def _forward_sub(L, b):
    y = np.zeros_like(b)
    for i in range(b.size):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def _backward_sub(U, y):
    x = np.zeros_like(y)
    for i in range(y.size - 1, -1, -1):
        x[i] = (y[i] - U[i, i + 1:] @ x[i + 1:]) / U[i, i]
    return x


# ----------------------------------------------------------------------------
# Error metric
# ----------------------------------------------------------------------------
def rel_err(x, ref, mask) -> dict:
    """Relative L2 error over kept pixels, per Stokes component and jointly."""
    keep = ~np.asarray(mask, bool)
    xs, rs = np.asarray(x)[keep], np.asarray(ref)[keep]
    out = {}
    for k in range(xs.shape[1]):
        den = np.sqrt(np.sum(rs[:, k] ** 2))
        out[k] = float(np.sqrt(np.sum((xs[:, k] - rs[:, k]) ** 2)) / den) if den > 0 else 0.0
    den = np.sqrt(np.sum(rs ** 2))
    out["all"] = float(np.sqrt(np.sum((xs - rs) ** 2)) / den) if den > 0 else 0.0
    return out
