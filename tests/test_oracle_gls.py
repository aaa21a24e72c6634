"""Pins of the oracle's GLS pieces against closed forms, the dense definition,
a direct solve, invariants and statistics (none of them re-derives the
oracle's own code path)."""
import math

import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import gls


def make_case(nside, ndet, ns, seed, solver=3, flag=0.0, noise="white", chunk=None,
              nlags=None, fknee=0.1, min_hits=None, max_cond=1e3):
    e = synth.make_experiment(nside, ndet, ns, seed)
    pt = synth.pointing(e, flag_frac=flag)
    if noise == "white":
        N = gls.WhiteNoise(1.0 / e.sigma ** 2, e.det_offsets)
    else:
        c = synth.toeplitz_band(e.sigma, fknee, 1.0, 20.0, max(chunk, 2 * nlags), nlags)
        N = gls.ToeplitzNoise(c, e.det_offsets, chunk, 1.0 / e.sigma ** 2)
    mh = {3: 3, 2: 2, 1: 1}[solver] if min_hits is None else min_hits
    S = gls.System(pt["pix"], pt["psi"], solver, e.npix, N, min_hits=mh, max_cond=max_cond)
    return e, pt, S


# ---------------------------------------------------------------- pointing

@pytest.mark.parametrize("solver", [1, 2, 3])
def test_pointing_rows_follow_eq8(solver):
    e, pt, S = make_case(2, 2, 150, 3, solver=solver, flag=0.05)
    P = gls.dense_pointing(S.pe, S.v, e.npix)
    for t in range(P.shape[0]):
        nz = np.nonzero(P[t])[0]
        if S.pe[t] < 0:
            assert nz.size == 0
            continue
        p = S.pe[t]
        a = 2 * pt["psi"][t]
        row = {3: [1.0, math.cos(a), math.sin(a)], 2: [math.cos(a), math.sin(a)], 1: [1.0]}[solver]
        np.testing.assert_allclose(P[t, p * solver:(p + 1) * solver], row, rtol=0, atol=1e-15)
        assert set(nz) <= set(range(p * solver, (p + 1) * solver))
    rng = np.random.default_rng(0)
    x = rng.normal(size=(e.npix, solver))
    y = rng.normal(size=P.shape[0])
    np.testing.assert_allclose(gls.apply_P(S.pe, S.v, x), P @ x.ravel(), atol=1e-12)
    np.testing.assert_allclose(gls.apply_PT(S.pe, S.v, y, e.npix).ravel(), P.T @ y, atol=1e-12)


# ------------------------------------------------------------ preconditioner

def test_block_hand_example():
    rows = read_golden("block_hand_example.txt")
    cs = np.array([[float(r[0]), float(r[1])] for r in rows if r[0] not in ("B", "M")])
    B_ref = np.array([float(x) for x in next(r for r in rows if r[0] == "B")[1:]]).reshape(3, 3)
    M_ref = np.array([float(x) for x in next(r for r in rows if r[0] == "M")[1:]]).reshape(3, 3)
    v = np.column_stack([np.ones(len(cs)), cs])
    B = gls.block_matrices(np.zeros(len(cs), np.int64), v, np.ones(len(cs)), 1)
    assert np.array_equal(B[0], B_ref)
    M = gls.block_inverse(B, np.array([False]))
    np.testing.assert_allclose(M[0], M_ref, atol=1e-15)


@pytest.mark.parametrize("solver", [1, 2, 3])
def test_blocks_are_the_diagonal_of_dense_PtWP(solver):
    e, pt, S = make_case(2, 3, 200, 4, solver=solver, flag=0.05)
    pe_all = np.where(S.pix >= 0, S.pix, -1)
    P = gls.dense_pointing(pe_all, S.v, e.npix)
    W = np.diag(S.noise.white_level())
    D = P.T @ W @ P
    n = solver
    for p in range(e.npix):
        np.testing.assert_allclose(D[p * n:(p + 1) * n, p * n:(p + 1) * n], S.B[p], atol=1e-12)
        off = D[p * n:(p + 1) * n].copy()
        off[:, p * n:(p + 1) * n] = 0
        assert np.all(off == 0)  # block-diagonal (Eq. 7 discussion)


def test_condition_number_known_spectrum():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    B = np.stack([Q @ np.diag([1.0, 2.0, 4.0]) @ Q.T, np.diag([3.0, 3.0, 3.0]),
                  np.diag([1.0, 0.0, 2.0]), np.diag([1.0, -1.0, 2.0])])
    lmin, lmax, cond = gls.block_condition(B)
    np.testing.assert_allclose(cond[:2], [4.0, 1.0], rtol=1e-13)
    assert np.isinf(cond[2]) and np.isinf(cond[3])


def test_mask_rule():
    B = np.stack([np.diag([1000.0, 1.0, 1.0]), np.diag([1000.0 * (1 + 1e-12), 1.0, 1.0]),
                  np.eye(3), np.eye(3), np.diag([1.0, 0.0, 1.0])])
    h = np.array([5, 5, 3, 2, 9])
    mask = gls.pixel_mask(h, B, 3, 1e3)
    # cond exactly 1e3 kept (strict), above masked, hits 2 < 3 masked, singular masked
    assert mask.tolist() == [False, True, False, True, True]
    Bi = np.array([[[2.0]], [[0.0]], [[1.0]]])
    assert gls.pixel_mask(np.array([1, 4, 0]), Bi, 1, 1e3).tolist() == [False, True, True]


# ------------------------------------------------------------------- system A

@pytest.mark.parametrize("noise", ["white", "toeplitz"])
def test_A_symmetric_positive(noise):
    e, pt, S = make_case(4, 4, 2000, 5, noise=noise, chunk=300, nlags=24, flag=0.02)
    rng = np.random.default_rng(3)
    keep = ~S.mask
    for _ in range(3):
        x = rng.normal(size=(e.npix, 3)) * keep[:, None]
        y = rng.normal(size=(e.npix, 3)) * keep[:, None]
        a, b = np.sum(x * S.matvec(y)), np.sum(y * S.matvec(x))
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
        assert np.sum(x * S.matvec(x)) > 0
    assert np.all(S.matvec(np.ones((e.npix, 3)))[S.mask] == 0)


@pytest.mark.parametrize("solver", [1, 2, 3])
@pytest.mark.parametrize("noise", ["white", "toeplitz"])
def test_pcg_agrees_with_dense_cholesky(solver, noise):
    e, pt, S = make_case(2, 3, 600, 6 + solver, solver=solver, noise=noise, chunk=128, nlags=16,
                         flag=0.03)
    sky = synth.sky_map(e.npix, 6)[:, {3: [0, 1, 2], 2: [1, 2], 1: [0]}[solver]]
    full = np.zeros((e.npix, 3))
    full[:, {3: [0, 1, 2], 2: [1, 2], 1: [0]}[solver]] = sky
    d = synth.tod(e, pt["pix"], pt["psi"], full, solver=solver)
    x_dense = gls.dense_gls(S, d)
    x, info = gls.gls_map(S, d, tol=1e-14, maxiter=500)
    keep = ~S.mask
    assert keep.sum() > 3
    err = np.max(np.abs(x[keep] - x_dense[keep])) / np.max(np.abs(x_dense[keep]))
    assert err < 1e-12, err
    assert np.all(np.isnan(x[S.mask]))


def test_dense_solve_of_tiny_case_against_numpy_solve():
    e, pt, S = make_case(1, 2, 400, 11)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 11))
    keep = np.repeat(~S.mask, 3)
    P = gls.dense_pointing(S.pe, S.v, e.npix)[:, keep]
    Ni = gls.dense_inv_noise(S.noise, P.shape[0])
    ref = np.linalg.solve(P.T @ Ni @ P, P.T @ Ni @ S.masked_tod(d))
    np.testing.assert_allclose(gls.dense_gls(S, d).ravel()[keep], ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("solver", [1, 2, 3])
@pytest.mark.parametrize("noise", ["white", "toeplitz"])
def test_noiseless_recovery(solver, noise):
    # d = P s exactly  =>  x = s on every kept pixel, for any SPD N^-1 (Eq. 4-5).
    e, pt, S = make_case(8, 4, 20_000, 20 + solver, solver=solver, noise=noise, chunk=4096,
                         nlags=64, flag=0.01)
    cols = {3: [0, 1, 2], 2: [1, 2], 1: [0]}[solver]
    full = synth.sky_map(e.npix, 21)
    if solver == 2:
        full[:, 0] = 0
    if solver == 1:
        full[:, 1:] = 0
    d = synth.tod(e, pt["pix"], pt["psi"], full, solver=solver, white=False)
    x, info = gls.gls_map(S, d, tol=1e-14, maxiter=1000)
    assert info.converged
    err = gls.rel_err(x, full[:, cols], S.mask)
    assert all(v < 1e-11 for v in err.values()), err


def test_white_noise_converges_in_one_iteration():
    # For diagonal N^-1, A is itself the block-diagonal matrix of Eq. 7, so
    # M = A^-1 and PCG from x = 0 finishes after one step with x = M b.
    e, pt, S = make_case(16, 4, 65_536, 1000)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 1000))
    b = S.rhs(d)
    x, info = gls.pcg(S, b, tol=1e-10, maxiter=10)
    assert info.iterations == 1 and info.rel_residual < 1e-13
    np.testing.assert_allclose(x, S.precond(b), rtol=1e-12, atol=1e-12)


def test_white_noise_chi_square():
    # (x - s)^T A (x - s) ~ chi^2 with one degree of freedom per kept unknown.
    e, pt, S = make_case(16, 4, 65_536, 1000)
    sky = synth.sky_map(e.npix, 1000)
    d = synth.tod(e, pt["pix"], pt["psi"], sky)
    x, info = gls.pcg(S, S.rhs(d), tol=1e-12, maxiter=10)
    r = (x - sky) * (~S.mask)[:, None]
    chi2 = np.sum(r * S.matvec(r))
    dof = 3 * int((~S.mask).sum())
    assert abs(chi2 - dof) < 5 * math.sqrt(2 * dof), (chi2, dof)


# ------------------------------------------------------------------- Toeplitz

def test_toeplitz_band_against_double_loop_and_fft():
    rng = np.random.default_rng(4)
    L, n = 7, 40
    c = rng.normal(size=L)
    y = rng.normal(size=n)
    kernel = np.concatenate([c[:0:-1], c])
    z = gls.toeplitz_band_apply(y, kernel)
    ref = np.zeros(n)
    for t in range(n):
        for s in range(n):
            if abs(t - s) < L:
                ref[t] += c[abs(t - s)] * y[s]
    np.testing.assert_allclose(z, ref, atol=1e-13)
    m = n + 2 * L
    fz = np.fft.irfft(np.fft.rfft(y, m) * np.fft.rfft(kernel, m), m)[L - 1:L - 1 + n]
    np.testing.assert_allclose(z, fz, atol=1e-12)


def test_toeplitz_chunks_do_not_couple():
    c = np.array([[2.0, 0.5, 0.25]])
    N = gls.ToeplitzNoise(c, np.array([0, 10]), 4, np.array([1.0]))
    y = np.zeros(10)
    y[3] = 1.0  # last sample of chunk 0
    z = N.apply(y)
    assert z[4] == 0 and z[5] == 0  # chunk 1 sees nothing
    assert z.tolist()[:4] == [0.0, 0.25, 0.5, 2.0]


def test_toeplitz_section_is_spd():
    e = synth.make_experiment(4, 2, 512, 7)
    c = synth.toeplitz_band(e.sigma, 0.1, 1.0, 20.0, 4096, 64)
    N = gls.ToeplitzNoise(c, e.det_offsets, 300, 1 / e.sigma ** 2)
    D = gls.dense_inv_noise(N, e.nsamples)
    assert np.allclose(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0


# -------------------------------------------------------- planted mistakes

def test_planted_angle_mistake_breaks_recovery(monkeypatch):
    orig = gls.pointing_weights
    monkeypatch.setattr(gls, "pointing_weights", lambda psi, n: orig(np.asarray(psi) / 2, n))
    e, pt, S = make_case(8, 4, 20_000, 31)
    sky = synth.sky_map(e.npix, 31)
    d = synth.tod(e, pt["pix"], pt["psi"], sky, white=False)
    x, _ = gls.gls_map(S, d, tol=1e-14, maxiter=100)
    assert gls.rel_err(x, sky, S.mask)["all"] > 1e-3


def test_planted_transpose_mistake_breaks_dense_block_check(monkeypatch):
    def wrong(pix, v, w, npix):
        ok = pix >= 0
        n = v.shape[1]
        B = np.zeros((npix, n, n))
        for i in range(n):
            for j in range(n):
                B[:, i, j] = np.bincount(pix[ok], weights=w[ok] * v[ok, i] * v[ok, i], minlength=npix)
        return B
    e, pt, S = make_case(2, 3, 200, 4)
    W = np.diag(S.noise.white_level())
    P = gls.dense_pointing(np.where(S.pix >= 0, S.pix, -1), S.v, e.npix)
    D = P.T @ W @ P
    Bw = wrong(S.pix, S.v, S.noise.white_level(), e.npix)
    assert not all(np.allclose(D[3 * p:3 * p + 3, 3 * p:3 * p + 3], Bw[p]) for p in range(e.npix))


def test_planted_dropped_noise_term_is_caught():
    # Dropping N^-1 from the matvec (a plausible slip) changes the solution,
    # and the dense Cholesky solve of Eq. 5 catches it.
    e, pt, S = make_case(2, 3, 600, 8, noise="toeplitz", chunk=128, nlags=16)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 8))

    class Wrong(gls.System):
        def matvec(self, x):
            return gls.apply_PT(self.pe, self.v, gls.apply_P(self.pe, self.v, x), self.npix)
    W = Wrong.__new__(Wrong)
    W.__dict__.update(S.__dict__)
    x, info = gls.gls_map(W, d, tol=1e-14, maxiter=200)
    ref = gls.dense_gls(S, d)
    keep = ~S.mask
    assert not np.allclose(x[keep], ref[keep], rtol=1e-6)


def test_precomputed_trig_rows_and_recovery():
    # Rows built from given (cos 2psi, sin 2psi) equal the angle form when the
    # given values are the FP64 trig; with FP32-rounded values the system is
    # the operator of those numbers, and noiseless data made with the same
    # numbers is recovered exactly.
    e = synth.make_experiment(8, 4, 20_000, 41)
    pt = synth.pointing(e)
    a = 2 * pt["psi"]
    assert np.array_equal(gls.pointing_weights_trig(np.cos(a), np.sin(a), 3), gls.pointing_weights(pt["psi"], 3))
    c32, s32 = synth.trig32(pt["psi"])
    assert c32.dtype == np.float32 and np.array_equal(c32, np.cos(a).astype(np.float32))
    S = gls.System(pt["pix"], None, 3, e.npix, gls.WhiteNoise(1 / e.sigma ** 2, e.det_offsets), trig=(c32, s32))
    sky = synth.sky_map(e.npix, 41)
    d = synth.tod(e, pt["pix"], pt["psi"], sky, white=False, trig=(c32, s32))
    x, info = gls.gls_map(S, d, tol=1e-14)
    assert gls.rel_err(x, sky, S.mask)["all"] < 1e-12


# ------------------------------------------------ per-sample weights (Eq. 4)

def test_sample_weights_equal_per_detector_weights():
    # W = diag(w_t) with w_t = 1/sigma_d^2 of the sample's detector is the
    # white-noise N^-1: same blocks, mask, operator, RHS and map.
    e, pt, S = make_case(8, 4, 8000, 41, flag=0.02)
    w = (1.0 / e.sigma ** 2)[np.repeat(np.arange(e.ndet), e.ns)]
    S2 = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.SampleWeightNoise(w), min_hits=3, max_cond=1e3)
    assert np.array_equal(S.B, S2.B) and np.array_equal(S.mask, S2.mask)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 41))
    np.testing.assert_array_equal(S.rhs(d), S2.rhs(d))
    x1, _ = gls.gls_map(S, d)
    x2, _ = gls.gls_map(S2, d)
    np.testing.assert_array_equal(np.nan_to_num(x1), np.nan_to_num(x2))


def test_zero_weights_are_gaps():
    # A weight of 0 takes a sample out of every sum: the map equals the one
    # with those samples flagged (on the pixels both keep; the hit counts,
    # hence min_hits, still see the zero-weight samples).
    e, pt, S = make_case(8, 4, 8000, 42)
    rng = np.random.default_rng(42)
    gap = rng.random(e.nsamples) < 0.15
    w = (1.0 / e.sigma ** 2)[np.repeat(np.arange(e.ndet), e.ns)] * rng.uniform(0.5, 2.0, e.nsamples)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 42))
    Sg = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.SampleWeightNoise(np.where(gap, 0.0, w)), min_hits=3,
                    max_cond=1e3)
    pix_f = np.where(gap, -1, pt["pix"])
    Sf = gls.System(pix_f, pt["psi"], 3, e.npix, gls.SampleWeightNoise(w), min_hits=3, max_cond=1e3)
    np.testing.assert_allclose(Sg.B, Sf.B, rtol=0, atol=1e-9 * np.abs(Sf.B).max())
    xg, _ = gls.gls_map(Sg, d, tol=1e-13)
    xf, _ = gls.gls_map(Sf, d, tol=1e-13)
    both = ~Sg.mask & ~Sf.mask
    assert both.sum() > 100
    np.testing.assert_allclose(xg[both], xf[both], rtol=1e-9, atol=1e-9 * np.abs(xf[both]).max())


def test_sample_weights_dense_definition():
    # Eq. 4 with a diagonal W, against the dense solve of P^T W P x = P^T W d.
    e, pt, S = make_case(1, 2, 400, 43)
    w = np.random.default_rng(43).uniform(0.0, 3.0, e.nsamples)
    S2 = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.SampleWeightNoise(w), min_hits=3, max_cond=1e3)
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 43))
    keep = np.repeat(~S2.mask, 3)
    P = gls.dense_pointing(S2.pe, S2.v, e.npix)[:, keep]
    W = np.diag(w)
    ref = np.linalg.solve(P.T @ W @ P, P.T @ W @ S2.masked_tod(d))
    x, _ = gls.gls_map(S2, d, tol=1e-14)
    np.testing.assert_allclose(x.ravel()[keep], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


# ------------------------------------------- baseline-offset template (Eq. 4)

def _offset_case(seed, baseline_len, flag=0.02):
    e = synth.make_experiment(8, 4, 6000, seed)
    pt = synth.pointing(e, flag_frac=flag)
    N = gls.OffsetFilterNoise(1.0 / e.sigma ** 2, e.det_offsets, baseline_len)
    S = gls.System(pt["pix"], pt["psi"], 3, e.npix, N, min_hits=3, max_cond=1e3)
    return e, pt, S


def test_offset_filter_is_the_marginalised_projector():
    # W = Nk - Nk F (F^T Nk F)^+ F^T Nk written out densely on a small case.
    e, pt, S = _offset_case(51, 700)
    n = S.noise
    nt = e.nsamples
    F = np.zeros((nt, sum(1 for _ in n.intervals())))
    for j, (a, b) in enumerate(n.intervals()):
        F[a:b, j] = 1.0
    Nk = np.diag(n.white_level() * n.kept)
    W = Nk - Nk @ F @ np.linalg.pinv(F.T @ Nk @ F) @ F.T @ Nk
    rng = np.random.default_rng(51)
    for _ in range(3):
        y = rng.normal(size=nt)
        np.testing.assert_allclose(n.apply(y), W @ y, rtol=1e-10, atol=1e-10 * np.abs(W @ y).max())
    # interval-constant vectors are annihilated; W is symmetric
    a = rng.normal(size=F.shape[1])
    assert np.abs(n.apply(F @ a)).max() < 1e-12 * np.abs(a).max() * n.white_level().max()
    x, y = rng.normal(size=nt), rng.normal(size=nt)
    assert abs(x @ n.apply(y) - y @ n.apply(x)) < 1e-10 * abs(x @ n.apply(y))


def test_offset_filter_removes_offsets_from_the_map():
    # d = P s + F a: the GLS map with the offsets marginalised recovers s on
    # the kept pixels, Q and U exactly and I up to its monopole (a constant I
    # map is an offset on every interval, hence in the null space of A).
    e, pt, S = _offset_case(52, 500)
    sky = synth.sky_map(e.npix, 52)
    d = synth.tod(e, pt["pix"], pt["psi"], sky, white=False)
    rng = np.random.default_rng(52)
    for a, b in S.noise.intervals():
        d[a:b] += rng.normal(0.0, 300.0)
    x, info = gls.gls_map(S, d, tol=1e-12, maxiter=3000)
    assert info.converged, info
    keep = ~S.mask
    assert keep.sum() > 100
    for k in (1, 2):
        np.testing.assert_allclose(x[keep, k], sky[keep, k], rtol=0, atol=1e-8 * np.abs(sky[keep, k]).max())
    di = (x[keep, 0] - x[keep, 0].mean()) - (sky[keep, 0] - sky[keep, 0].mean())
    assert np.abs(di).max() < 1e-8 * np.abs(sky[keep, 0]).max()


def test_offset_filter_special_cases():
    # closed forms of W = Nk - Nk F (F^T Nk F)^+ F^T Nk on ragged detectors
    off = np.array([0, 7, 20, 21, 40])
    iv = np.array([0.5, 1.0, 2.0, 4.0])
    rng = np.random.default_rng(61)
    y = rng.normal(size=40) + 3.0
    w = iv[gls.sample_detector(off)]
    # a baseline as long as the longest detector: each detector's mean removed
    z = gls.OffsetFilterNoise(iv, off, 40).apply(y)
    ref = np.concatenate([w[a:b] * (y[a:b] - y[a:b].mean()) for a, b in zip(off[:-1], off[1:])])
    np.testing.assert_allclose(z, ref, rtol=1e-13, atol=1e-13)
    # a baseline of one sample: every sample is its own offset, W = 0
    assert np.all(gls.OffsetFilterNoise(iv, off, 1).apply(y) == 0.0)
    # samples that are not kept neither receive a value nor enter any mean
    kept = np.ones(40, bool)
    kept[8:12] = False                                 # detector 1's intervals (baseline 5): [7, 12) keeps 7 only,
    kept[12:17] = False                                # [12, 17) keeps none
    n = gls.OffsetFilterNoise(iv, off, 5).with_kept(kept)
    y2 = y.copy()
    y2[~kept] = rng.normal(size=(~kept).sum()) * 1e3
    z1, z2 = n.apply(y), n.apply(y2)
    assert np.all(z1[~kept] == 0.0)
    np.testing.assert_array_equal(z1, z2)
    a, b = 7, 12                                       # the interval [7, 12): kept samples 7 only
    np.testing.assert_allclose(z1[a:b][kept[a:b]], 0.0, atol=1e-15)


# ---------------------------------------------------------------- HWP angles
def test_hwp_angles_without_rotation_are_the_detector_angles():
    """nu = 0: every sample of detector d has theta = psi_d + 2 phi0."""
    off = np.array([0, 7, 20, 21])
    psi_d = np.array([0.1, 2.0, 3.0])
    th = gls.hwp_angles(off, psi_d, 0.0, 0.25)
    for d in range(3):
        assert np.all(th[off[d]:off[d + 1]] == psi_d[d] + 0.5)


def test_hwp_angles_quarter_turn_per_sample():
    """nu = 1/4 (exact in binary): phi_hwp advances by pi/2 a sample, theta by
    pi, so theta(k) - theta(0) = pi (k mod 4) and cos 2 theta is constant."""
    off = np.array([0, 1001])
    th = gls.hwp_angles(off, [0.3], 0.25, 0.1)
    k = np.arange(1001)
    np.testing.assert_allclose(th - th[0], np.pi * (k % 4), rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.cos(2 * th), np.cos(2 * th[0]), rtol=0, atol=1e-13)


def test_hwp_angles_against_the_closed_form_and_the_scan_generator():
    """nu = 1 Hz / 20 Hz: near the start the unreduced closed form
    psi_d + 2 (2 pi nu k + phi0) is exact to FP64 rounding (equal angles up
    to whole turns, so equal cos 2 theta and sin 2 theta), and over a whole
    detector the seeded scan generator's angles (C, theta reduced with fmod in
    FP64, a separate implementation) give the same cos 2 theta, sin 2 theta."""
    import synth
    e = synth.make_experiment(8, 3, 40_000, 77)
    nu = e.scan.hwp_hz / e.scan.fsamp
    th = gls.hwp_angles(e.det_offsets, e.psi_det, nu, e.hwp_phase0)
    k = np.arange(2000)
    for d in range(3):
        naive = e.psi_det[d] + 2.0 * (2.0 * np.pi * nu * k + e.hwp_phase0)
        for f in (np.cos, np.sin):
            np.testing.assert_allclose(f(2 * th[d * e.ns + k]), f(2 * naive), rtol=0, atol=1e-11)
    psi = synth.pointing(e)["psi"]
    np.testing.assert_allclose(np.cos(2 * th), np.cos(2 * psi), rtol=0, atol=1e-10)
    np.testing.assert_allclose(np.sin(2 * th), np.sin(2 * psi), rtol=0, atol=1e-10)


def test_hwp_angles_stay_exact_far_from_the_start():
    """The phase is reduced exactly: with nu = 1/20 the angle repeats every 20
    samples even 2^31 samples in (where nu k ~ 1e8 turns and the unreduced
    FP64 product has lost ~1e-8 of a turn)."""
    nu = 1.0 / 20.0
    from fractions import Fraction
    k0 = 2 ** 31
    fr = Fraction(nu)
    # the oracle's exact reduction at a large k equals its value at k mod 20
    # up to the (tiny) difference between the binary nu and 1/20
    assert abs(float((fr * k0) % 1) - float((fr * (k0 % 20)) % 1)) < 1e-6
    th = gls.hwp_angles(np.array([0, 40]), [0.0], nu, 0.0)
    np.testing.assert_allclose(th[20:40], th[0:20], rtol=0, atol=1e-12)
