"""Parity of the CUDA library (through the C-ABI) with the FP64 oracle on the
same seeded inputs.  Tolerances: integers bit-exact; FP64 path <= 1e-10
relative L2 per Stokes component on kept pixels; refined mixed path <= 1e-6
(the map accuracy targets of the workloads); single operators in FP64 <= 1e-12."""
import math

import numpy as np
import pytest

import synth
from oracle import gls, healpix

from gpucase import Case, stokes_cols

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_2501_16122_gb300 as pkg
    pkg.build()
    from paper_2501_16122_gb300 import _lib
    return _lib


@pytest.fixture(scope="module")
def ctx(L):
    c = L.bm_context_create(0)
    yield c
    L.bm_context_destroy(c)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


# ------------------------------------------------------------- HEALPix (K9)

@pytest.mark.parametrize("nside", [1, 2, 16, 256, 512, 8192])
def test_ang2pix_bit_exact(L, ctx, nside):
    rng = np.random.default_rng(nside)
    n = 200_000
    z = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * math.pi, n)
    # plus pixel centres, ring boundaries, poles and the z = +-2/3 transition
    pc = np.arange(min(12 * nside * nside, 50_000))
    zc, phc = healpix.pix2ang_ring(nside, pc)
    z = np.concatenate([z, zc, [1.0, -1.0, 2 / 3, -2 / 3, 0.0, np.nextafter(2 / 3, 1)]])
    phi = np.concatenate([phi, phc, [0.0, 6.0, 1.0, 2.0, 0.0, 0.5]])
    d_pix = torch.empty(z.size, dtype=torch.int32, device="cuda")
    L.bm_ang2pix_ring(ctx, nside, torch.from_numpy(z).cuda(), torch.from_numpy(phi).cuda(), d_pix)
    assert np.array_equal(d_pix.cpu().numpy(), healpix.ang2pix_ring(nside, z, phi))


def test_ang2pix_on_a_scan(L, ctx):
    e = synth.make_experiment(256, 16, 50_000, 1001)
    pt = synth.pointing(e, with_angles=True)
    d_pix = torch.empty(e.nsamples, dtype=torch.int32, device="cuda")
    L.bm_ang2pix_ring(ctx, 256, torch.from_numpy(pt["z"]).cuda(), torch.from_numpy(pt["phi"]).cuda(), d_pix)
    assert np.array_equal(d_pix.cpu().numpy(), healpix.ang2pix_ring(256, pt["z"], pt["phi"]))


# ------------------------------------------------------- pointing and blocks

@pytest.mark.parametrize("solver", [3, 2, 1])
def test_pointing_operators_and_hits(L, ctx, solver):
    c = Case(L, ctx, 16, 4, 20_000, 2000 + solver, solver=solver, flag=0.02)
    try:
        hits = torch.zeros(c.npix, dtype=torch.int32, device="cuda")
        L.bm_pointing_get_hits(c.p, hits)
        assert np.array_equal(hits.cpu().numpy(), gls.hits(c.pix, c.npix))
        rng = np.random.default_rng(1)
        x = rng.normal(size=(c.npix, solver))
        y = torch.zeros(c.e.nsamples, dtype=torch.float64, device="cuda")
        L.bm_pointing_apply(c.p, c.vec(x), y)
        pe_all = np.where(c.pix >= 0, c.pix, -1)
        v = gls.pointing_weights(c.psi, solver)
        assert rel(y.cpu().numpy(), gls.apply_P(pe_all, v, x)) < 1e-13
        yt = rng.normal(size=c.e.nsamples)
        xt = c.vec()
        L.bm_pointing_apply_transpose(c.p, torch.from_numpy(yt).cuda(), xt)
        assert rel(xt.cpu().numpy(), gls.apply_PT(pe_all, v, yt, c.npix).ravel()) < 1e-13
    finally:
        c.close()


def stable_order(pix):
    """The kept samples' time indices sorted by pixel, ties in time order."""
    kept = np.flatnonzero(pix >= 0)
    return kept[np.argsort(pix[kept], kind="stable")]


@pytest.mark.parametrize("nside,n", [(256, 2_000_003),   # 20 bits: two 10-bit passes, 16-bit keys between
                                     (2048, 1_000_003),  # 26 bits: three 9-bit passes, 32-bit keys between
                                     (4096, 300_007)])   # 28 bits: three 10-bit passes, 32-bit keys between
def test_sort_order_is_the_stable_sort(L, ctx, nside, n):
    """The order every operator runs in is, exactly, the stable sort of the
    kept samples by pixel: ties (runs of one pixel, and hot pixels hit from
    many tiles and ranges) in time order, and pixels just below npix, whose
    high digits the flagged samples' key npix shares."""
    npix = 12 * nside * nside
    rng = np.random.default_rng(nside + 1)
    pix = rng.integers(0, npix, size=n).astype(np.int32)
    pix[1::3] = pix[0::3][: pix[1::3].size]
    hot = rng.random(n) < 0.2
    pix[hot] = rng.integers(0, 100, size=hot.sum()) * (npix // 100)
    top = rng.random(n) < 0.05
    pix[top] = npix - 1 - rng.integers(0, 64, size=top.sum())
    pix[rng.random(n) < 0.1] = -1
    psi = rng.uniform(0, np.pi, size=n)
    p = L.bm_pointing_create(ctx, npix, torch.from_numpy(pix).cuda(), torch.from_numpy(psi).cuda(), 3)
    try:
        order = L.bm_pointing_get_order(p).cpu().numpy().astype(np.int64)
        assert np.array_equal(order, stable_order(pix))
    finally:
        L.bm_pointing_destroy(p)


@pytest.mark.parametrize("nside,n,trig", [(8, 200_003, False),       # 10-bit keys: one sort pass
                                          (64, 3_000_001, True),     # 16 bits: two passes, many ranges
                                          (1024, 500_009, False)])   # 24 bits: three passes
def test_sort_plans_random_pixels(L, ctx, nside, n, trig):
    """The pixel sort behind P^T for every pass count, on random pixels with
    10 % flagged samples and a ragged last tile: hit counts bit-exact, P^T y
    and P x against the oracle's definition of Eq. 8."""
    npix = 12 * nside * nside
    rng = np.random.default_rng(nside)
    pix = rng.integers(0, npix, size=n).astype(np.int32)
    # runs of repeated pixels, as a scan produces
    pix[1::3] = pix[0::3][: pix[1::3].size]
    pix[rng.random(n) < 0.1] = -1
    psi = rng.uniform(0, np.pi, size=n)
    d_pix = torch.from_numpy(pix).cuda()
    if trig:
        c32, s32 = synth.trig32(psi)
        p = L.bm_pointing_create_trig(ctx, npix, d_pix, torch.from_numpy(c32).cuda(), torch.from_numpy(s32).cuda(), 3)
        v = gls.pointing_weights_trig(c32, s32, 3)
    else:
        p = L.bm_pointing_create(ctx, npix, d_pix, torch.from_numpy(psi).cuda(), 3)
        v = gls.pointing_weights(psi, 3)
    try:
        hits = torch.zeros(npix, dtype=torch.int32, device="cuda")
        L.bm_pointing_get_hits(p, hits)
        assert np.array_equal(hits.cpu().numpy(), gls.hits(pix, npix))
        assert np.array_equal(L.bm_pointing_get_order(p).cpu().numpy().astype(np.int64), stable_order(pix))
        y = rng.normal(size=n)
        xt = torch.zeros(npix * 3, dtype=torch.float64, device="cuda")
        L.bm_pointing_apply_transpose(p, torch.from_numpy(y).cuda(), xt)
        assert rel(xt.cpu().numpy(), gls.apply_PT(pix, v, y, npix).ravel()) < 1e-13
        x = rng.normal(size=(npix, 3))
        yy = torch.zeros(n, dtype=torch.float64, device="cuda")
        L.bm_pointing_apply(p, torch.from_numpy(x.ravel()).cuda(), yy)
        assert rel(yy.cpu().numpy(), gls.apply_P(pix, v, x)) < 1e-13
    finally:
        L.bm_pointing_destroy(p)


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_blocks_cond_mask(L, ctx, solver):
    c = Case(L, ctx, 16, 4, 65_536, 1000, solver=solver)
    try:
        S = c.S
        B = torch.zeros(c.npix * solver * solver, dtype=torch.float64, device="cuda")
        cond = torch.zeros(c.npix, dtype=torch.float64, device="cuda")
        L.bm_precond_get_blocks(c.pc, B, cond)
        B = B.cpu().numpy().reshape(c.npix, solver, solver)
        assert rel(B, S.B) < 1e-13
        _, _, ocond = gls.block_condition(S.B)
        # mask bit-exact outside a guard band around the threshold
        g = 1e-9
        band = np.isfinite(ocond) & (np.abs(ocond - 1e3) <= g * 1e3)
        m = c.mask()
        assert np.array_equal(m[~band], S.mask[~band]), np.nonzero(m != S.mask)
        assert band.sum() == 0
        fin = np.isfinite(ocond) & (ocond < 1e6)
        cg = cond.cpu().numpy()
        np.testing.assert_allclose(cg[fin], ocond[fin], rtol=1e-9)
        assert np.all(~np.isfinite(cg[~np.isfinite(ocond)]) | (cg[~np.isfinite(ocond)] > 1e12))
        # M r against the oracle's inverse blocks
        r = np.random.default_rng(2).normal(size=(c.npix, solver))
        z = c.vec()
        L.bm_precond_apply(c.pc, c.vec(r), z)
        assert rel(z.cpu().numpy(), S.precond(r).ravel()) < 1e-12
    finally:
        c.close()


def test_blocks_and_rhs_many_hits_per_pixel(L, ctx):
    # About 87,000 samples a pixel (nside 2, 4 det x 2^20 samples, exact FP32
    # trig pairs, ~2,700 samples a lane): the block sums and the RHS,
    # accumulated per lane in lazily renormalised double-float (a few 2^-48
    # of the running sum per term), stay within 1e-11 of the sum of the terms'
    # magnitudes; the mask is the oracle's and the FP64 map meets the 1e-10
    # bound.
    c = Case(L, ctx, 2, 4, 2 ** 20, 1100, trig=True, flag=0.01)
    try:
        S = c.S
        B = torch.zeros(c.npix * 9, dtype=torch.float64, device="cuda")
        L.bm_precond_get_blocks(c.pc, B, None)
        B = B.cpu().numpy().reshape(c.npix, 3, 3)
        # errors against the sum of the terms' magnitudes (entries like
        # sum w cos sin cancel): per pixel sum w, and sum w |d| for the RHS
        ok = S.pix >= 0
        w = S.noise.white_level()
        sw = np.bincount(S.pix[ok], weights=w[ok], minlength=c.npix)
        hit = sw > 0
        err = np.abs(B - S.B).max(axis=(1, 2))[hit] / sw[hit]
        assert err.max() < 1e-11, err.max()
        assert np.array_equal(c.mask(), S.mask)
        b = c.vec()
        L.bm_rhs(c.p, c.n, c.pc, c.d_tod, 1, b)
        ref = S.rhs(c.tod).reshape(c.npix, 3)
        got = b.cpu().numpy().reshape(c.npix, 3)
        keep = ~S.mask
        swd = np.bincount(S.pix[ok], weights=(w * np.abs(c.tod))[ok], minlength=c.npix)
        rerr = np.abs(got - ref).max(axis=1)[keep] / swd[keep]
        assert rerr.max() < 1e-11, rerr.max()
        out = c.vec()
        st, info = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-13, 50, L.BM_PREC_FP64)
        assert st == L.BM_OK, info
        x, _ = gls.gls_map(S, c.tod, tol=1e-14)
        e = gls.rel_err(out.cpu().numpy().reshape(c.npix, 3), x, S.mask)
        assert all(v <= 1e-10 for v in e.values()), e
    finally:
        c.close()


# --------------------------------------------------------------- operator A

@pytest.mark.parametrize("noise", ["white", "toeplitz"])
@pytest.mark.parametrize("solver", [3, 2, 1])
def test_matvec_and_rhs(L, ctx, noise, solver):
    kw = dict(chunk=8192, nlags=64) if noise == "toeplitz" else {}
    c = Case(L, ctx, 16, 4, 30_000 + 77, 3000 + solver, solver=solver, noise=noise, flag=0.01, **kw)
    try:
        S = c.S
        rng = np.random.default_rng(3)
        x = rng.normal(size=(c.npix, solver)) * np.array([100.0, 10.0, 10.0])[stokes_cols(solver)]
        ref = S.matvec(x * (~S.mask)[:, None])
        for prec, tol in ((L.BM_PREC_FP64, 1e-12), (L.BM_PREC_MIXED, 2e-6)):
            q = c.vec()
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), q, prec)
            qh = q.cpu().numpy().reshape(c.npix, solver)
            for k in range(solver):
                assert rel(qh[:, k], ref[:, k]) < tol, (prec, k, rel(qh[:, k], ref[:, k]))
            assert np.all(qh[S.mask] == 0)
        b = c.vec()
        L.bm_rhs(c.p, c.n, c.pc, c.d_tod, 1, b)
        bref = S.rhs(c.tod)
        assert rel(b.cpu().numpy(), bref.ravel()) < 1e-12
    finally:
        c.close()


def test_matvec_symmetric_and_deterministic(L, ctx):
    c = Case(L, ctx, 16, 4, 40_000, 77, noise="toeplitz", chunk=5000, nlags=128, build_oracle=False)
    try:
        m = c.mask()
        rng = np.random.default_rng(4)
        x = rng.normal(size=(c.npix, 3)) * (~m)[:, None]
        y = rng.normal(size=(c.npix, 3)) * (~m)[:, None]
        for prec in (L.BM_PREC_FP64, L.BM_PREC_MIXED):
            ax, ay, ax2 = c.vec(), c.vec(), c.vec()
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), ax, prec)
            L.bm_matvec(c.p, c.n, c.pc, c.vec(y), ay, prec)
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), ax2, prec)
            assert torch.equal(ax, ax2)  # bitwise reproducible
            a = float((c.vec(y) * ax).sum())
            b = float((c.vec(x) * ay).sum())
            tol = 1e-12 if prec == L.BM_PREC_FP64 else 1e-5
            assert abs(a - b) <= tol * (abs(a) + abs(b))
    finally:
        c.close()


def test_inv_noise_apply(L, ctx):
    e = synth.make_experiment(8, 3, 3000, 5)
    c = synth.toeplitz_band(e.sigma, 0.1, 1.0, 20.0, 4096, 100)
    N = gls.ToeplitzNoise(c, e.det_offsets, 700, 1 / e.sigma ** 2)
    n = L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, 700, c, 1 / e.sigma ** 2)
    y = np.random.default_rng(5).normal(size=e.nsamples)
    z = torch.zeros(e.nsamples, dtype=torch.float64, device="cuda")
    L.bm_inv_noise_apply(n, torch.from_numpy(y).cuda(), z)
    assert rel(z.cpu().numpy(), N.apply(y)) < 1e-13
    L.bm_inv_noise_destroy(n)
    W = gls.WhiteNoise(1 / e.sigma ** 2, e.det_offsets)
    n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
    L.bm_inv_noise_apply(n, torch.from_numpy(y).cuda(), z)
    assert rel(z.cpu().numpy(), W.apply(y)) < 1e-15
    L.bm_inv_noise_destroy(n)


# ------------------------------------------------------------------- solves

def check_map(L, c, out, ref_x, tol):
    m = c.mask()
    xh = out.cpu().numpy().reshape(c.npix, c.nc)
    assert np.array_equal(np.isnan(xh).any(axis=1), m)
    err = gls.rel_err(xh, ref_x, m)
    assert all(v <= tol for v in err.values()), err
    return err


def test_config0_fp64_and_mixed(L, ctx):
    # nside 16, 4 detectors x 65536 samples, FP64, white noise, tol 1e-10.
    c = Case(L, ctx, 16, 4, 65_536, 1000)
    try:
        ref, info = gls.gls_map(c.S, c.tod, tol=1e-13)
        for prec, tol in ((L.BM_PREC_FP64, 1e-10), (L.BM_PREC_MIXED, 1e-10)):
            out = c.vec()
            st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-10, 100, prec)
            assert st == L.BM_OK, infos
            assert infos[0]["rel_residual"] <= 1e-10
            check_map(L, c, out, ref, tol)
        # white noise: one PCG iteration in the FP64 path
        out = c.vec()
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-10, 100, L.BM_PREC_FP64)
        assert infos[0]["iterations"] == 1
    finally:
        c.close()


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_toeplitz_solve(L, ctx, solver):
    c = Case(L, ctx, 8, 4, 2 ** 14 + 123, 4000 + solver, solver=solver, noise="toeplitz", chunk=4096,
             nlags=256, flag=0.01)
    try:
        ref, info = gls.gls_map(c.S, c.tod, tol=1e-13, maxiter=2000)
        assert info.converged
        out = c.vec()
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-12, 2000, L.BM_PREC_FP64)
        assert st == L.BM_OK, infos
        check_map(L, c, out, ref, 1e-10)
        out = c.vec()
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-8, 2000, L.BM_PREC_MIXED)
        assert st == L.BM_OK, infos
        assert infos[0]["outer_iterations"] >= 1
        check_map(L, c, out, ref, 1e-6)
    finally:
        c.close()


def test_noiseless_recovery_fp32_inputs(L, ctx):
    # FP32 TOD and FP32 psi (configs 1-3 store them so): x = s to the
    # precision of the stored TOD values.
    c = Case(L, ctx, 32, 16, 8192, 1001, tod_dtype=np.float32, psi_dtype=np.float32, noiseless=True,
             noise="toeplitz", chunk=2048, nlags=512)
    try:
        out = c.vec()
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-9, 3000, L.BM_PREC_MIXED)
        assert st == L.BM_OK, infos
        ref, _ = gls.gls_map(c.S, c.tod.astype(np.float64), tol=1e-13, maxiter=3000)
        check_map(L, c, out, ref, 1e-6)
        # and the oracle's map equals the input sky up to FP32 TOD rounding
        err = gls.rel_err(ref, c.sky, c.S.mask)
        assert err["all"] < 1e-5
    finally:
        c.close()


@pytest.mark.parametrize("solver,R", [(3, 5), (3, 40), (3, 70), (2, 3), (1, 3)])
def test_batched_multi_rhs(L, ctx, solver, R):
    # R realisations (sky + white noise) sharing one pointing, solved as one
    # batched mixed-precision PCG: every map matches the oracle and the
    # one-at-a-time solve, and the batched solve is bitwise reproducible.
    c = Case(L, ctx, 16, 4, 16_384 + 5, 11 + solver, solver=solver, tod_dtype=np.float32, trig=True)
    try:
        tods = []
        for r in range(R):
            sky = synth.sky_map(c.npix, 100 + r)
            if solver == 2:
                sky[:, 0] = 0
            if solver == 1:
                sky[:, 1:] = 0
            tods.append(synth.tod(c.e, c.pix, c.psi, sky, solver=solver, noise_seed=500 + r,
                                  dtype=np.float32, trig=c.trig))
        d = torch.from_numpy(np.stack(tods)).cuda()
        nv = c.npix * solver
        out = torch.zeros(R * nv, dtype=torch.float64, device="cuda")
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, d, R, out, 1e-10, 50, L.BM_PREC_MIXED)
        assert st == L.BM_OK, infos
        out2 = torch.zeros_like(out)
        L.bm_pcg_solve(c.p, c.n, c.pc, d, R, out2, 1e-10, 50, L.BM_PREC_MIXED)
        assert torch.equal(torch.nan_to_num(out), torch.nan_to_num(out2))
        for r in (0, R // 2, R - 1):
            ref, _ = gls.gls_map(c.S, tods[r].astype(np.float64), tol=1e-13)
            check_map(L, c, out[r * nv:(r + 1) * nv], ref, 1e-9)
            one = c.vec()
            st1, _ = L.bm_pcg_solve(c.p, c.n, c.pc, d[r].contiguous(), 1, one, 1e-10, 50, L.BM_PREC_MIXED)
            a, b = one.cpu().numpy(), out[r * nv:(r + 1) * nv].cpu().numpy()
            keep = ~np.isnan(a)
            assert np.array_equal(keep, ~np.isnan(b))
            assert rel(b[keep], a[keep]) < 1e-9
    finally:
        c.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_multi_rhs_toeplitz(L, ctx, prec):
    # Three correlated-noise realisations (sky + 1/f noise through a 48-lag
    # band) sharing one pointing, in one call: each map matches the oracle's
    # GLS map of its TOD and the same RHS solved alone, bitwise.
    c = Case(L, ctx, 8, 4, 8192 + 13, 37, noise="toeplitz", chunk=2048, nlags=48, psi_dtype=np.float64)
    try:
        R = 3
        tods = [c.tod]
        for r in range(1, R):
            extra = synth.one_over_f_noise(c.e, 2048, 0.1, 1.0, seed=700 + r)
            tods.append(synth.tod(c.e, c.pix, c.psi, synth.sky_map(c.npix, 200 + r), white=False, extra=extra,
                                  dtype=np.float64))
        d = torch.from_numpy(np.stack(tods)).cuda()
        nv = c.npix * 3
        out = torch.zeros(R * nv, dtype=torch.float64, device="cuda")
        tol = 1e-12 if prec == 0 else 1e-10
        st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, d, R, out, tol, 500, prec)
        assert st == L.BM_OK, infos
        for r in range(R):
            ref, _ = gls.gls_map(c.S, tods[r], tol=1e-13)
            check_map(L, c, out[r * nv:(r + 1) * nv], ref, 1e-10 if prec == 0 else 1e-6)
            one = c.vec()
            L.bm_pcg_solve(c.p, c.n, c.pc, d[r].contiguous(), 1, one, tol, 500, prec)
            assert torch.equal(torch.nan_to_num(one), torch.nan_to_num(out[r * nv:(r + 1) * nv]))
    finally:
        c.close()


# --------------------------------------------------------------- edge cases

def test_invalid_pixel_rejected(L, ctx):
    pix = torch.tensor([0, 1, 5, 12], dtype=torch.int32, device="cuda")  # 12 >= npix
    psi = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(L.BrahmapError) as ei:
        L.bm_pointing_create(ctx, 12, pix, psi, 3)
    assert ei.value.status == L.BM_ERR_INVALID
    pix = torch.tensor([0, -2], dtype=torch.int32, device="cuda")
    with pytest.raises(L.BrahmapError):
        L.bm_pointing_create(ctx, 12, pix, psi[:2], 3)


def test_all_flagged_and_tiny(L, ctx):
    pix = torch.full((7,), -1, dtype=torch.int32, device="cuda")
    psi = torch.zeros(7, dtype=torch.float64, device="cuda")
    p = L.bm_pointing_create(ctx, 12, pix, psi, 3)
    n = L.bm_inv_noise_create_diag(ctx, np.array([0, 7]), np.array([1.0]))
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    out = torch.zeros(36, dtype=torch.float64, device="cuda")
    st, infos = L.bm_pcg_solve(p, n, pc, torch.ones(7, dtype=torch.float64, device="cuda"), 1, out, 1e-8, 10)
    assert st == L.BM_OK and infos[0]["rel_residual"] == 0.0
    assert torch.isnan(out).all()
    for h in (pc, n, p):
        (L.bm_precond_destroy if h is pc else L.bm_inv_noise_destroy if h is n else L.bm_pointing_destroy)(h)
    # a single sample
    p = L.bm_pointing_create(ctx, 12, torch.tensor([3], dtype=torch.int32, device="cuda"),
                             torch.zeros(1, dtype=torch.float64, device="cuda"), 1)
    n = L.bm_inv_noise_create_diag(ctx, np.array([0, 1]), np.array([4.0]))
    pc = L.bm_blockdiag_precond_create(p, n, 1, 1e3)
    out = torch.zeros(12, dtype=torch.float64, device="cuda")
    st, infos = L.bm_pcg_solve(p, n, pc, torch.tensor([2.5], dtype=torch.float64, device="cuda"), 1, out,
                               1e-12, 10)
    assert st == L.BM_OK and out[3].item() == 2.5
    L.bm_precond_destroy(pc)
    L.bm_inv_noise_destroy(n)
    L.bm_pointing_destroy(p)


def test_bad_arguments(L, ctx):
    e = synth.make_experiment(4, 2, 100, 1)
    with pytest.raises(L.BrahmapError):
        L.bm_inv_noise_create_diag(ctx, np.array([0, 50, 40]), np.array([1.0, 1.0]))
    with pytest.raises(L.BrahmapError):
        L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, 10, np.zeros((2, 2000)), np.ones(2))
    with pytest.raises(L.BrahmapError):
        L.bm_inv_noise_create_diag(ctx, e.det_offsets, np.array([1.0, -1.0]))


# ------------------------------------------------ precomputed FP32 trig input

@pytest.mark.parametrize("noise", ["white", "toeplitz"])
def test_trig_input_blocks_matvec_rhs(L, ctx, noise):
    kw = dict(chunk=4096, nlags=128) if noise == "toeplitz" else {}
    c = Case(L, ctx, 16, 4, 40_000, 6100, noise=noise, tod_dtype=np.float32, trig=True, flag=0.01, **kw)
    try:
        S = c.S
        B = torch.zeros(c.npix * 9, dtype=torch.float64, device="cuda")
        L.bm_precond_get_blocks(c.pc, B, None)
        assert rel(B.cpu().numpy().reshape(c.npix, 3, 3), S.B) < 1e-13
        assert np.array_equal(c.mask(), S.mask)
        x = np.random.default_rng(7).normal(size=(c.npix, 3)) * np.array([100.0, 10.0, 10.0])
        ref = S.matvec(x * (~S.mask)[:, None])
        for prec, tol in ((L.BM_PREC_FP64, 1e-12), (L.BM_PREC_MIXED, 2e-6)):
            q = c.vec()
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), q, prec)
            qh = q.cpu().numpy().reshape(c.npix, 3)
            for k in range(3):
                assert rel(qh[:, k], ref[:, k]) < tol, (prec, k)
        b = c.vec()
        L.bm_rhs(c.p, c.n, c.pc, c.d_tod, 1, b)
        assert rel(b.cpu().numpy(), S.rhs(c.tod.astype(np.float64)).ravel()) < 1e-12
    finally:
        c.close()


def test_trig_input_alignment_and_host_memory(L, ctx):
    """Given cos/sin in device memory at 16-byte boundaries, the first sort
    pass reads them itself and writes the time-ordered pairs; off a boundary
    or in host memory the validation pass does.  Every form gives the same
    handle: the order, P x over the time-ordered pairs and P^T y bitwise
    equal.  A cos or sin outside [-1, 1] (or NaN) is refused in every form."""
    nside, n = 16, 300_001
    npix = 12 * nside * nside
    rng = np.random.default_rng(77)
    pix = rng.integers(0, npix, size=n).astype(np.int32)
    pix[rng.random(n) < 0.05] = -1
    c32, s32 = synth.trig32(rng.uniform(0, np.pi, size=n))
    y = torch.from_numpy(rng.normal(size=n)).cuda()
    x = torch.from_numpy(rng.normal(size=npix * 3)).cuda()

    def forms(c, s):
        dc, ds = torch.from_numpy(c).cuda(), torch.from_numpy(s).cuda()
        oc, os_ = torch.zeros(n + 1, dtype=torch.float32, device="cuda"), torch.zeros(n + 1, dtype=torch.float32,
                                                                                     device="cuda")
        oc[1:], os_[1:] = dc, ds
        assert oc[1:].data_ptr() % 16 != 0
        return {"aligned": (dc, ds), "offset": (oc[1:], os_[1:]),
                "host": (torch.from_numpy(c).pin_memory(), torch.from_numpy(s).pin_memory())}

    d_pix = torch.from_numpy(pix).cuda()
    got = {}
    for name, (c, s_) in forms(c32, s32).items():
        p = L.bm_pointing_create_trig(ctx, npix, d_pix, c, s_, 3)
        try:
            yy = torch.zeros(n, dtype=torch.float64, device="cuda")
            L.bm_pointing_apply(p, x, yy)
            xt = torch.zeros(npix * 3, dtype=torch.float64, device="cuda")
            L.bm_pointing_apply_transpose(p, y, xt)
            got[name] = (L.bm_pointing_get_order(p).cpu().numpy(), yy.cpu().numpy(), xt.cpu().numpy())
        finally:
            L.bm_pointing_destroy(p)
    for name in ("offset", "host"):
        for a, b in zip(got["aligned"], got[name]):
            assert np.array_equal(np.nan_to_num(a), np.nan_to_num(b)), name
    v = gls.pointing_weights_trig(c32, s32, 3)
    assert rel(got["aligned"][1], gls.apply_P(pix, v, x.cpu().numpy().reshape(npix, 3))) < 1e-13
    for bad in (1.5, np.nan):
        cb = c32.copy()
        cb[n // 3] = bad
        for name, (c, s_) in forms(cb, s32).items():
            with pytest.raises(L.BrahmapError) as ei:
                L.bm_pointing_create_trig(ctx, npix, d_pix, c, s_, 3)
            assert ei.value.status == L.BM_ERR_INVALID and "trig value" in str(ei.value), (bad, name)


def test_trig_input_config1_like_solve(L, ctx):
    # The config-1 input format (int32 pix, FP32 cos/sin, FP32 TOD, white
    # noise) on a reduced scan: mixed solve to 1e-8 matches the oracle to 1e-6,
    # and the FP64 path to 1e-10.
    c = Case(L, ctx, 64, 16, 65_536, 1001, tod_dtype=np.float32, trig=True)
    try:
        ref, _ = gls.gls_map(c.S, c.tod.astype(np.float64), tol=1e-13)
        for prec, tol_solve, tol_err in ((L.BM_PREC_MIXED, 1e-8, 1e-6), (L.BM_PREC_FP64, 1e-10, 1e-10)):
            out = c.vec()
            st, infos = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, tol_solve, 100, prec)
            assert st == L.BM_OK, infos
            check_map(L, c, out, ref, tol_err)
    finally:
        c.close()


def test_pinned_host_inputs_match_device_inputs(L, ctx):
    """Page-locked host pix / trig / TOD go through the same computation as
    device arrays: hits, P^T y and the solved map are bitwise equal."""
    c = Case(L, ctx, 16, 4, 40_000, 4242, flag=0.01, trig=True, tod_dtype=np.float32, build_oracle=False)
    try:
        c32, s32 = c.trig
        dev = L.bm_pointing_create_trig(ctx, c.npix, c.d_pix, torch.from_numpy(c32).cuda(),
                                        torch.from_numpy(s32).cuda(), 3)
        host = L.bm_pointing_create_trig(ctx, c.npix, torch.from_numpy(c.pix).pin_memory(),
                                         torch.from_numpy(c32).pin_memory(), torch.from_numpy(s32).pin_memory(), 3)
        with pytest.raises(Exception):  # pageable host memory is refused
            L.bm_pointing_create_trig(ctx, c.npix, torch.from_numpy(c.pix), torch.from_numpy(c32),
                                      torch.from_numpy(s32), 3)
        try:
            h1 = torch.zeros(c.npix, dtype=torch.int32, device="cuda")
            h2 = torch.zeros_like(h1)
            L.bm_pointing_get_hits(dev, h1)
            L.bm_pointing_get_hits(host, h2)
            assert torch.equal(h1, h2)
            y = torch.randn(c.e.nsamples, dtype=torch.float64, device="cuda")
            x1 = torch.zeros(c.npix * 3, dtype=torch.float64, device="cuda")
            x2 = torch.zeros_like(x1)
            L.bm_pointing_apply_transpose(dev, y, x1)
            L.bm_pointing_apply_transpose(host, y, x2)
            assert torch.equal(x1, x2)
            n = L.bm_inv_noise_create_diag(ctx, c.e.det_offsets, 1.0 / c.e.sigma ** 2)
            pc1 = L.bm_blockdiag_precond_create(dev, n, 3, 1e3)
            pc2 = L.bm_blockdiag_precond_create(host, n, 3, 1e3)
            m1 = torch.zeros(c.npix * 3, dtype=torch.float64, device="cuda")
            m2 = torch.zeros_like(m1)
            L.bm_pcg_solve(dev, n, pc1, c.d_tod, 1, m1, 1e-8, 100, L.BM_PREC_MIXED)
            L.bm_pcg_solve(host, n, pc2, torch.from_numpy(c.tod).pin_memory(), 1, m2, 1e-8, 100, L.BM_PREC_MIXED)
            assert torch.equal(torch.nan_to_num(m1, 7.0), torch.nan_to_num(m2, 7.0))
            L.bm_precond_destroy(pc1)
            L.bm_precond_destroy(pc2)
            L.bm_inv_noise_destroy(n)
        finally:
            L.bm_pointing_destroy(dev)
            L.bm_pointing_destroy(host)
    finally:
        c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_detector_lengths(L, ctx, prec):
    """Detectors of different lengths (the offsets' binary search; equal
    lengths take the t / ns path): blocks, RHS, matvec and the solve against
    the oracle."""
    e = synth.make_experiment(16, 4, 20_000, 515)
    pt = synth.pointing(e, flag_frac=0.01)
    det_off = np.array([0, 7_000, 29_000, 29_001, 80_000], np.int64)
    inv_var = np.array([1.0, 0.4, 2.5, 0.7])
    sky = synth.sky_map(e.npix, 515)
    tod = synth.tod(e, pt["pix"], pt["psi"], sky, white=False)
    tod = tod + np.random.default_rng(5).normal(size=tod.size) / np.sqrt(inv_var[gls.sample_detector(det_off)])
    S = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.WhiteNoise(inv_var, det_off))
    p = L.bm_pointing_create(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(pt["psi"]).cuda(), 3)
    n = L.bm_inv_noise_create_diag(ctx, det_off, inv_var)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    try:
        P = L.BM_PREC_FP64 if prec == "fp64" else L.BM_PREC_MIXED
        x = np.random.default_rng(6).normal(size=(e.npix, 3))
        q = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
        L.bm_matvec(p, n, pc, torch.from_numpy(x.ravel()).cuda(), q, P)
        ref = S.matvec(x * (~S.mask)[:, None])
        assert rel(q.cpu().numpy(), ref.ravel()) < (1e-12 if prec == "fp64" else 2e-6)
        out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
        st, _ = L.bm_pcg_solve(p, n, pc, torch.from_numpy(tod).cuda(), 1, out, 1e-11, 200, P)
        assert st == L.BM_OK
        oref, _ = gls.gls_map(S, tod, tol=1e-13)
        err = gls.rel_err(out.cpu().numpy().reshape(e.npix, 3), oref, S.mask)
        assert max(err.values()) < (1e-10 if prec == "fp64" else 1e-6), err
    finally:
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)


@pytest.mark.parametrize("prec", [0, 1])
def test_graphs_on_and_off_same_bits(L, ctx, prec):
    """The PCG iterations as a CUDA graph (the default) and driven from the
    host (bm_context_set_graphs(ctx, 0)) run the same kernels in the same
    order: Toeplitz solves (single RHS) and a batched white-noise solve give
    the same maps bit for bit."""
    c = Case(L, ctx, 8, 4, 8192 + 13, 41, noise="toeplitz", chunk=2048, nlags=48, psi_dtype=np.float64,
             build_oracle=False)
    w = Case(L, ctx, 8, 4, 6000, 42, build_oracle=False)
    try:
        tol = 1e-12 if prec == 0 else 1e-10
        d = torch.from_numpy(np.stack([w.tod, w.tod[::-1].copy(), 0.5 * w.tod])).cuda()
        maps = []
        for graphs in (True, False):
            L.bm_context_set_graphs(ctx, graphs)
            one = c.vec()
            st, info = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, one, tol, 500, prec)
            assert st == L.BM_OK and info[0]["iterations"] > 1, info
            many = torch.zeros(3 * w.npix * 3, dtype=torch.float64, device="cuda")
            st, infos = L.bm_pcg_solve(w.p, w.n, w.pc, d, 3, many, 1e-10, 500, L.BM_PREC_MIXED)
            assert st == L.BM_OK, infos
            maps.append((one, many))
        for a, b in zip(maps[0], maps[1]):
            assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))
    finally:
        L.bm_context_set_graphs(ctx, True)
        c.close()
        w.close()
