"""Parity at the full workload sizes, in the launch configuration bench.py
times, on outputs the FP64 oracle can compute one pixel at a time:

  * config 1 (nside 256, 256 det x 2^22 samples, FP32 trig and TOD, white
    noise): hit counts for every pixel (bit-exact) and the solved map on
    sampled pixels -- for white noise the GLS system decouples per pixel, so
    the oracle solves each sampled pixel from its own samples;
  * config 2 (same scan, 512-lag Toeplitz noise per 2^20-sample chunk): the
    FP64 matvec on sampled pixels (each needs only +-511-sample windows
    around its samples), and exact recovery of the sky from noiseless TOD;
  * config 3 (nside 512, 64 det x 2^22 samples, 64 right-hand sides): every
    right-hand side's map on sampled pixels;
  * the offset template on config 2's scan: the operators on sampled pixels
    (each needs only the baselines its samples fall in), the I monopole in the
    null space, symmetry, and the solve of a sky plus baseline offsets.
"""
import gc

import numpy as np
import pytest

import synth
from oracle import gls

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    import paper_2501_16122_gb300 as pkg
    pkg.build()
    from paper_2501_16122_gb300 import _lib
    return _lib


@pytest.fixture
def ctx(L):
    c = L.bm_context_create(0)
    yield c
    L.bm_context_destroy(c)
    gc.collect()
    torch.cuda.empty_cache()


def sampled_pixels(hits, mask, rng, n=24):
    kept = np.nonzero(~mask)[0]
    hk = hits[kept]
    picks = list(rng.choice(kept, n - 4, replace=False))
    picks += [kept[np.argmin(hk)], kept[np.argmax(hk)]]          # fewest / most hits
    picks += [kept[0], kept[-1]]                                   # ring ends
    return np.unique(np.asarray(picks))


def select_samples(pix, npix, pixels):
    lut = np.zeros(npix, bool)
    lut[pixels] = True
    return np.nonzero(lut[np.where(pix >= 0, pix, 0)] & (pix >= 0))[0]


def oracle_white_pixels(e, pix, c32, s32, idx, tod_rows, pixels):
    """GLS maps of the sampled pixels from their own samples (white noise):
    idx = the samples falling in those pixels, tod_rows = TOD values at idx."""
    sub_pix = pix[idx].astype(np.int64)
    w = (1.0 / e.sigma ** 2)[idx // e.ns]
    v = gls.pointing_weights_trig(c32[idx], s32[idx], 3)
    B = gls.block_matrices(sub_pix, v, w, e.npix)[pixels]
    hits = np.bincount(sub_pix, minlength=e.npix)[pixels]
    mask = gls.pixel_mask(hits, B, 3, 1e3)
    Minv = gls.block_inverse(B, mask)
    out = []
    for d in tod_rows:
        dv = np.asarray(d, np.float64)
        b = np.stack([np.bincount(sub_pix, weights=w * dv * v[:, j], minlength=e.npix)[pixels] for j in range(3)],
                     axis=1)
        out.append(gls.precond_apply(Minv, b))
    return out, mask


def test_config1_full_size(L, ctx):
    e = synth.make_experiment(256, 256, 2 ** 22, 1001)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    tod = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 1001), dtype=np.float32, trig=(c32, s32))
    d_pix = torch.from_numpy(pt["pix"]).cuda()
    p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, torch.from_numpy(c32).cuda(), torch.from_numpy(s32).cuda(), 3)
    n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    st, info = L.bm_pcg_solve(p, n, pc, torch.from_numpy(tod).cuda(), 1, out, 1e-8, 200, L.BM_PREC_MIXED)
    assert st == L.BM_OK and info[0]["rel_residual"] <= 1e-8
    hits = torch.zeros(e.npix, dtype=torch.int32, device="cuda")
    mask = torch.zeros(e.npix, dtype=torch.uint8, device="cuda")
    L.bm_precond_get_mask(pc, mask, hits)
    hits, mask = hits.cpu().numpy(), mask.cpu().numpy().astype(bool)
    assert np.array_equal(hits, np.bincount(pt["pix"], minlength=e.npix))  # every pixel, bit-exact
    pixels = sampled_pixels(hits, mask, np.random.default_rng(0))
    idx = select_samples(pt["pix"], e.npix, pixels)
    (ref,), omask = oracle_white_pixels(e, pt["pix"], c32, s32, idx, [tod[idx]], pixels)
    assert np.array_equal(omask, mask[pixels])
    xg = out.cpu().numpy().reshape(e.npix, 3)[pixels]
    for k in range(3):
        err = np.linalg.norm(xg[:, k] - ref[:, k]) / np.linalg.norm(ref[:, k])
        assert err < 1e-6, (k, err)
    for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
        f(h)
    del d_pix
    gc.collect()
    torch.cuda.empty_cache()

    # The benchmarked path itself: pix, the trig pair and the TOD given as
    # page-locked host buffers, the TOD carried through the pixel sort and
    # read in sorted order by the RHS (the bench's end-to-end step).  Same
    # values summed in the same order: the map must equal the one above bit
    # for bit, and so meet the oracle on the sampled pixels.
    h_pix = torch.from_numpy(pt["pix"]).pin_memory()
    h_c, h_s = torch.from_numpy(c32).pin_memory(), torch.from_numpy(s32).pin_memory()
    h_tod = torch.from_numpy(tod).pin_memory()
    p2 = L.bm_pointing_create_with_tod(ctx, e.npix, h_pix, h_tod, cos2psi=h_c, sin2psi=h_s)
    n2 = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
    pc2 = L.bm_blockdiag_precond_create(p2, n2, 3, 1e3)
    out2 = torch.full_like(out, float("nan"))
    st2, info2 = L.bm_pcg_solve(p2, n2, pc2, None, 1, out2, 1e-8, 200, L.BM_PREC_MIXED)
    assert st2 == L.BM_OK and info2[0]["rel_residual"] <= 1e-8
    a, b = out.cpu().numpy(), out2.cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    x2 = b.reshape(e.npix, 3)[pixels]
    for k in range(3):
        assert np.linalg.norm(x2[:, k] - ref[:, k]) / np.linalg.norm(ref[:, k]) < 1e-6
    for h, f in ((pc2, L.bm_precond_destroy), (n2, L.bm_inv_noise_destroy), (p2, L.bm_pointing_destroy)):
        f(h)


def oracle_toeplitz_matvec_pixels(e, pix, c32, s32, coeffs, chunk, mask, x, pixels):
    """(P^T N^-1 P x)_p for the sampled pixels with the banded Toeplitz N^-1:
    each sample's filtered value needs only the window of +-(L-1) samples of
    its chunk around it."""
    Lg = coeffs.shape[1]
    idx = select_samples(pix, e.npix, pixels)
    keep_pix = np.where((pix >= 0) & ~mask[np.where(pix >= 0, pix, 0)], pix, -1)
    q = np.zeros((len(pixels), 3))
    where = {p: i for i, p in enumerate(pixels)}
    for t in idx:
        pt_ = keep_pix[t]
        if pt_ < 0:
            continue
        d = t // e.ns
        cs = d * e.ns + ((t - d * e.ns) // chunk) * chunk
        ce = min(cs + chunk, (d + 1) * e.ns)
        a, b = max(cs, t - (Lg - 1)), min(ce, t + Lg)
        win = np.arange(a, b)
        v = gls.pointing_weights_trig(c32[win], s32[win], 3)
        y = gls.apply_P(keep_pix[win], v, x)
        z = np.dot(coeffs[d][np.abs(win - t)], y)  # z_t = sum_t' c_|t - t'| y_t' within the chunk
        q[where[pt_]] += z * gls.pointing_weights_trig(c32[t:t + 1], s32[t:t + 1], 3)[0]
    return q


def test_config2_full_size(L, ctx):
    e = synth.make_experiment(256, 256, 2 ** 22, 1002)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    sky = synth.sky_map(e.npix, 1002)
    tod = synth.tod(e, pt["pix"], pt["psi"], sky, white=False, dtype=np.float64, trig=(c32, s32))  # noiseless
    chunk = 2 ** 20
    coeffs = synth.toeplitz_band(e.sigma, 0.1, 1.0, 20.0, chunk, 512)
    p = L.bm_pointing_create_trig(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(c32).cuda(),
                                  torch.from_numpy(s32).cuda(), 3)
    n = L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, chunk, coeffs, 1 / e.sigma ** 2)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    mask = torch.zeros(e.npix, dtype=torch.uint8, device="cuda")
    hits = torch.zeros(e.npix, dtype=torch.int32, device="cuda")
    L.bm_precond_get_mask(pc, mask, hits)
    mask_h, hits_h = mask.cpu().numpy().astype(bool), hits.cpu().numpy()
    # FP64 matvec on sampled pixels against the oracle's windowed evaluation
    rng = np.random.default_rng(1)
    x = rng.normal(size=(e.npix, 3)) * np.array([100.0, 10.0, 10.0])
    q = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    L.bm_matvec(p, n, pc, torch.from_numpy(x.ravel()).cuda(), q, L.BM_PREC_FP64)
    pixels = sampled_pixels(hits_h, mask_h, rng, n=6)
    ref = oracle_toeplitz_matvec_pixels(e, pt["pix"], c32, s32, coeffs, chunk, mask_h, x * (~mask_h)[:, None], pixels)
    qg = q.cpu().numpy().reshape(e.npix, 3)[pixels]
    assert np.linalg.norm(qg - ref) / np.linalg.norm(ref) < 1e-10
    # noiseless TOD: the mixed solve recovers the sky on every kept pixel
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    st, info = L.bm_pcg_solve(p, n, pc, torch.from_numpy(tod).cuda(), 1, out, 1e-9, 3000, L.BM_PREC_MIXED)
    assert st == L.BM_OK, info
    err = gls.rel_err(out.cpu().numpy().reshape(e.npix, 3), sky, mask_h)
    assert all(v < 1e-6 for v in err.values()), err
    for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
        f(h)


def test_toeplitz_mixed_matvec_over_time_chunks(L, ctx):
    """The mixed-precision Toeplitz matvec, whose transpose runs one time chunk
    of 2^24 samples at a time, over three chunks with a ragged last one
    (8 det x (2^22 + 4097) samples): against the oracle's windowed evaluation
    on sampled pixels (the FP32 operator's tolerance), next to the FP64 path."""
    e = synth.make_experiment(64, 8, 2 ** 22 + 4097, 1404)
    pt = synth.pointing(e, flag_frac=0.01)
    c32, s32 = synth.trig32(pt["psi"])
    chunk = 2 ** 20
    coeffs = synth.toeplitz_band(e.sigma, 0.1, 1.0, 20.0, chunk, 128)
    p = L.bm_pointing_create_trig(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(c32).cuda(),
                                  torch.from_numpy(s32).cuda(), 3)
    n = L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, chunk, coeffs, 1 / e.sigma ** 2)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    mask = torch.zeros(e.npix, dtype=torch.uint8, device="cuda")
    hits = torch.zeros(e.npix, dtype=torch.int32, device="cuda")
    L.bm_precond_get_mask(pc, mask, hits)
    mask_h, hits_h = mask.cpu().numpy().astype(bool), hits.cpu().numpy()
    rng = np.random.default_rng(2)
    x = rng.normal(size=(e.npix, 3)) * np.array([100.0, 10.0, 10.0])
    pixels = sampled_pixels(hits_h, mask_h, rng, n=10)
    ref = oracle_toeplitz_matvec_pixels(e, pt["pix"], c32, s32, coeffs, chunk, mask_h, x * (~mask_h)[:, None], pixels)
    for prec, tol in ((L.BM_PREC_FP64, 1e-10), (L.BM_PREC_MIXED, 2e-6)):
        q = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
        L.bm_matvec(p, n, pc, torch.from_numpy(x.ravel()).cuda(), q, prec)
        qh = q.cpu().numpy().reshape(e.npix, 3)
        for k in range(3):
            err = np.linalg.norm(qh[pixels, k] - ref[:, k]) / np.linalg.norm(ref[:, k])
            assert err < tol, (prec, k, err)
        assert np.all(qh[mask_h] == 0)
        if prec == L.BM_PREC_MIXED:  # deterministic: a second call gives the same bits
            q2 = torch.zeros_like(q)
            L.bm_matvec(p, n, pc, torch.from_numpy(x.ravel()).cuda(), q2, prec)
            assert torch.equal(q, q2)
    for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
        f(h)


def oracle_offset_matvec_pixels(e, pix, c32, s32, bl, mask, x, pixels):
    """(P^T W P x)_p for the sampled pixels with the baseline-offset W: each
    sample t of p contributes w_d v_t (y_t - m_I), m_I the mean of y = P x
    over the kept samples of t's interval I, so only the intervals the
    sampled pixels touch are evaluated (all their samples)."""
    idx = select_samples(pix, e.npix, pixels)
    keep_pix = np.where((pix >= 0) & ~mask[np.where(pix >= 0, pix, 0)], pix, -1)
    idx = idx[keep_pix[idx] >= 0]
    d = idx // e.ns
    ipd = -(-e.ns // bl)                                   # intervals per detector
    I = d * ipd + (idx - d * e.ns) // bl
    m = {}
    for j in np.unique(I):
        dd, k = divmod(int(j), ipd)
        a = dd * e.ns + k * bl
        win = np.arange(a, min(a + bl, (dd + 1) * e.ns))
        kp = keep_pix[win]
        v = gls.pointing_weights_trig(c32[win], s32[win], 3)
        y = gls.apply_P(kp, v, x)                          # 0 on samples that are not kept
        m[int(j)] = y.sum() / max(int((kp >= 0).sum()), 1)
    w = 1.0 / e.sigma ** 2
    v = gls.pointing_weights_trig(c32[idx], s32[idx], 3)
    y = gls.apply_P(keep_pix[idx], v, x)
    z = w[d] * (y - np.array([m[int(j)] for j in I]))
    where = {p: i for i, p in enumerate(pixels)}
    q = np.zeros((len(pixels), 3))
    np.add.at(q, np.array([where[p] for p in keep_pix[idx]]), z[:, None] * v)
    return q


def test_offsets_full_size(L, ctx):
    """The offset template at the bench's size (config 2's scan, 1.07e9
    samples, 1200-sample baselines): the FP64 and mixed operators on sampled
    pixels against the oracle's evaluation; the I monopole in the null space
    and the symmetry of the operator (properties at any size); and a mixed
    solve of a noiseless sky plus a random offset per baseline, which gives
    back Q and U and the I map up to its monopole."""
    e = synth.make_experiment(256, 256, 2 ** 22, 1002)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    bl = 1200
    p = L.bm_pointing_create_trig(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(c32).cuda(),
                                  torch.from_numpy(s32).cuda(), 3)
    n = L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, 1 / e.sigma ** 2, bl)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    mask = torch.zeros(e.npix, dtype=torch.uint8, device="cuda")
    hits = torch.zeros(e.npix, dtype=torch.int32, device="cuda")
    L.bm_precond_get_mask(pc, mask, hits)
    mask_h, hits_h = mask.cpu().numpy().astype(bool), hits.cpu().numpy()
    rng = np.random.default_rng(3)
    x = rng.normal(size=(e.npix, 3)) * np.array([100.0, 10.0, 10.0])
    xm = x * (~mask_h)[:, None]
    pixels = sampled_pixels(hits_h, mask_h, rng, n=6)
    ref = oracle_offset_matvec_pixels(e, pt["pix"], c32, s32, bl, mask_h, xm, pixels)

    def mv(vec, prec):
        q = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
        L.bm_matvec(p, n, pc, torch.from_numpy(np.ascontiguousarray(vec).ravel()).cuda(), q, prec)
        return q.cpu().numpy().reshape(e.npix, 3)

    for prec, tol in ((L.BM_PREC_FP64, 1e-10), (L.BM_PREC_MIXED, 2e-6)):
        qh = mv(x, prec)
        for k in range(3):
            err = np.linalg.norm(qh[pixels, k] - ref[:, k]) / np.linalg.norm(ref[:, k])
            assert err < tol, (prec, k, err)
        assert np.all(qh[mask_h] == 0)
        # a constant I map is an offset on every baseline: A maps it to ~0
        one = np.zeros((e.npix, 3))
        one[:, 0] = 1.0
        B1 = np.linalg.norm(hits_h[~mask_h] / e.sigma.min() ** 2)
        assert np.linalg.norm(mv(one, prec)) < (1e-12 if prec == L.BM_PREC_FP64 else 1e-6) * B1
    y2 = rng.normal(size=(e.npix, 3)) * np.array([100.0, 10.0, 10.0]) * (~mask_h)[:, None]
    a, b = np.sum(xm * mv(y2, L.BM_PREC_FP64)), np.sum(y2 * mv(xm, L.BM_PREC_FP64))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))
    # noiseless sky + offsets: the mixed solve recovers the sky up to the I monopole
    sky = synth.sky_map(e.npix, 1002)
    tod = synth.tod(e, pt["pix"], pt["psi"], sky, white=False, dtype=np.float64, trig=(c32, s32))
    ipd = -(-e.ns // bl)
    off = rng.normal(0.0, 30.0, (e.ndet, ipd))
    tod += np.repeat(off, bl, axis=1)[:, :e.ns].ravel()
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    st, info = L.bm_pcg_solve(p, n, pc, torch.from_numpy(tod).cuda(), 1, out, 1e-9, 3000, L.BM_PREC_MIXED)
    assert st == L.BM_OK, info
    got = out.cpu().numpy().reshape(e.npix, 3)
    keep = ~mask_h
    got[keep, 0] -= got[keep, 0].mean()
    sky = sky.copy()
    sky[keep, 0] -= sky[keep, 0].mean()
    err = gls.rel_err(got, sky, mask_h)
    assert all(v < 1e-6 for v in err.values()), err
    for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
        f(h)


def test_config3_full_size(L, ctx):
    e = synth.make_experiment(512, 64, 2 ** 22, 1003)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    d_pix = torch.from_numpy(pt["pix"]).cuda()
    d_c, d_s = torch.from_numpy(c32).cuda(), torch.from_numpy(s32).cuda()
    R = 64
    # TOD of 64 realisations synthesised on the device (signal of a seeded sky
    # gathered at each sample's pixel + white noise from a seeded generator)
    gen = torch.Generator(device="cuda").manual_seed(1003)
    tod = torch.empty((R, e.nsamples), dtype=torch.float32, device="cuda")
    sig = torch.from_numpy(np.repeat(e.sigma, e.ns).astype(np.float32)).cuda()
    pl = d_pix.long()
    for r in range(R):
        sky = torch.randn((e.npix, 3), generator=gen, device="cuda", dtype=torch.float64) * \
            torch.tensor([100.0, 10.0, 10.0], device="cuda", dtype=torch.float64)
        tod[r] = (sky[pl, 0] + sky[pl, 1] * d_c.double() + sky[pl, 2] * d_s.double()).float() + \
            sig * torch.randn(e.nsamples, generator=gen, device="cuda")
        del sky
    p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, d_c, d_s, 3)
    n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    out = torch.zeros(R * e.npix * 3, dtype=torch.float64, device="cuda")
    st, infos = L.bm_pcg_solve(p, n, pc, tod, R, out, 1e-8, 100, L.BM_PREC_MIXED)
    assert st == L.BM_OK and max(i["rel_residual"] for i in infos) <= 1e-8
    hits = torch.zeros(e.npix, dtype=torch.int32, device="cuda")
    mask = torch.zeros(e.npix, dtype=torch.uint8, device="cuda")
    L.bm_precond_get_mask(pc, mask, hits)
    hits, mask = hits.cpu().numpy(), mask.cpu().numpy().astype(bool)
    pixels = sampled_pixels(hits, mask, np.random.default_rng(2), n=16)
    idx = select_samples(pt["pix"], e.npix, pixels)
    rows = tod[:, torch.from_numpy(idx).cuda()].cpu().numpy()  # the sampled pixels' TOD values
    refs, omask = oracle_white_pixels(e, pt["pix"], c32, s32, idx, list(rows), pixels)
    assert np.array_equal(omask, mask[pixels])
    xg = out.cpu().numpy().reshape(R, e.npix, 3)[:, pixels]
    for r in range(R):
        err = np.linalg.norm(xg[r] - refs[r]) / np.linalg.norm(refs[r])
        assert err < 1e-6, (r, err)
    for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
        f(h)
