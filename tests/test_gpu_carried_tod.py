"""A TOD sorted along with the pointing (bm_pointing_create_with_tod): the
pixel-sorted copy it leaves must give the same b = P^T N^-1 d (Eq. 6) and
the same maps as the time-ordered TOD gathered through the permutation --
bitwise, since both read the same FP32 values and add them in the same
order -- and match the oracle.  Every sort plan (one, two and three radix
passes), angles and trig pairs, flagged samples and a ragged last tile."""
import numpy as np
import pytest

import synth
from oracle import gls

from gpucase import Case

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


@pytest.mark.parametrize("nside,n,trig", [(8, 200_003, False),       # one sort pass
                                          (64, 3_000_001, True),     # two passes
                                          (1024, 500_009, False)])   # three passes
def test_carried_tod_rhs_matches_gathered_tod(L, ctx, nside, n, trig):
    npix = 12 * nside * nside
    rng = np.random.default_rng(100 + nside)
    pix = rng.integers(0, npix, size=n).astype(np.int32)
    pix[1::3] = pix[0::3][: pix[1::3].size]
    pix[rng.random(n) < 0.1] = -1
    psi = rng.uniform(0, np.pi, size=n)
    tod = rng.normal(size=n).astype(np.float32)
    ndet = 5
    off = np.linspace(0, n, ndet + 1).astype(np.int64)
    inv_var = rng.uniform(0.5, 2.0, ndet)
    d_pix, d_tod = torch.from_numpy(pix).cuda(), torch.from_numpy(tod).cuda()
    if trig:
        c32, s32 = synth.trig32(psi)
        kw = dict(cos2psi=torch.from_numpy(c32).cuda(), sin2psi=torch.from_numpy(s32).cuda())
        p0 = L.bm_pointing_create_trig(ctx, npix, d_pix, kw["cos2psi"], kw["sin2psi"], 3)
    else:
        kw = dict(psi=torch.from_numpy(psi).cuda())
        p0 = L.bm_pointing_create(ctx, npix, d_pix, kw["psi"], 3)
    p1 = L.bm_pointing_create_with_tod(ctx, npix, d_pix, d_tod, **kw)
    n_ = L.bm_inv_noise_create_diag(ctx, off, inv_var)
    pc0 = L.bm_blockdiag_precond_create(p0, n_, 1, 1e6)
    pc1 = L.bm_blockdiag_precond_create(p1, n_, 1, 1e6)
    try:
        b0 = torch.zeros(npix * 3, dtype=torch.float64, device="cuda")
        b1 = torch.zeros_like(b0)
        L.bm_rhs(p0, n_, pc0, d_tod, 1, b0)
        L.bm_rhs(p1, n_, pc1, None, 1, b1)
        assert torch.equal(b0, b1)
        # against the oracle on the kept pixels
        m = torch.zeros(npix, dtype=torch.uint8, device="cuda")
        L.bm_precond_get_mask(pc1, m, None)
        kept = m.cpu().numpy() == 0
        v = gls.pointing_weights_trig(c32, s32, 3) if trig else gls.pointing_weights(psi, 3)
        w = np.repeat(inv_var, np.diff(off))
        pe = np.where(pix >= 0, pix, -1)
        pe = np.where((pe >= 0) & kept[np.maximum(pe, 0)], pe, -1)
        want = gls.apply_PT(pe, v, w * np.where(pe >= 0, tod.astype(np.float64), 0.0), npix)
        assert rel(b1.cpu().numpy(), want.ravel()) < 1e-12
    finally:
        L.bm_precond_destroy(pc0)
        L.bm_precond_destroy(pc1)
        L.bm_inv_noise_destroy(n_)
        L.bm_pointing_destroy(p0)
        L.bm_pointing_destroy(p1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("host", [False, True])
def test_carried_tod_solve(L, ctx, prec, host):
    """The solve with the carried TOD equals the solve with the time-ordered
    TOD bit for bit, and the map matches the oracle's (the parity bars of the
    FP64 and refined paths); a page-locked host TOD gives the same handle."""
    c = Case(L, ctx, 16, 4, 40_000, 777, flag=0.01, trig=True, tod_dtype=np.float32)
    P = L.BM_PREC_FP64 if prec == "fp64" else L.BM_PREC_MIXED
    try:
        c32, s32 = c.trig
        tod = torch.from_numpy(c.tod).pin_memory() if host else c.d_tod
        p1 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc1 = L.bm_blockdiag_precond_create(p1, c.n, 3, 1e3)
        try:
            m0, m1 = c.vec(), c.vec()
            st0, _ = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, m0, 1e-10, 200, P)
            st1, info = L.bm_pcg_solve(p1, c.n, pc1, None, 1, m1, 1e-10, 200, P)
            assert st0 == st1 == L.BM_OK
            assert torch.equal(torch.nan_to_num(m0, 7.0), torch.nan_to_num(m1, 7.0))
            want, _ = gls.gls_map(c.S, c.tod.astype(np.float64), tol=1e-13)
            err = gls.rel_err(m1.cpu().numpy().reshape(c.npix, 3), want, c.S.mask)
            assert all(v <= 1e-8 for v in err.values()), err
        finally:
            L.bm_precond_destroy(pc1)
            L.bm_pointing_destroy(p1)
    finally:
        c.close()


def test_carried_tod_pointing_with_time_ordered_operators(L, ctx):
    """A pointing that carries a TOD, given pixels and cos/sin in device
    memory, builds its time-ordered pixels and trig pairs only when a
    time-ordered operator first needs them: with Toeplitz noise its matvecs
    (FP64 and mixed), its P x and its refined solve, and with the offset
    template its matvecs, are bitwise those of the same pointing made
    without the TOD (which keeps both at creation)."""
    c = Case(L, ctx, 16, 4, 40_000, 4321, noise="toeplitz", chunk=4096, nlags=64, flag=0.01, trig=True,
             tod_dtype=np.float32, build_oracle=False)
    try:
        c32, s32 = c.trig
        p1 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc1 = L.bm_blockdiag_precond_create(p1, c.n, 3, 1e3)
        try:
            x = c.vec(np.random.default_rng(5).normal(size=(c.npix, 3)))
            y0 = torch.zeros(c.e.nsamples, dtype=torch.float64, device="cuda")
            y1 = torch.zeros_like(y0)
            L.bm_pointing_apply(p1, x, y1)  # the first time-ordered call builds the pairs
            L.bm_pointing_apply(c.p, x, y0)
            assert torch.equal(y0, y1)
            for prec in (L.BM_PREC_FP64, L.BM_PREC_MIXED):
                q0, q1 = c.vec(), c.vec()
                L.bm_matvec(c.p, c.n, c.pc, x, q0, prec)
                L.bm_matvec(p1, c.n, pc1, x, q1, prec)
                assert torch.equal(torch.nan_to_num(q0), torch.nan_to_num(q1)), prec
            m0, m1 = c.vec(), c.vec()
            st0, _ = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, m0, 1e-8, 300, L.BM_PREC_MIXED)
            st1, _ = L.bm_pcg_solve(p1, c.n, pc1, c.d_tod, 1, m1, 1e-8, 300, L.BM_PREC_MIXED)
            assert st0 == st1 == L.BM_OK
            assert torch.equal(torch.nan_to_num(m0, 7.0), torch.nan_to_num(m1, 7.0))
        finally:
            L.bm_precond_destroy(pc1)
            L.bm_pointing_destroy(p1)
        # the offset template's operators (time-ordered interval means) on a
        # fresh carried pointing: bitwise those of the plain pointing
        inv_var = 1.0 / c.e.sigma ** 2
        n_o = L.bm_inv_noise_create_offset_filter(ctx, c.e.det_offsets, inv_var, 700)
        p3 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc_o0 = L.bm_blockdiag_precond_create(c.p, n_o, 3, 1e3)
        pc_o3 = L.bm_blockdiag_precond_create(p3, n_o, 3, 1e3)
        try:
            x = c.vec(np.random.default_rng(6).normal(size=(c.npix, 3)))
            for prec in (L.BM_PREC_FP64, L.BM_PREC_MIXED):
                q0, q3 = c.vec(), c.vec()
                L.bm_matvec(c.p, n_o, pc_o0, x, q0, prec)
                L.bm_matvec(p3, n_o, pc_o3, x, q3, prec)
                assert torch.equal(torch.nan_to_num(q0), torch.nan_to_num(q3)), prec
        finally:
            L.bm_precond_destroy(pc_o3)
            L.bm_precond_destroy(pc_o0)
            L.bm_pointing_destroy(p3)
            L.bm_inv_noise_destroy(n_o)
        # a fresh carried pointing whose first time-ordered operator is the solve
        p2 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc2 = L.bm_blockdiag_precond_create(p2, c.n, 3, 1e3)
        try:
            m2 = c.vec()
            st2, _ = L.bm_pcg_solve(p2, c.n, pc2, c.d_tod, 1, m2, 1e-8, 300, L.BM_PREC_MIXED)
            assert st2 == L.BM_OK and torch.equal(torch.nan_to_num(m0, 7.0), torch.nan_to_num(m2, 7.0))
        finally:
            L.bm_precond_destroy(pc2)
            L.bm_pointing_destroy(p2)
    finally:
        c.close()


def test_carried_tod_errors(L, ctx):
    c = Case(L, ctx, 8, 2, 5_000, 31, noise="toeplitz", chunk=1000, nlags=8, tod_dtype=np.float32,
             build_oracle=False)
    try:
        b = c.vec()
        with pytest.raises(Exception):  # the pointing carries no TOD
            L.bm_rhs(c.p, c.n, c.pc, None, 1, b)
        p1 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, psi=c.d_psi)
        pc1 = L.bm_blockdiag_precond_create(p1, c.n, 3, 1e3)
        n_w = L.bm_inv_noise_create_diag(ctx, c.e.det_offsets, np.ones(c.e.ndet))
        pc_w = L.bm_blockdiag_precond_create(p1, n_w, 3, 1e3)
        try:
            with pytest.raises(Exception):  # Toeplitz noise filters in time order
                L.bm_rhs(p1, c.n, pc1, None, 1, b)
            with pytest.raises(Exception):  # one carried right-hand side
                L.bm_rhs(p1, n_w, pc_w, None, 2, torch.zeros(2 * c.npix * 3, dtype=torch.float64, device="cuda"))
            L.bm_rhs(p1, n_w, pc_w, None, 1, b)  # white noise, one RHS: fine
        finally:
            L.bm_precond_destroy(pc_w)
            L.bm_inv_noise_destroy(n_w)
            L.bm_precond_destroy(pc1)
            L.bm_pointing_destroy(p1)
        c32, s32 = synth.trig32(c.psi.astype(np.float64))
        with pytest.raises(Exception):  # both angles and trig pairs
            L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, psi=c.d_psi,
                                          cos2psi=torch.from_numpy(c32).cuda(), sin2psi=torch.from_numpy(s32).cuda())
        with pytest.raises(Exception):  # neither
            L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod)
    finally:
        c.close()


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_carried_tod_off_a_16_byte_boundary(L, ctx, offset):
    """A TOD view that starts 4, 8 or 12 bytes past a 16-byte boundary is read
    with plain loads instead of bulk copies by the first sort pass: the same
    RHS, bit for bit, as the gathered time-ordered TOD (two sort passes, a
    ragged last tile)."""
    c = Case(L, ctx, 64, 3, 400_001, 91 + offset, flag=0.02, trig=True, tod_dtype=np.float32)
    try:
        c32, s32 = c.trig
        full = torch.zeros(c.e.nsamples + offset, dtype=torch.float32, device="cuda")
        full[offset:] = c.d_tod
        tod = full[offset:]
        assert tod.data_ptr() % 16 != 0
        p1 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc1 = L.bm_blockdiag_precond_create(p1, c.n, 3, 1e3)
        try:
            b0, b1 = c.vec(), c.vec()
            L.bm_rhs(c.p, c.n, c.pc, c.d_tod, 1, b0)
            L.bm_rhs(p1, c.n, pc1, None, 1, b1)
            assert torch.equal(b0, b1)
        finally:
            L.bm_precond_destroy(pc1)
            L.bm_pointing_destroy(p1)
    finally:
        c.close()
