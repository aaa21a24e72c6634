"""Diagonal N^-1 with a weight per sample (bm_inv_noise_create_sample_weights;
Eq. 4 with a diagonal W), against the oracle's SampleWeightNoise on the same
seeded inputs: blocks and mask, the operator in FP64 and mixed precision, the
RHS, the solve, N^-1 itself, a TOD sorted along with the pointing, and the
argument checks.  15 % of the samples carry weight 0 (gaps)."""
import numpy as np
import pytest

import synth
from oracle import gls

from gpucase import MIN_HITS, stokes_cols

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


class WCase:
    """A seeded scan with per-sample weights (gaps included), the oracle's
    system and the library's handles."""

    def __init__(self, L, ctx, nside, ndet, ns, seed, solver=3, trig=False):
        self.L, self.solver = L, solver
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        pt = synth.pointing(e, flag_frac=0.01)
        self.pix, self.psi = pt["pix"], pt["psi"]
        rng = np.random.default_rng(seed)
        w = (1.0 / e.sigma ** 2)[np.repeat(np.arange(ndet), ns)] * rng.uniform(0.3, 3.0, e.nsamples)
        self.w = np.where(rng.random(e.nsamples) < 0.15, 0.0, w)
        sky = synth.sky_map(e.npix, seed)
        if solver == 2:
            sky[:, 0] = 0
        if solver == 1:
            sky[:, 1:] = 0
        self.trig = synth.trig32(self.psi) if trig else None
        self.tod = synth.tod(e, self.pix, self.psi, sky, solver=solver, dtype=np.float32, trig=self.trig)
        self.S = gls.System(self.pix, self.psi, solver, e.npix, gls.SampleWeightNoise(self.w),
                            min_hits=MIN_HITS[solver], max_cond=1e3, trig=self.trig)
        self.npix = e.npix
        self.d_pix = torch.from_numpy(self.pix).cuda()
        self.d_tod = torch.from_numpy(self.tod).cuda()
        if trig:
            self.p = L.bm_pointing_create_trig(ctx, e.npix, self.d_pix, torch.from_numpy(self.trig[0]).cuda(),
                                               torch.from_numpy(self.trig[1]).cuda(), solver)
        else:
            self.p = L.bm_pointing_create(ctx, e.npix, self.d_pix, torch.from_numpy(self.psi).cuda(), solver)
        self.n = L.bm_inv_noise_create_sample_weights(ctx, torch.from_numpy(self.w).cuda())
        self.pc = L.bm_blockdiag_precond_create(self.p, self.n, MIN_HITS[solver], 1e3)

    def vec(self, a=None):
        if a is None:
            return torch.zeros(self.npix * self.solver, dtype=torch.float64, device="cuda")
        return torch.from_numpy(np.ascontiguousarray(a, np.float64).ravel()).cuda()

    def close(self):
        self.L.bm_precond_destroy(self.pc)
        self.L.bm_inv_noise_destroy(self.n)
        self.L.bm_pointing_destroy(self.p)


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_blocks_matvec_rhs(L, ctx, solver):
    c = WCase(L, ctx, 16, 4, 30_011, 500 + solver, solver=solver)
    try:
        S = c.S
        B = torch.zeros(c.npix * solver * solver, dtype=torch.float64, device="cuda")
        L.bm_precond_get_blocks(c.pc, B, None)
        assert rel(B.cpu().numpy(), S.B.ravel()) < 1e-13
        m = torch.zeros(c.npix, dtype=torch.uint8, device="cuda")
        L.bm_precond_get_mask(c.pc, m, None)
        assert np.array_equal(m.cpu().numpy().astype(bool), S.mask)
        rng = np.random.default_rng(7)
        x = rng.normal(size=(c.npix, solver)) * np.array([100.0, 10.0, 10.0])[stokes_cols(solver)]
        ref = S.matvec(x * (~S.mask)[:, None])
        for prec, tol in ((L.BM_PREC_FP64, 1e-12), (L.BM_PREC_MIXED, 2e-6)):
            q = c.vec()
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), q, prec)
            qh = q.cpu().numpy().reshape(c.npix, solver)
            for k in range(solver):
                assert rel(qh[:, k], ref[:, k]) < tol, (prec, k)
            assert np.all(qh[S.mask] == 0)
        b = c.vec()
        L.bm_rhs(c.p, c.n, c.pc, c.d_tod, 1, b)
        assert rel(b.cpu().numpy(), S.rhs(c.tod.astype(np.float64)).ravel()) < 1e-12
    finally:
        c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve(L, ctx, prec):
    c = WCase(L, ctx, 16, 4, 50_003, 600, trig=True)
    P = L.BM_PREC_FP64 if prec == "fp64" else L.BM_PREC_MIXED
    try:
        out = c.vec()
        st, info = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-10, 100, P)
        assert st == L.BM_OK, info
        ref, _ = gls.gls_map(c.S, c.tod.astype(np.float64), tol=1e-13)
        got = out.cpu().numpy().reshape(c.npix, 3)
        assert np.array_equal(np.isnan(got).any(axis=1), c.S.mask)
        err = gls.rel_err(got, ref, c.S.mask)
        assert all(v <= 1e-9 for v in err.values()), err
    finally:
        c.close()


def test_inv_noise_apply_and_carried_tod(L, ctx):
    c = WCase(L, ctx, 16, 4, 20_001, 700, trig=True)
    try:
        y = torch.randn(c.e.nsamples, dtype=torch.float64, device="cuda")
        z = torch.zeros_like(y)
        L.bm_inv_noise_apply(c.n, y, z)
        assert torch.equal(z, torch.from_numpy(c.w).cuda() * y)
        # the TOD sorted along with the pointing: the same maps, bit for bit
        c32, s32 = c.trig
        p1 = L.bm_pointing_create_with_tod(ctx, c.npix, c.d_pix, c.d_tod, cos2psi=torch.from_numpy(c32).cuda(),
                                           sin2psi=torch.from_numpy(s32).cuda())
        pc1 = L.bm_blockdiag_precond_create(p1, c.n, 3, 1e3)
        try:
            for P in (L.BM_PREC_FP64, L.BM_PREC_MIXED):
                m0, m1 = c.vec(), c.vec()
                L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, m0, 1e-10, 100, P)
                L.bm_pcg_solve(p1, c.n, pc1, None, 1, m1, 1e-10, 100, P)
                assert torch.equal(torch.nan_to_num(m0, 7.0), torch.nan_to_num(m1, 7.0))
        finally:
            L.bm_precond_destroy(pc1)
            L.bm_pointing_destroy(p1)
    finally:
        c.close()


def test_bad_weights_rejected(L, ctx):
    w = torch.ones(1000, dtype=torch.float64, device="cuda")
    for bad in (-1.0, float("nan"), float("inf")):
        w2 = w.clone()
        w2[517] = bad
        with pytest.raises(Exception):
            L.bm_inv_noise_create_sample_weights(ctx, w2)
    with pytest.raises(Exception):  # pageable host memory
        L.bm_inv_noise_create_sample_weights(ctx, torch.ones(1000, dtype=torch.float64))
    n = L.bm_inv_noise_create_sample_weights(ctx, torch.ones(1000, dtype=torch.float64).pin_memory())
    L.bm_inv_noise_destroy(n)
