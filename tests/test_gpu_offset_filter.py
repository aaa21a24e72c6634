"""White N^-1 with a baseline offset per interval marginalised out
(bm_inv_noise_create_offset_filter; Eq. 4 with the offsets as a filtering
template), against the oracle's OffsetFilterNoise on the same seeded inputs:
blocks and mask, the operator in FP64 and mixed precision, the RHS from FP32
and FP64 TODs, the solve (Q and U exactly, I up to its monopole, which is in
the null space of A), N^-1 itself on ragged detectors and intervals, and the
argument checks."""
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


class OCase:
    """A seeded scan with a random offset on every interval, the oracle's
    system and the library's handles."""

    def __init__(self, L, ctx, nside, ndet, ns, seed, baseline_len, solver=3, flag=0.02):
        self.L, self.solver = L, solver
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        pt = synth.pointing(e, flag_frac=flag)
        self.pix, self.psi = pt["pix"], pt["psi"]
        sky = synth.sky_map(e.npix, seed)
        if solver == 2:
            sky[:, 0] = 0
        if solver == 1:
            sky[:, 1:] = 0
        inv_var = 1.0 / e.sigma ** 2
        N = gls.OffsetFilterNoise(inv_var, e.det_offsets, baseline_len)
        d = synth.tod(e, self.pix, self.psi, sky, solver=solver)
        rng = np.random.default_rng(seed)
        for a, b in N.intervals():
            d[a:b] += rng.normal(0.0, 30.0)
        self.tod = d
        self.S = gls.System(self.pix, self.psi, solver, e.npix, N, min_hits=MIN_HITS[solver], max_cond=1e3)
        self.npix = e.npix
        self.d_tod = torch.from_numpy(d).cuda()
        self.p = L.bm_pointing_create(ctx, e.npix, torch.from_numpy(self.pix).cuda(),
                                      torch.from_numpy(self.psi).cuda(), solver)
        self.n = L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, inv_var, baseline_len)
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
    # 30_011 samples a detector, baselines of 1000: a short last interval
    c = OCase(L, ctx, 16, 4, 30_011, 800 + solver, 1000, solver=solver)
    try:
        S = c.S
        B = torch.zeros(c.npix * solver * solver, dtype=torch.float64, device="cuda")
        L.bm_precond_get_blocks(c.pc, B, None)
        assert rel(B.cpu().numpy(), S.B.ravel()) < 1e-13
        m = torch.zeros(c.npix, dtype=torch.uint8, device="cuda")
        L.bm_precond_get_mask(c.pc, m, None)
        assert np.array_equal(m.cpu().numpy().astype(bool), S.mask)
        rng = np.random.default_rng(9)
        x = rng.normal(size=(c.npix, solver)) * np.array([100.0, 10.0, 10.0])[stokes_cols(solver)]
        ref = S.matvec(x * (~S.mask)[:, None])
        for prec, tol in ((L.BM_PREC_FP64, 1e-12), (L.BM_PREC_MIXED, 2e-6)):
            q = c.vec()
            L.bm_matvec(c.p, c.n, c.pc, c.vec(x), q, prec)
            qh = q.cpu().numpy().reshape(c.npix, solver)
            for k in range(solver):
                assert rel(qh[:, k], ref[:, k]) < tol, (prec, k)
            assert np.all(qh[S.mask] == 0)
        ref_b = S.rhs(c.tod).ravel()
        for d, tol in ((c.d_tod, 1e-12), (c.d_tod.float(), 1e-12)):
            b = c.vec()
            L.bm_rhs(c.p, c.n, c.pc, d, 1, b)
            want = ref_b if d.dtype == torch.float64 else S.rhs(d.cpu().numpy().astype(np.float64)).ravel()
            assert rel(b.cpu().numpy(), want) < tol
    finally:
        c.close()


def _demeaned_I(x, keep):
    y = np.array(x, np.float64)
    y[keep, 0] -= y[keep, 0].mean()
    return y


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve(L, ctx, prec):
    c = OCase(L, ctx, 16, 4, 40_003, 900, 700)
    P = L.BM_PREC_FP64 if prec == "fp64" else L.BM_PREC_MIXED
    try:
        out = c.vec()
        st, info = L.bm_pcg_solve(c.p, c.n, c.pc, c.d_tod, 1, out, 1e-10, 300, P)
        assert st == L.BM_OK, info
        ref, rinfo = gls.gls_map(c.S, c.tod, tol=1e-13, maxiter=3000)
        assert rinfo.converged
        got = out.cpu().numpy().reshape(c.npix, 3)
        assert np.array_equal(np.isnan(got).any(axis=1), c.S.mask)
        keep = ~c.S.mask
        err = gls.rel_err(_demeaned_I(got, keep), _demeaned_I(ref, keep), c.S.mask)
        assert all(v <= 1e-8 for v in err.values()), err
    finally:
        c.close()


@pytest.mark.parametrize("offsets,bl", [([0, 1000, 2500, 2501, 5000], 300),   # ragged detectors and intervals
                                        ([0, 4096, 8192], 1 << 40),           # one interval a detector
                                        ([0, 777, 5000], 1)])                 # W = 0
def test_inv_noise_apply(L, ctx, offsets, bl):
    off = np.array(offsets, np.int64)
    nd = off.size - 1
    iv = np.linspace(0.5, 2.0, nd)
    n = L.bm_inv_noise_create_offset_filter(ctx, off, iv, bl)
    try:
        rng = np.random.default_rng(int(off[-1]))
        y = rng.normal(size=off[-1]) + 5.0
        z = torch.zeros(off[-1], dtype=torch.float64, device="cuda")
        L.bm_inv_noise_apply(n, torch.from_numpy(y).cuda(), z)
        ref = gls.OffsetFilterNoise(iv, off, min(bl, int(off[-1]))).apply(y)
        if bl == 1:
            assert torch.count_nonzero(z) == 0
        else:
            assert rel(z.cpu().numpy(), ref) < 1e-13
    finally:
        L.bm_inv_noise_destroy(n)


def test_argument_checks(L, ctx):
    e = synth.make_experiment(8, 2, 3000, 5)
    with pytest.raises(Exception):
        L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, 1 / e.sigma ** 2, 0)
    with pytest.raises(Exception):
        L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, -1 / e.sigma ** 2, 100)
    pt = synth.pointing(e)
    p = L.bm_pointing_create(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(pt["psi"]).cuda(), 3)
    nw = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
    no = L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, 1 / e.sigma ** 2, 100)
    pc = L.bm_blockdiag_precond_create(p, nw, 3, 1e3)
    try:
        x = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
        q = torch.zeros_like(x)
        with pytest.raises(Exception):  # a preconditioner built from another noise handle
            L.bm_matvec(p, no, pc, x, q, L.BM_PREC_FP64)
    finally:
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(no)
        L.bm_inv_noise_destroy(nw)
        L.bm_pointing_destroy(p)
