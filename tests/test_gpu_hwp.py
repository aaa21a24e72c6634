"""The half-wave-plate pointing (bm_pointing_create_hwp): the angle of every
sample is rebuilt on the device from (psi_d, nu, phi0) and the sample's time
index (Eq. 2 with theta = psi_d + 2 phi_hwp), against the oracle's system
built from the oracle's own angles of the same model (gls.hwp_angles):
hits and mask exact; the FP64 operator within 1e-12; the mixed operator (its
FP32 angle rebuilt per sorted sample from 4 bytes) within 2e-6 and bitwise
reproducible; maps within 1e-10 (FP64) and 1e-6 (mixed) of the oracle's GLS
map; uniform and ragged detector lengths; detectors of 2^22 samples, where
the phase must be reduced exactly."""
import numpy as np
import pytest

import synth
from gpucase import MIN_HITS
from oracle import gls

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
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


class HwpCase:
    """A seeded scan's pixels, the HWP angle model of its experiment, the
    oracle's system from the oracle's angles, and the library's handles."""

    def __init__(self, L, ctx, nside, ndet, ns, seed, solver=3, det_offsets=None, flag=0.01):
        self.L, self.solver = L, solver
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        self.pix = synth.pointing(e, flag_frac=flag)["pix"]
        self.off = e.det_offsets if det_offsets is None else np.asarray(det_offsets, np.int64)
        nd = self.off.size - 1
        rng = np.random.default_rng(seed)
        self.psi_d = e.psi_det if nd == ndet else rng.uniform(0, np.pi, nd)
        self.nu, self.phi0 = e.scan.hwp_hz / e.scan.fsamp, e.hwp_phase0
        self.theta = gls.hwp_angles(self.off, self.psi_d, self.nu, self.phi0)
        self.inv_var = rng.uniform(0.25, 1.0, nd)
        self.npix = e.npix
        sky = synth.sky_map(e.npix, seed)
        if solver == 2:
            sky[:, 0] = 0
        if solver == 1:
            sky[:, 1:] = 0
        # white noise of each detector's level, drawn here (the TOD is the
        # oracle's P s from its own angles plus that noise)
        v = gls.pointing_weights(self.theta, solver)
        pe = np.where(self.pix >= 0, self.pix, -1).astype(np.int64)
        cols = {3: [0, 1, 2], 2: [1, 2], 1: [0]}[solver]
        sig = 1.0 / np.sqrt(self.inv_var)[gls.sample_detector(self.off)]
        self.tod = gls.apply_P(pe, v, sky[:, cols]) + rng.normal(size=self.pix.size) * sig
        self.S = gls.System(self.pix, self.theta, solver, e.npix, gls.WhiteNoise(self.inv_var, self.off),
                            min_hits=MIN_HITS[solver])
        self.p = L.bm_pointing_create_hwp(ctx, e.npix, torch.from_numpy(self.pix).cuda(), self.off, self.psi_d,
                                          self.nu, self.phi0, solver)
        self.n = L.bm_inv_noise_create_diag(ctx, self.off, self.inv_var)
        self.pc = L.bm_blockdiag_precond_create(self.p, self.n, MIN_HITS[solver], 1e3)

    def mask_hits(self):
        m = torch.zeros(self.npix, dtype=torch.uint8, device="cuda")
        h = torch.zeros(self.npix, dtype=torch.int32, device="cuda")
        self.L.bm_precond_get_mask(self.pc, m, h)
        return m.cpu().numpy().astype(bool), h.cpu().numpy()

    def matvec(self, x, prec):
        q = torch.zeros(self.npix * self.solver, dtype=torch.float64, device="cuda")
        self.L.bm_matvec(self.p, self.n, self.pc, torch.from_numpy(x.ravel()).cuda(), q, prec)
        return q.cpu().numpy().reshape(self.npix, self.solver)

    def close(self):
        self.L.bm_precond_destroy(self.pc)
        self.L.bm_inv_noise_destroy(self.n)
        self.L.bm_pointing_destroy(self.p)


def check_operators(c, seed):
    L = c.L
    mask, hits = c.mask_hits()
    assert np.array_equal(hits, c.S.hits)
    assert np.array_equal(mask, c.S.mask)
    x = np.random.default_rng(seed).normal(size=(c.npix, c.solver)) * 30.0
    want = c.S.matvec(x)
    q64 = c.matvec(x, L.BM_PREC_FP64)
    qm = c.matvec(x, L.BM_PREC_MIXED)
    for k in range(c.solver):
        assert rel(q64[~mask, k], want[~mask, k]) < 1e-12, k
        assert rel(qm[~mask, k], want[~mask, k]) < 2e-6, k
    assert np.all(q64[mask] == 0) and np.all(qm[mask] == 0)
    assert np.array_equal(c.matvec(x, L.BM_PREC_MIXED), qm)  # deterministic


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_hwp_operators_and_maps(L, ctx, solver):
    c = HwpCase(L, ctx, 16, 4, 65_536, 6100 + solver, solver=solver)
    try:
        check_operators(c, solver)
        ref, _ = gls.gls_map(c.S, c.tod, tol=1e-13)
        out = torch.zeros(c.npix * solver, dtype=torch.float64, device="cuda")
        tod = torch.from_numpy(c.tod).cuda()
        for prec, tol in ((L.BM_PREC_FP64, 1e-10), (L.BM_PREC_MIXED, 1e-6)):
            st, info = L.bm_pcg_solve(c.p, c.n, c.pc, tod, 1, out, 1e-11, 200, prec)
            assert st == L.BM_OK, info
            err = gls.rel_err(out.cpu().numpy().reshape(c.npix, solver), ref, c.S.mask)
            assert max(err.values()) < tol, (prec, err)
    finally:
        c.close()


def test_hwp_ragged_detectors(L, ctx):
    """Detectors of different lengths: the detector is found by a search of
    the offsets, and each detector's phase restarts at k = 0."""
    off = [0, 50_000, 131_089, 200_000, 262_144]
    c = HwpCase(L, ctx, 16, 4, 65_536, 6200, det_offsets=off)
    try:
        check_operators(c, 7)
    finally:
        c.close()


def test_hwp_long_detectors(L, ctx):
    """Two detectors of 2^22 samples: nu k reaches 2^22 / 20 ~ 2e5 turns, where
    an unreduced FP32 phase would be meaningless and an unreduced FP64 one
    off by ~1e-10 rad."""
    c = HwpCase(L, ctx, 8, 2, 2 ** 22, 6300, flag=0.0)
    try:
        check_operators(c, 8)
    finally:
        c.close()


def test_hwp_rejects_bad_models(L, ctx):
    pix = torch.zeros(100, dtype=torch.int32, device="cuda")
    for off, psi_d, nu in (([0, 60], [0.1], 0.05),                # offsets do not cover the samples
                           ([0, 60, 100], [0.1, np.nan], 0.05),   # non-finite angle
                           ([0, 60, 100], [0.1, 0.2], np.inf)):   # non-finite rate
        with pytest.raises(L.BrahmapError) as ei:
            L.bm_pointing_create_hwp(ctx, 12, pix, np.array(off), np.array(psi_d), nu, 0.0, 3)
        assert ei.value.status == L.BM_ERR_INVALID
