"""Resident pointings and batched requests in the request loop (bm_serve_*
with pointing_key): requests that share a pointing reuse its ingested form,
noise model and preconditioner; queued white-noise requests of one key are
solved together by the multi-RHS PCG; idle entries are released for memory.
Maps: a request solved on a resident pointing alone is bitwise the map of the
same request solved from scratch; a request solved in a batch matches its
solo map to the rounding of the CG scalars (1e-9) and the oracle's GLS map
(1e-6), and is bitwise the map of the same right-hand sides solved by
bm_pcg_solve with nrhs = batch size."""
import time

import numpy as np
import pytest

import synth
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


def wait(L, srv, t, timeout_s=120):
    t0 = time.time()
    while True:
        st, res = L.bm_serve_poll(srv, t, 200)
        if st == L.BM_OK:
            return res
        assert st == L.BM_ERR_TIMEOUT
        assert time.time() - t0 < timeout_s, "request did not finish"


def rel(a, b):
    a, b = np.nan_to_num(np.asarray(a)), np.nan_to_num(np.asarray(b))
    return np.linalg.norm(a - b) / np.linalg.norm(b)


class Scan:
    """One seeded pointing on the device and TOD realisations on it (a sky
    and white noise of its own per realisation)."""

    def __init__(self, nside, ndet, ns, seed, nreal):
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        pt = synth.pointing(e)
        self.pix, self.psi = pt["pix"], pt["psi"]
        self.trig = synth.trig32(self.psi)
        self.inv_var = 1.0 / e.sigma ** 2
        self.d_pix = torch.from_numpy(self.pix).cuda()
        self.d_c = torch.from_numpy(self.trig[0]).cuda()
        self.d_s = torch.from_numpy(self.trig[1]).cuda()
        self.tods = []
        for k in range(nreal):
            sky = synth.sky_map(e.npix, seed * 100 + k)
            self.tods.append(synth.tod(e, self.pix, self.psi, sky, noise_seed=seed * 100 + k, dtype=np.float32,
                                       trig=self.trig))
        self.d_tods = [torch.from_numpy(t).cuda() for t in self.tods]
        self.outs = [torch.full((e.npix * 3,), 7.0, dtype=torch.float64, device="cuda") for _ in range(nreal)]

    def request(self, L, k, key, tol=1e-8, coeffs=None, chunk=0):
        kw = dict(coeffs=coeffs, chunk_len=chunk) if coeffs is not None else {}
        return L.make_request(self.e.npix, self.d_pix, self.d_tods[k], self.outs[k], self.e.det_offsets,
                              self.inv_var, cos2psi=self.d_c, sin2psi=self.d_s, tol=tol, maxiter=500,
                              pointing_key=key, **kw)

    def handles(self, L, ctx, coeffs=None, chunk=0):
        p = L.bm_pointing_create_trig(ctx, self.e.npix, self.d_pix, self.d_c, self.d_s, 3)
        if coeffs is None:
            n = L.bm_inv_noise_create_diag(ctx, self.e.det_offsets, self.inv_var)
        else:
            n = L.bm_inv_noise_create_toeplitz(ctx, self.e.det_offsets, chunk, coeffs, self.inv_var)
        return p, n, L.bm_blockdiag_precond_create(p, n, 3, 1e3)

    def solve_alone(self, L, ctx, k, tol=1e-8, coeffs=None, chunk=0):
        p, n, pc = self.handles(L, ctx, coeffs, chunk)
        out = torch.zeros_like(self.outs[k])
        st, _ = L.bm_pcg_solve(p, n, pc, self.d_tods[k], 1, out, tol, 500, L.BM_PREC_MIXED)
        assert st == L.BM_OK
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)
        return out


def blocker(L):
    """An unkeyed Toeplitz request that keeps a one-slot server busy while
    the keyed requests queue up behind it."""
    e = synth.make_experiment(32, 9, 40_000, 4242)
    pt = synth.pointing(e)
    coeffs = synth.toeplitz_band(e.sigma, 0.2, 1.0, 20.0, 8192, 256)
    tod = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 4242), white=False,
                    extra=synth.one_over_f_noise(e, 4096, 0.2, 1.0), dtype=np.float32)
    bufs = [torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(pt["psi"]).cuda(), torch.from_numpy(tod).cuda(),
            torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")]
    req, keep = L.make_request(e.npix, bufs[0], bufs[2], bufs[3], e.det_offsets, 1 / e.sigma ** 2, psi=bufs[1],
                               coeffs=coeffs, chunk_len=4096, tol=1e-7, maxiter=2000)
    return req, (keep, bufs)


def test_batched_and_resident_requests(L, ctx):
    sc = Scan(32, 8, 40_000, 5100, 5)
    srv = L.bm_serve_create(ctx, 8 << 30, 1)
    try:
        bq, bkeep = blocker(L)
        tb = L.bm_serve_submit(srv, bq)
        keep = [sc.request(L, k, key=77) for k in range(4)]
        tickets = [L.bm_serve_submit(srv, rq) for rq, _ in keep]
        assert wait(L, srv, tb)["status"] == L.BM_OK
        results = [wait(L, srv, t) for t in tickets]
        sizes = [r["batch_size"] for r in results]
        assert all(r["status"] == L.BM_OK for r in results), results
        assert all(r["rel_residual"] <= 1e-8 for r in results)
        assert max(sizes) >= 2, sizes  # queued behind the blocker, they were solved together
        st = L.bm_serve_get_stats(srv)
        assert st["batches"] >= 1 and st["batched_requests"] == sum(1 for s in sizes if s > 1)
        assert st["resident_bytes"] > 0
        # each batched map: its solo map to the CG scalars' rounding, and the oracle
        for k in range(4):
            alone = sc.solve_alone(L, ctx, k)
            assert rel(sc.outs[k].cpu().numpy(), alone.cpu().numpy()) < 1e-9, k
        S = gls.System(sc.pix, sc.psi, 3, sc.e.npix, gls.WhiteNoise(sc.inv_var, sc.e.det_offsets), trig=sc.trig)
        ref, _ = gls.gls_map(S, sc.tods[0].astype(np.float64), tol=1e-13)
        err = gls.rel_err(sc.outs[0].cpu().numpy().reshape(sc.e.npix, 3), ref, S.mask)
        assert max(err.values()) < 1e-6, err
        # a batch of all four: bitwise the multi-RHS solve of bm_pcg_solve
        if sizes == [4, 4, 4, 4]:
            p, n, pc = sc.handles(L, ctx)
            tod = torch.stack(sc.d_tods[:4])
            out = torch.zeros(4 * sc.e.npix * 3, dtype=torch.float64, device="cuda")
            s2, _ = L.bm_pcg_solve(p, n, pc, tod, 4, out, 1e-8, 500, L.BM_PREC_MIXED)
            assert s2 == L.BM_OK
            for k in range(4):
                assert torch.equal(torch.nan_to_num(out[k * sc.e.npix * 3:(k + 1) * sc.e.npix * 3]),
                                   torch.nan_to_num(sc.outs[k]))
            L.bm_precond_destroy(pc)
            L.bm_inv_noise_destroy(n)
            L.bm_pointing_destroy(p)
        # a later request of the key alone: on the resident pointing, bitwise its solo map
        rq, kp = sc.request(L, 4, key=77)
        r5 = wait(L, srv, L.bm_serve_submit(srv, rq))
        assert r5["status"] == L.BM_OK and r5["resident"] == 1 and r5["batch_size"] == 1
        assert torch.equal(torch.nan_to_num(sc.outs[4]), torch.nan_to_num(sc.solve_alone(L, ctx, 4)))
        assert L.bm_serve_get_stats(srv)["resident_hits"] >= 1
    finally:
        L.bm_serve_destroy(srv)


def test_resident_pointing_with_another_noise_model(L, ctx):
    """The same key with a Toeplitz N^-1: the pointing is reused, the noise
    model and preconditioner are rebuilt; the map is bitwise the solo one."""
    sc = Scan(16, 4, 30_000, 5200, 2)
    coeffs = synth.toeplitz_band(sc.e.sigma, 0.2, 1.0, 20.0, 8192, 128)
    srv = L.bm_serve_create(ctx, 8 << 30, 2)
    try:
        rq0, k0 = sc.request(L, 0, key=5)
        assert wait(L, srv, L.bm_serve_submit(srv, rq0))["status"] == L.BM_OK
        rq1, k1 = sc.request(L, 1, key=5, tol=1e-7, coeffs=coeffs, chunk=4096)
        r1 = wait(L, srv, L.bm_serve_submit(srv, rq1))
        assert r1["status"] == L.BM_OK and r1["resident"] == 1
        alone = sc.solve_alone(L, ctx, 1, tol=1e-7, coeffs=coeffs, chunk=4096)
        assert torch.equal(torch.nan_to_num(sc.outs[1]), torch.nan_to_num(alone))
        # the key reused with another shape is refused
        other = Scan(16, 4, 20_000, 5201, 1)
        rq2, k2 = other.request(L, 0, key=5)
        r2 = wait(L, srv, L.bm_serve_submit(srv, rq2))
        assert r2["status"] == L.BM_ERR_INVALID and "another shape" in r2["message"]
    finally:
        L.bm_serve_destroy(srv)


def test_idle_resident_pointing_released_for_memory(L, ctx):
    a, b = Scan(16, 4, 40_000, 5300, 1), Scan(16, 4, 40_000, 5301, 1)
    # room for one request built from scratch plus one resident pointing of
    # 160k samples (~5.7 MB), not for two resident pointings and a build
    budget = 160_000 * 48 + 3072 * 477 + (64 << 20) + (3 << 20)
    srv = L.bm_serve_create(ctx, budget, 1)
    try:
        qa, ka = a.request(L, 0, key=1)
        qb, kb = b.request(L, 0, key=2)
        ra = wait(L, srv, L.bm_serve_submit(srv, qa))
        rb = wait(L, srv, L.bm_serve_submit(srv, qb))
        assert ra["status"] == L.BM_OK and rb["status"] == L.BM_OK
        st = L.bm_serve_get_stats(srv)
        assert st["evictions"] == 1 and st["peak_reserved_bytes"] <= budget
        assert 0 < st["resident_bytes"] < 6 << 20  # b's pointing alone
        ra2 = wait(L, srv, L.bm_serve_submit(srv, qa))
        assert ra2["status"] == L.BM_OK and ra2["resident"] == 0  # rebuilt after its release
        assert torch.equal(torch.nan_to_num(a.outs[0]), torch.nan_to_num(a.solve_alone(L, ctx, 0)))
        assert torch.equal(torch.nan_to_num(b.outs[0]), torch.nan_to_num(b.solve_alone(L, ctx, 0)))
    finally:
        L.bm_serve_destroy(srv)
