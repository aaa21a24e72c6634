"""The continuous-batching request loop (bm_serve_*): requests of different
sizes and noise models run concurrently, are admitted against the memory
budget, and each map is the same alone and in the mix."""
import threading
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


class Req:
    """A seeded request: device inputs, output buffer and the oracle's inputs."""

    def __init__(self, L, nside, ndet, ns, seed, noise="white", solver=3, trig=True):
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        pt = synth.pointing(e)
        self.pix, self.psi = pt["pix"], pt["psi"]
        self.solver, self.noise = solver, noise
        self.trig = synth.trig32(self.psi) if trig else None
        sky = synth.sky_map(e.npix, seed)
        if solver == 2:
            sky[:, 0] = 0
        self.inv_var = 1.0 / e.sigma ** 2
        extra, self.coeffs, self.chunk = None, None, 0
        if noise == "toeplitz":
            self.chunk = 4096
            self.coeffs = synth.toeplitz_band(e.sigma, 0.2, 1.0, 20.0, 8192, 256)
            extra = synth.one_over_f_noise(e, self.chunk, 0.2, 1.0)
        self.tod = synth.tod(e, self.pix, self.psi, sky, solver=solver, white=noise == "white", extra=extra,
                             dtype=np.float32, trig=self.trig)
        self.d_pix = torch.from_numpy(self.pix).cuda()
        self.d_tod = torch.from_numpy(self.tod).cuda()
        if trig:
            self.d_c = torch.from_numpy(self.trig[0]).cuda()
            self.d_s = torch.from_numpy(self.trig[1]).cuda()
        else:
            self.d_psi = torch.from_numpy(self.psi).cuda()
        self.out = torch.full((e.npix * solver,), 7.0, dtype=torch.float64, device="cuda")

    def request(self, L, tol=1e-7):
        kw = dict(cos2psi=self.d_c, sin2psi=self.d_s) if self.trig is not None else dict(psi=self.d_psi)
        if self.noise == "toeplitz":
            kw.update(coeffs=self.coeffs, chunk_len=self.chunk)
        return L.make_request(self.e.npix, self.d_pix, self.d_tod, self.out, self.e.det_offsets, self.inv_var,
                              solver=self.solver, min_hits={3: 3, 2: 2, 1: 1}[self.solver], tol=tol,
                              maxiter=2000, **kw)

    def solve_alone(self, L, ctx, tol=1e-7):
        if self.trig is not None:
            p = L.bm_pointing_create_trig(ctx, self.e.npix, self.d_pix, self.d_c, self.d_s, self.solver)
        else:
            p = L.bm_pointing_create(ctx, self.e.npix, self.d_pix, self.d_psi, self.solver)
        if self.noise == "white":
            n = L.bm_inv_noise_create_diag(ctx, self.e.det_offsets, self.inv_var)
        else:
            n = L.bm_inv_noise_create_toeplitz(ctx, self.e.det_offsets, self.chunk, self.coeffs, self.inv_var)
        pc = L.bm_blockdiag_precond_create(p, n, {3: 3, 2: 2, 1: 1}[self.solver], 1e3)
        out = torch.zeros_like(self.out)
        st, info = L.bm_pcg_solve(p, n, pc, self.d_tod, 1, out, tol, 2000, L.BM_PREC_MIXED)
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)
        return st, out

    def oracle(self):
        noise = gls.WhiteNoise(self.inv_var, self.e.det_offsets) if self.noise == "white" else \
            gls.ToeplitzNoise(self.coeffs, self.e.det_offsets, self.chunk, self.inv_var)
        S = gls.System(self.pix, self.psi, self.solver, self.e.npix, noise, min_hits={3: 3, 2: 2, 1: 1}[self.solver],
                       trig=self.trig)
        x, _ = gls.gls_map(S, self.tod.astype(np.float64), tol=1e-13, maxiter=3000)
        return x, S.mask


def wait(L, srv, t, timeout_s=120):
    t0 = time.time()
    while True:
        st, res = L.bm_serve_poll(srv, t, 200)
        if st == L.BM_OK:
            return res
        assert st == L.BM_ERR_TIMEOUT
        assert time.time() - t0 < timeout_s, "request did not finish"


def test_mixed_requests_equal_alone(L, ctx):
    reqs = [Req(L, 16, 4, 30_000, 71), Req(L, 32, 9, 20_000, 72, noise="toeplitz"),
            Req(L, 8, 4, 25_000, 73, solver=2), Req(L, 16, 16, 8_000, 74, noise="toeplitz", trig=False),
            Req(L, 64, 25, 12_000, 75)]
    srv = L.bm_serve_create(ctx, 8 << 30, 3)
    try:
        keep = [r.request(L) for r in reqs]
        tickets = [L.bm_serve_submit(srv, rq) for rq, _ in keep]
        results = [wait(L, srv, t) for t in tickets]
        for r, res in zip(reqs, results):
            assert res["status"] == L.BM_OK, res
            assert res["rel_residual"] <= 1e-7
            st, alone = r.solve_alone(L, ctx)
            assert st == L.BM_OK
            assert torch.equal(torch.nan_to_num(r.out), torch.nan_to_num(alone))  # same map alone and in the mix
        # and the served maps match the oracle (mixed precision to 1e-7 residual)
        for r in (reqs[0], reqs[1]):
            ref, mask = r.oracle()
            xh = r.out.cpu().numpy().reshape(r.e.npix, r.solver)
            err = gls.rel_err(xh, ref, mask)
            assert max(err.values()) < 1e-6, err
        st = L.bm_serve_get_stats(srv)
        assert st["completed"] == len(reqs) and st["rejected"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"]
        assert st["peak_reserved_bytes"] <= st["budget_bytes"]
    finally:
        L.bm_serve_destroy(srv)


def test_budget_admission_serialises(L, ctx):
    a, b = Req(L, 16, 4, 40_000, 81), Req(L, 16, 4, 40_000, 82)
    ka, kb = a.request(L), b.request(L)
    # a budget that holds one of these requests but not two
    one = 60 * 160_000 + 3072 * 600 + (64 << 20)
    srv = L.bm_serve_create(ctx, int(one * 1.5), 4)
    try:
        ta, tb = L.bm_serve_submit(srv, ka[0]), L.bm_serve_submit(srv, kb[0])
        ra, rb = wait(L, srv, ta), wait(L, srv, tb)
        assert ra["status"] == L.BM_OK and rb["status"] == L.BM_OK
        # b could only start after a released its memory
        assert rb["queue_ms"] >= ra["run_ms"] * 0.5
        assert L.bm_serve_get_stats(srv)["peak_reserved_bytes"] <= int(one * 1.5)
    finally:
        L.bm_serve_destroy(srv)


def test_reject_cancel_timeout_unknown(L, ctx):
    big, small = Req(L, 16, 4, 40_000, 91), Req(L, 8, 2, 5_000, 92)
    kb, ks = big.request(L), small.request(L)
    srv = L.bm_serve_create(ctx, 1 << 20, 1)  # 1 MiB: nothing fits
    try:
        with pytest.raises(L.BrahmapError) as ei:
            L.bm_serve_submit(srv, kb[0])
        assert ei.value.status == L.BM_ERR_BUSY
        assert L.bm_serve_get_stats(srv)["rejected"] == 1
    finally:
        L.bm_serve_destroy(srv)
    srv = L.bm_serve_create(ctx, 8 << 30, 1)
    try:
        t1 = L.bm_serve_submit(srv, kb[0])
        t2 = L.bm_serve_submit(srv, ks[0])
        st = L.bm_serve_cancel(srv, t2)
        assert st in (L.BM_OK, L.BM_ERR_BUSY)
        if st == L.BM_OK:
            s2, r2 = L.bm_serve_poll(srv, t2, 1000)
            assert s2 == L.BM_OK and r2["status"] == L.BM_ERR_NOT_FOUND
        r1 = wait(L, srv, t1)
        assert r1["status"] == L.BM_OK
        assert L.bm_serve_poll(srv, t1, 0)[0] == L.BM_ERR_NOT_FOUND  # released
        assert L.bm_serve_poll(srv, 123456789, 0)[0] == L.BM_ERR_NOT_FOUND
    finally:
        L.bm_serve_destroy(srv)


def test_concurrent_submitters(L, ctx):
    reqs = [Req(L, 8, 4, 6_000, 100 + i) for i in range(6)]
    keep = [r.request(L) for r in reqs]
    srv = L.bm_serve_create(ctx, 8 << 30, 4)
    tickets = [None] * len(reqs)
    try:
        def submit(i):
            tickets[i] = L.bm_serve_submit(srv, keep[i][0])
        th = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert len(set(tickets)) == len(reqs)
        for r, t in zip(reqs, tickets):
            res = wait(L, srv, t)
            assert res["status"] == L.BM_OK
            st, alone = r.solve_alone(L, ctx)
            assert torch.equal(torch.nan_to_num(r.out), torch.nan_to_num(alone))
    finally:
        L.bm_serve_destroy(srv)
