"""bm_matvec_white_static: the white-noise FP32-product matvec for callers
that cannot allocate device memory while it runs.  It must give the same q as
the allocating entry point bm_matvec(..., BM_PREC_MIXED), call after call
(the fixed scratch array keeps the previous call's contents).  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

from gpucase import Case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-6  # the tolerance the mixed-precision matvec parity tests use


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


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_static_scratch_matvec_matches_bm_matvec(L, ctx, solver):
    c = Case(L, ctx, 16, 4, 65_536 + 321, 5000 + solver, solver=solver, flag=0.01, build_oracle=False)
    try:
        rng = np.random.default_rng(solver)
        m = c.mask()
        for call in range(2):  # two calls in a row: the shared array is reused
            x = c.vec(rng.normal(size=(c.npix, solver)) * 50.0)
            ref = c.vec()
            L.bm_matvec(c.p, c.n, c.pc, x, ref, L.BM_PREC_MIXED)
            q = torch.full_like(ref, float("nan"))
            L.bm_matvec_white_static(c.p, c.n, c.pc, x, q)
            qh, rh = q.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(qh))
            for k in range(solver):
                assert rel(qh[k::solver], rh[k::solver]) <= TOL, (call, k)
            assert np.all(qh.reshape(c.npix, solver)[m] == 0)
    finally:
        c.close()


def test_static_scratch_rejects_toeplitz_noise(L, ctx):
    c = Case(L, ctx, 8, 2, 4096, 7, noise="toeplitz", chunk=1024, nlags=16, build_oracle=False)
    try:
        with pytest.raises(L.BrahmapError) as ei:
            L.bm_matvec_white_static(c.p, c.n, c.pc, c.vec(), c.vec())
        assert ei.value.status == L.BM_ERR_INVALID
    finally:
        c.close()
