"""bm_matvec_white_static: the white-noise FP32-product matvec for callers
that cannot allocate device memory while it runs (a process whose free
device memory already belongs to another allocator, or a pipeline that fixes
its memory budget before it starts).  It runs the same kernels as the
allocating entry point bm_matvec(..., BM_PREC_MIXED), so the two must give
the same bits, call after call (the fixed scratch array keeps the previous
call's contents), and both must match the oracle's FP64 operator within the
mixed-precision tolerance.  Its first call after bm_context_create must not
change the device's free memory.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from gpucase import Case, MIN_HITS
from oracle import gls

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 2e-6  # the mixed-precision matvec's tolerance against the FP64 operator
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def check_static_equals_matvec(L, p, n, pc, npix, nc, S, seed):
    """Two calls in a row: bitwise equal to bm_matvec(MIXED), within the mixed
    tolerance of the oracle's operator, exact zeros on masked pixels."""
    rng = np.random.default_rng(seed)
    dm = torch.zeros(npix, dtype=torch.uint8, device="cuda")
    L.bm_precond_get_mask(pc, dm, None)
    m = dm.cpu().numpy().astype(bool)
    for call in range(2):  # the shared array is reused by the second call
        xh = rng.normal(size=(npix, nc)) * 50.0
        x = torch.from_numpy(xh.ravel()).cuda()
        ref = torch.zeros(npix * nc, dtype=torch.float64, device="cuda")
        L.bm_matvec(p, n, pc, x, ref, L.BM_PREC_MIXED)
        q = torch.full_like(ref, float("nan"))
        L.bm_matvec_white_static(p, n, pc, x, q)
        qh, rh = q.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(qh.view(np.uint64), rh.view(np.uint64)), f"call {call}: not bitwise equal"
        assert np.all(qh.reshape(npix, nc)[m] == 0)
        if S is not None:
            want = S.matvec(xh).reshape(npix, nc)
            got = qh.reshape(npix, nc)
            for k in range(nc):
                assert rel(got[~m, k], want[~m, k]) <= TOL_MIXED, (call, k)


@pytest.mark.parametrize("solver", [3, 2, 1])
def test_static_matvec_bitwise_on_a_scan(L, ctx, solver):
    c = Case(L, ctx, 16, 4, 65_536 + 321, 5000 + solver, solver=solver, flag=0.01, trig=True)
    try:
        check_static_equals_matvec(L, c.p, c.n, c.pc, c.npix, solver, c.S, solver)
    finally:
        c.close()


@pytest.mark.parametrize("solver", [3, 1])
def test_static_matvec_bitwise_full_work_items(L, ctx, solver):
    """12 pixels with ~16,700 samples each: every pixel has four work items
    of the full 4096 samples and a ragged one."""
    rng = np.random.default_rng(77 + solver)
    npix, ndet, ns = 12, 4, 50_000
    pix = rng.integers(0, npix, ndet * ns).astype(np.int32)
    psi = rng.uniform(0.0, np.pi, ndet * ns)
    c32, s32 = synth.trig32(psi)
    det_off = np.arange(ndet + 1, dtype=np.int64) * ns
    inv_var = 1.0 / rng.uniform(1.0, 2.0, ndet) ** 2
    S = gls.System(pix, psi, solver, npix, gls.WhiteNoise(inv_var, det_off), min_hits=MIN_HITS[solver],
                   max_cond=1e3, trig=(c32, s32))
    assert np.bincount(pix, minlength=npix).min() > 4 * 4096
    p = L.bm_pointing_create_trig(ctx, npix, torch.from_numpy(pix).cuda(), torch.from_numpy(c32).cuda(),
                                  torch.from_numpy(s32).cuda(), solver)
    n = L.bm_inv_noise_create_diag(ctx, det_off, inv_var)
    pc = L.bm_blockdiag_precond_create(p, n, MIN_HITS[solver], 1e3)
    try:
        check_static_equals_matvec(L, p, n, pc, npix, solver, S, 11)
    finally:
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)


def test_static_matvec_bitwise_sample_weights(L, ctx):
    """A weight per sample (15 % zeros), the other diagonal N^-1."""
    e = synth.make_experiment(16, 4, 32_768, 4242)
    pt = synth.pointing(e, flag_frac=0.01)
    rng = np.random.default_rng(4242)
    w = (1.0 / e.sigma ** 2)[np.repeat(np.arange(4), 32_768)] * rng.uniform(0.3, 3.0, e.nsamples)
    w = np.where(rng.random(e.nsamples) < 0.15, 0.0, w)
    S = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.SampleWeightNoise(w), min_hits=3, max_cond=1e3)
    p = L.bm_pointing_create(ctx, e.npix, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(pt["psi"]).cuda(), 3)
    n = L.bm_inv_noise_create_sample_weights(ctx, torch.from_numpy(w).cuda())
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    try:
        check_static_equals_matvec(L, p, n, pc, e.npix, 3, S, 5)
    finally:
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)


def test_static_matvec_rejects_more_than_its_scratch(L, ctx):
    """I-only, nside 512: 3,145,728 one-sample work items > 2^21 values."""
    npix = 12 * 512 ** 2
    pix = torch.arange(npix, dtype=torch.int32, device="cuda")
    psi = torch.zeros(npix, dtype=torch.float64, device="cuda")
    p = L.bm_pointing_create(ctx, npix, pix, psi, 1)
    n = L.bm_inv_noise_create_diag(ctx, np.array([0, npix], np.int64), np.array([0.25]))
    pc = L.bm_blockdiag_precond_create(p, n, 1, 1e3)
    try:
        x = torch.ones(npix, dtype=torch.float64, device="cuda")
        q = torch.zeros_like(x)
        with pytest.raises(L.BrahmapError) as ei:
            L.bm_matvec_white_static(p, n, pc, x, q)
        assert ei.value.status == L.BM_ERR_INVALID
        L.bm_matvec(p, n, pc, x, q, L.BM_PREC_MIXED)  # the allocating entry point takes it
        assert torch.all(q == 0.25)
    finally:
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)


def test_static_matvec_rejects_toeplitz_noise(L, ctx):
    c = Case(L, ctx, 8, 2, 4096, 7, noise="toeplitz", chunk=1024, nlags=16, build_oracle=False)
    try:
        with pytest.raises(L.BrahmapError) as ei:
            L.bm_matvec_white_static(c.p, c.n, c.pc, c.vec(), c.vec())
        assert ei.value.status == L.BM_ERR_INVALID
    finally:
        c.close()


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path[:0] = [ROOT, ROOT + "/tests"]
from paper_2501_16122_gb300 import _lib as L
from gpucase import Case
ctx = L.bm_context_create(0)
c = Case(L, ctx, 16, 4, 65_536, 31, trig=True, build_oracle=False)
x = c.vec(np.random.default_rng(1).normal(size=(c.npix, 3)))
q = c.vec()
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
L.bm_matvec_white_static(c.p, c.n, c.pc, x, q)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
L.bm_matvec_white_static(c.p, c.n, c.pc, x, q)
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info()[0]
print("FREE", free0, free1, free2)
c.close()
L.bm_context_destroy(ctx)
"""


def test_static_matvec_first_call_maps_no_memory(L):
    """In a fresh process (the library loaded there for the first time), the
    device's free memory is the same before and after the first and second
    calls made after bm_context_create."""
    code = _FRESH.replace("ROOT", repr(ROOT), 2)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [s for s in r.stdout.splitlines() if s.startswith("FREE")][-1]
    free0, free1, free2 = (int(v) for v in line.split()[1:])
    assert free0 == free1 == free2, (free0, free1, free2)
