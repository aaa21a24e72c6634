"""Shared set-up for the GPU parity tests: one seeded synthetic case, the
oracle's FP64 system on the host, and the library's handles on the device
built from the same inputs."""
from __future__ import annotations

import numpy as np

import synth
from oracle import gls

MIN_HITS = {3: 3, 2: 2, 1: 1}


def stokes_cols(solver):
    return {3: [0, 1, 2], 2: [1, 2], 1: [0]}[solver]


class Case:
    def __init__(self, L, ctx, nside, ndet, ns, seed, solver=3, noise="white", chunk=None, nlags=None,
                 fknee=0.1, flag=0.0, tod_dtype=np.float64, psi_dtype=np.float64, noiseless=False,
                 max_cond=1e3, build_oracle=True, trig=False):
        import torch
        self.L, self.ctx = L, ctx
        self.solver, self.noise_kind = solver, noise
        self.e = e = synth.make_experiment(nside, ndet, ns, seed)
        pt = synth.pointing(e, flag_frac=flag)
        self.pix = pt["pix"]
        self.psi = pt["psi"].astype(psi_dtype)
        sky = synth.sky_map(e.npix, seed)
        if solver == 2:
            sky[:, 0] = 0
        if solver == 1:
            sky[:, 1:] = 0
        self.sky = sky
        extra = None
        if noise == "white":
            self.coeffs = None
        else:
            self.coeffs = synth.toeplitz_band(e.sigma, fknee, 1.0, 20.0, max(chunk, 2 * nlags), nlags)
            if not noiseless:
                extra = synth.one_over_f_noise(e, chunk, fknee, 1.0)
        self.chunk = chunk
        self.trig = synth.trig32(self.psi.astype(np.float64)) if trig else None
        self.tod = synth.tod(e, self.pix, self.psi.astype(np.float64), sky, solver=solver,
                             white=(not noiseless) and noise == "white", extra=extra, dtype=tod_dtype,
                             trig=self.trig)
        inv_var = 1.0 / e.sigma ** 2
        if noise == "white":
            self.onoise = gls.WhiteNoise(inv_var, e.det_offsets)
        else:
            self.onoise = gls.ToeplitzNoise(self.coeffs, e.det_offsets, chunk, inv_var)
        self.S = None
        if build_oracle:
            self.S = gls.System(self.pix, self.psi.astype(np.float64), solver, e.npix, self.onoise,
                                min_hits=MIN_HITS[solver], max_cond=max_cond, trig=self.trig)
        # device
        dev = torch.device("cuda:0")
        self.d_pix = torch.from_numpy(self.pix).to(dev)
        self.d_psi = torch.from_numpy(np.ascontiguousarray(self.psi)).to(dev)
        self.d_tod = torch.from_numpy(np.ascontiguousarray(self.tod)).to(dev)
        if trig:
            self.p = L.bm_pointing_create_trig(ctx, e.npix, self.d_pix, torch.from_numpy(self.trig[0]).to(dev),
                                               torch.from_numpy(self.trig[1]).to(dev), solver)
        else:
            self.p = L.bm_pointing_create(ctx, e.npix, self.d_pix, self.d_psi, solver)
        if noise == "white":
            self.n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, inv_var)
        else:
            self.n = L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, chunk, self.coeffs, inv_var)
        self.pc = L.bm_blockdiag_precond_create(self.p, self.n, MIN_HITS[solver], max_cond)
        self.nc = solver
        self.npix = e.npix

    def vec(self, a=None, dtype=None):
        import torch
        if a is None:
            return torch.zeros(self.npix * self.nc, dtype=torch.float64, device="cuda")
        return torch.from_numpy(np.ascontiguousarray(a, np.float64).ravel()).cuda()

    def mask(self):
        import torch
        m = torch.zeros(self.npix, dtype=torch.uint8, device="cuda")
        self.L.bm_precond_get_mask(self.pc, m, None)
        return m.cpu().numpy().astype(bool)

    def close(self):
        self.L.bm_precond_destroy(self.pc)
        self.L.bm_inv_noise_destroy(self.n)
        self.L.bm_pointing_destroy(self.p)
