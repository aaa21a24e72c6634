"""One rank of a detector-sharded solve through the library (run by
tests/test_gpu_sharded.py as a child process): gloo process group on
127.0.0.1, the library context made a shard by bm_context_set_allreduce with
the binding's torch.distributed reduction, this rank's detectors only.  Rank
0 saves what every rank computed identically (maps, A x, b, mask, hits).

usage: python shard_worker.py RANK WORLD PORT CASE OUT.npz
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]


def case_inputs(case):
    """The full seeded inputs of a case (every rank builds them and keeps its
    detectors' slice)."""
    import synth
    if case == "white":
        e = synth.make_experiment(16, 4, 65_536, 2024)
        pt = synth.pointing(e, flag_frac=0.01)
        c32, s32 = synth.trig32(pt["psi"])
        tod = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 2024), dtype=np.float32, trig=(c32, s32))
        return dict(e=e, pix=pt["pix"], psi=pt["psi"], c32=c32, s32=s32, tod=tod, coeffs=None, chunk=None)
    e = synth.make_experiment(8, 4, 16_384, 2025)
    pt = synth.pointing(e, flag_frac=0.01)
    chunk, nlags = 4096, 64
    coeffs = synth.toeplitz_band(e.sigma, 0.1, 1.0, 20.0, chunk, nlags)
    extra = synth.one_over_f_noise(e, chunk, 0.1, 1.0)
    tod = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, 2025), white=False, extra=extra,
                    dtype=np.float64)
    return dict(e=e, pix=pt["pix"], psi=pt["psi"], c32=None, s32=None, tod=tod, coeffs=coeffs, chunk=chunk)


def solve(L, ctx, inp, d0, d1, sub_off):
    """Handles over detectors [d0, d1) (all of them for an unsharded run),
    the maps, one matvec per precision and the RHS; returns a dict of host
    arrays."""
    import torch
    e = inp["e"]
    s0, s1 = int(e.det_offsets[d0]), int(e.det_offsets[d1])
    dev = torch.device("cuda:0")
    pix = torch.from_numpy(inp["pix"][s0:s1]).to(dev)
    inv_var = (1.0 / e.sigma ** 2)[d0:d1]
    out = {}
    if inp["coeffs"] is None:
        c = torch.from_numpy(inp["c32"][s0:s1]).to(dev)
        s = torch.from_numpy(inp["s32"][s0:s1]).to(dev)
        tod = torch.from_numpy(inp["tod"][s0:s1]).to(dev)
        p = L.bm_pointing_create_with_tod(ctx, e.npix, pix, tod, cos2psi=c, sin2psi=s)
        n = L.bm_inv_noise_create_diag(ctx, sub_off, inv_var)
    else:
        p = L.bm_pointing_create(ctx, e.npix, pix, torch.from_numpy(inp["psi"][s0:s1]).to(dev), 3)
        tod = torch.from_numpy(inp["tod"][s0:s1]).to(dev)
        n = L.bm_inv_noise_create_toeplitz(ctx, sub_off, inp["chunk"], inp["coeffs"][d0:d1], inv_var)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    mask = torch.zeros(e.npix, dtype=torch.uint8, device=dev)
    hits = torch.zeros(e.npix, dtype=torch.int32, device=dev)
    L.bm_precond_get_mask(pc, mask, hits)
    out["mask"], out["hits"] = mask.cpu().numpy(), hits.cpu().numpy()
    x = torch.from_numpy(np.random.default_rng(9).normal(size=e.npix * 3)).to(dev)
    for name, prec in (("fp64", L.BM_PREC_FP64), ("mixed", L.BM_PREC_MIXED)):
        q = torch.zeros(e.npix * 3, dtype=torch.float64, device=dev)
        L.bm_matvec(p, n, pc, x, q, prec)
        out["q_" + name] = q.cpu().numpy()
        m = torch.zeros(e.npix * 3, dtype=torch.float64, device=dev)
        st, info = L.bm_pcg_solve(p, n, pc, tod, 1, m, 1e-12 if prec == L.BM_PREC_FP64 else 1e-9, 500, prec)
        assert st == L.BM_OK, (name, st, info)
        out["map_" + name] = m.cpu().numpy()
        out["iters_" + name] = np.array([info[0]["iterations"]])
    b = torch.zeros(e.npix * 3, dtype=torch.float64, device=dev)
    L.bm_rhs(p, n, pc, tod, 1, b)
    out["b"] = b.cpu().numpy()
    if inp["coeffs"] is None:  # the TOD carried through the sort (its b summed with the blocks)
        m = torch.zeros(e.npix * 3, dtype=torch.float64, device=dev)
        st, info = L.bm_pcg_solve(p, n, pc, None, 1, m, 1e-8, 500, L.BM_PREC_MIXED)
        assert st == L.BM_OK
        out["map_carried"] = m.cpu().numpy()
    y = torch.from_numpy(np.random.default_rng(10).normal(size=e.nsamples)[s0:s1].copy()).to(dev)
    xt = torch.zeros(e.npix * 3, dtype=torch.float64, device=dev)
    L.bm_pointing_apply_transpose(p, y, xt)
    out["pt_y"] = xt.cpu().numpy()
    L.bm_precond_destroy(pc)
    L.bm_inv_noise_destroy(n)
    L.bm_pointing_destroy(p)
    return out


def main():
    rank, world, port, case, path = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), sys.argv[4], sys.argv[5]
    import torch
    import torch.distributed as dist
    from paper_2501_16122_gb300 import _lib as L
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = case_inputs(case)
        d0, d1, sub_off = L.detector_shard(inp["e"].det_offsets, rank, world)
        ctx = L.bm_context_create(0)
        L.bm_context_set_allreduce(ctx, L.torch_allreduce())
        out = solve(L, ctx, inp, d0, d1, sub_off)
        L.bm_context_destroy(ctx)
        if rank == 0:
            np.savez(path, **out)
    finally:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
