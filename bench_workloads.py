"""Benchmark workloads other than the default one of bench.py (config 1).

  config0  nside 16, 4 detectors x 65,536 samples, FP64 inputs, white noise,
           tol 1e-10: time-to-map of the FP64 and mixed paths (launch-bound).
  config2  the config-1 scan with 1/f noise and the 512-lag banded Toeplitz
           N^-1 per 2^20-sample chunk: mixed-precision PCG, FP32 filter.
  config3  nside 512, 64 detectors x 2^22 samples, 64 right-hand sides
           sharing one pointing: one batched solve vs one-at-a-time solves.
  config4  Poisson arrivals of requests of mixed size and noise model through
           the serving loop: p50/p99 latency and throughput.
  hwp      the config-1 scan with its angle rebuilt on the device from the
           half-wave-plate model (bm_pointing_create_hwp): the whole step and
           the matvec that reads 4 bytes a sample, beside the stored-trig one.

Each prints one JSON line.  Large TODs are synthesised on the device from the
seeded pointing (signal gathered from a seeded sky, noise from a seeded torch
generator) because host generation of 10^10 samples would dominate the run.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

import synth
from bench import METRIC, ClockSampler, peaks


def _L():
    from paper_2501_16122_gb300 import _lib
    return _lib


# ---------------------------------------------------------- device synthesis
def device_signal(d_pix, d_c, d_s, sky, out, step=1 << 26):
    """out[t] = I + Q cos + U sin at the pixel of t (0 for flagged); FP64 sums, FP32 out."""
    import torch
    n = d_pix.numel()
    for a in range(0, n, step):
        p = d_pix[a:a + step].long()
        valid = p >= 0
        pc = p.clamp(min=0)
        v = sky[pc, 0] + sky[pc, 1] * d_c[a:a + step].double() + sky[pc, 2] * d_s[a:a + step].double()
        out[a:a + step] = torch.where(valid, v, torch.zeros_like(v)).float()


def device_white(out, sigma, ns, gen):
    import torch
    for d, sg in enumerate(sigma):
        out[d * ns:(d + 1) * ns] += float(sg) * torch.randn(ns, generator=gen, device=out.device)


def device_one_over_f(out, sigma, ns, chunk, fknee, alpha, fs, gen):
    """Noise with spectrum sigma_d^2 (1 + (fknee/f)^alpha), shaped per chunk in
    the Fourier domain (a ragged last chunk takes the head of a full one)."""
    import torch
    f = torch.fft.rfftfreq(chunk, 1.0 / fs, device=out.device, dtype=torch.float64)
    g = torch.empty_like(f)
    g[1:] = torch.sqrt(1.0 + (fknee / f[1:]) ** alpha)
    g[0] = g[1]
    g = g.float()
    nch = -(-ns // chunk)
    for d, sg in enumerate(sigma):
        w = torch.randn(nch, chunk, generator=gen, device=out.device) * float(sg)
        n = torch.fft.irfft(torch.fft.rfft(w, dim=1) * g, n=chunk, dim=1).reshape(-1)
        out[d * ns:(d + 1) * ns] += n[:ns]


def pointing_on_device(nside, ndet, ns, seed):
    import torch
    e = synth.make_experiment(nside, ndet, ns, seed)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    return e, torch.from_numpy(pt["pix"]).cuda(), torch.from_numpy(c32).cuda(), torch.from_numpy(s32).cuda()


def fp32_nominal_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp64_nominal_tflops(sm_mhz):
    # 1.25 TFLOP/s dense FP64 at the maximum SM clock (2070 MHz), scaled by the clock
    return 1.25 * sm_mhz / 2070.0


def measured_fma_tflops(L, ctx):
    """FP32 and FP64 FMA rates measured on this GPU by the library's own
    microbenchmark (bm_measure_fma_peak), in TFLOP/s."""
    return (L.bm_measure_fma_peak(ctx, L.BM_F32) / 1e12, L.bm_measure_fma_peak(ctx, L.BM_F64) / 1e12)


def hbm_peak():
    return peaks()[0]


def fft_size(L, chunk_len, cap):
    """The library's FFT length for an L-lag band (smallest power of two with
    H = N - 2(L-1) >= N/2, grown toward a whole chunk, at most cap; 0: direct)."""
    if L < 32:
        return 0
    N = 64
    while N < 4 * (L - 1):
        N <<= 1
    while N < cap and N < chunk_len + 2 * (L - 1):
        N <<= 1
    return N if N <= cap else 0


# ------------------------------------------------------------------ config 0
def run_config0(args):
    import torch
    from oracle import gls
    L = _L()
    e = synth.make_experiment(16, 4, 65_536, 1000)
    pt = synth.pointing(e)
    sky = synth.sky_map(e.npix, 1000)
    tod = synth.tod(e, pt["pix"], pt["psi"], sky)
    ctx = L.bm_context_create(0)
    d_pix, d_psi, d_tod = (torch.from_numpy(a).cuda() for a in (pt["pix"], pt["psi"], tod))
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    S = gls.System(pt["pix"], pt["psi"], 3, e.npix, gls.WhiteNoise(1 / e.sigma ** 2, e.det_offsets))
    ref, _ = gls.gls_map(S, tod, tol=1e-13)
    res = {}
    for name, prec in (("fp64", L.BM_PREC_FP64), ("mixed", L.BM_PREC_MIXED)):
        def step():
            p = L.bm_pointing_create(ctx, e.npix, d_pix, d_psi, 3)
            n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, 1 / e.sigma ** 2)
            pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
            st, info = L.bm_pcg_solve(p, n, pc, d_tod, 1, out, 1e-10, 100, prec)
            for h, f in ((pc, L.bm_precond_destroy), (n, L.bm_inv_noise_destroy), (p, L.bm_pointing_destroy)):
                f(h)
            return info[0]
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        l0 = L.bm_kernel_launches()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            info = step()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1000 / args.steps
        err = gls.rel_err(out.cpu().numpy().reshape(e.npix, 3), ref, S.mask)
        res[name] = {"ms_per_solve": ms, "launches_per_solve": (L.bm_kernel_launches() - l0) / args.steps,
                     "iterations": info["iterations"], "rel_residual": info["rel_residual"],
                     "max_rel_err_vs_oracle": max(err.values())}
    L.bm_context_destroy(ctx)
    print(json.dumps({"workload": "config0", "metric": "time-to-map (ms), host wall clock, incl. ingest",
                      "nsamples": e.nsamples, "npix": e.npix, "steps": args.steps, "results": res}), flush=True)


# ------------------------------------------------------------------ config 2
def run_config2(args, noise="toeplitz"):
    """The correlated-noise solve: a 512-lag Toeplitz N^-1 (noise = "toeplitz"),
    or white N^-1 with a baseline offset per 60 s interval marginalised out
    (noise = "offsets"), on the same 1/f TOD."""
    import torch
    L = _L()
    nside, ndet, ns = args.nside, args.ndet, args.ns
    chunk, nlags, fknee, alpha = 2 ** 20, 512, 0.1, 1.0
    baseline_len = 1200  # 60 s at 20 Hz
    chunk = min(chunk, ns)
    tol = 1e-7
    t_gen = time.perf_counter()
    e, d_pix, d_c, d_s = pointing_on_device(nside, ndet, ns, args.seed + 1)
    gen = torch.Generator(device="cuda").manual_seed(args.seed + 1)
    sky = torch.from_numpy(synth.sky_map(e.npix, args.seed + 1)).cuda()
    d_tod = torch.empty(e.nsamples, dtype=torch.float32, device="cuda")
    device_signal(d_pix, d_c, d_s, sky, d_tod)
    device_one_over_f(d_tod, e.sigma, ns, chunk, fknee, alpha, 20.0, gen)
    coeffs = synth.toeplitz_band(e.sigma, fknee, alpha, 20.0, chunk, nlags)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    ctx = L.bm_context_create(0)
    fp32_tf, fp64_tf = measured_fma_tflops(L, ctx)
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    inv_var = 1 / e.sigma ** 2
    infos = []

    def make():
        p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, d_c, d_s, 3)
        if noise == "toeplitz":
            n = L.bm_inv_noise_create_toeplitz(ctx, e.det_offsets, chunk, coeffs, inv_var)
        else:
            n = L.bm_inv_noise_create_offset_filter(ctx, e.det_offsets, inv_var, baseline_len)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        return p, n, pc

    def free(h):
        p, n, pc = h
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)

    def step():
        h = make()
        st, info = L.bm_pcg_solve(h[0], h[1], h[2], d_tod, 1, out, tol, 3000, L.BM_PREC_MIXED)
        infos.append((st, info[0]))
        free(h)

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(0)
    sampler.start()
    L.bm_context_set_timing(ctx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000 / args.steps
    clocks = sampler.stop()
    fam = {}
    for name in ("ingest", "blocks", "rhs", "toeplitz_f32", "toeplitz_px", "toeplitz_refine", "toeplitz_px_df",
                 "toeplitz_f64", "toeplitz_pt", "toeplitz_pt_df", "toeplitz_pt_bounds", "offset_filter_f64",
                 "offset_means_f32",
                 "offset_matvec_f32", "offset_means_df", "offset_pt_df", "ingest_validate", "ingest_hist",
                 "ingest_scatter"):
        tot, cnt = L.bm_context_kernel_time(ctx, name)
        if cnt:
            fam[name] = {"ms_per_launch": tot / cnt, "launches_per_step": cnt / args.steps}
    # one FP64 matvec, and the solve alone (RHS + PCG on handles already
    # built) in both precisions: the plain FP64 solve against the refined
    # mixed-precision one, to the same tolerance
    L.bm_context_set_timing(ctx, False)
    h = make()
    x = torch.nan_to_num(out)
    q = torch.empty_like(x)
    L.bm_matvec(h[0], h[1], h[2], x, q, L.BM_PREC_FP64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.bm_matvec(h[0], h[1], h[2], x, q, L.BM_PREC_FP64)
    torch.cuda.synchronize()
    fp64_mv_ms = (time.perf_counter() - t1) * 1000
    solve_only = {}
    if not args.no_fp64_solve:
        for name, prec in (("mixed", L.BM_PREC_MIXED), ("fp64", L.BM_PREC_FP64)):
            o = torch.zeros_like(out)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            st_s, inf_s = L.bm_pcg_solve(h[0], h[1], h[2], d_tod, 1, o, tol, 3000, prec, raise_on_error=False)
            torch.cuda.synchronize()
            solve_only[name] = {"ms": (time.perf_counter() - t1) * 1000, "status": st_s,
                                "iterations": inf_s[0]["iterations"],
                                "outer_iterations": inf_s[0]["outer_iterations"],
                                "rel_residual": inf_s[0]["rel_residual"]}
            if name == "mixed":
                o_mixed = o
            else:  # the two maps agree on observed pixels
                m = torch.isfinite(o_mixed) & torch.isfinite(o)
                solve_only["mixed_vs_fp64_rel_l2"] = float(torch.linalg.norm(o_mixed[m] - o[m]) /
                                                           torch.linalg.norm(o[m]))
            del o
        if "fp64" in solve_only:
            solve_only["fp64_over_mixed"] = solve_only["fp64"]["ms"] / solve_only["mixed"]["ms"]
    free(h)
    L.bm_context_set_timing(ctx, False)
    L.bm_context_destroy(ctx)
    st, info = infos[-1]
    sm = clocks["sm_mhz"] if clocks else 2070.0
    if noise == "offsets":
        # dominant family of the inner operator: the time-ordered means pass
        # (pix 4 + FP32 trig 8 per sample; the map gathers hit L2)
        of = fam.get("offset_means_f32", {})
        ms_l = of.get("ms_per_launch")
        gbs = e.nsamples * 12.0 / (ms_l * 1e-3) / 1e9 if ms_l else None
        line = {
            "workload": "offsets", "metric": METRIC, "value": e.nsamples / (ms * 1e-3), "unit": "TOD samples/s",
            "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"GLS map-making, nside {nside}, {ndet} det x {ns} samples, 1/f noise "
                                   f"(fknee {fknee} Hz, alpha {alpha}), white N^-1 with one offset per "
                                   f"{baseline_len}-sample baseline marginalised out, mixed precision PCG to {tol:g}",
                       "nsamples": e.nsamples},
            "solve": {"status": st, **info},
            "step_breakdown": fam,
            "fp64_matvec_ms": fp64_mv_ms,
            "roofline": {"bound": "hbm", "kernel": "offset_means_f32_kernel (pix + FP32 trig: 12 B a sample)",
                         "achieved": gbs, "peak": hbm_peak(), "unit": "GB/s",
                         "frac": gbs / hbm_peak() if gbs else None, "traffic": None},
            "clocks": clocks, "input_generation_s": t_gen,
        }
        print(json.dumps(line), flush=True)
        return
    # The band is applied by FFT overlap-save: per tile of H = N - 2(L-1)
    # outputs one real N-point transform pair (5 N log2 N flops) and the
    # spectrum product (2N); it reads the window of y = P x (4 B FP32, 8 B
    # double-float or FP64 per input sample) and writes z (4 B / 8 B).  The
    # FP32 and double-float families also hold the P x pass (timed on its
    # own as toeplitz_px / toeplitz_px_df: pix + trig read, y written, 16 B
    # a sample FP32 and 28 B double-float), which is taken out of the
    # transform's time here.
    def fft_tiles(N):
        H = N - 2 * (nlags - 1)
        per_chunk = -(-chunk // H)
        return per_chunk * (ns // chunk) * ndet, H
    fam_fft = {}
    # (the refinement operator's double-float transform is counted in FP64
    #  flops against the FP32 pipes' rate / 20, about the cost of one
    #  double-float multiply-add)
    for name, px, N, zb, peak, unit in (("toeplitz_f32", "toeplitz_px", fft_size(nlags, chunk, 8192), 4, fp32_tf,
                                         "FP32"),
                                        ("toeplitz_refine", "toeplitz_px_df", fft_size(nlags, chunk, 4096), 8,
                                         fp32_tf / 20, "FP32 double-float"),
                                        ("toeplitz_f64", None, fft_size(nlags, chunk, 4096), 8, fp64_tf, "FP64")):
        ms_l = fam.get(name, {}).get("ms_per_launch")
        if not N or not ms_l:
            continue
        px_ms = fam.get(px, {}).get("ms_per_launch", 0.0) if px else 0.0
        ms_l = ms_l - px_ms
        tiles, H = fft_tiles(N)
        flops = tiles * (5.0 * N * math.log2(N) + 2.0 * N)
        bytes_ = tiles * N * zb + e.nsamples * zb
        fam_fft[name] = {"fft_n": N, "tiles": tiles, "ms_per_launch": ms_l, "px_ms": px_ms,
                         "px_hbm_frac": (e.nsamples * (16 if zb == 4 else 28) / (px_ms * 1e-3) / 1e9 / hbm_peak()
                                         if px_ms else None),
                         "tflops": flops / (ms_l * 1e-3) / 1e12, "peak_tflops": peak, "pipe": unit,
                         "flop_frac": flops / (ms_l * 1e-3) / 1e12 / peak,
                         "gbs": bytes_ / (ms_l * 1e-3) / 1e9, "hbm_frac": bytes_ / (ms_l * 1e-3) / 1e9 / hbm_peak()}
    # the dominant kernel family of the step
    dom = max(("toeplitz_f32", "toeplitz_refine", "toeplitz_f64"),
              key=lambda k: fam.get(k, {}).get("ms_per_launch", 0) * fam.get(k, {}).get("launches_per_step", 0))
    d = fam_fft.get(dom, {})
    line = {
        "workload": "config2", "metric": METRIC, "value": e.nsamples / (ms * 1e-3), "unit": "TOD samples/s",
        "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": f"GLS map-making, nside {nside}, {ndet} det x {ns} samples, 1/f noise "
                               f"(fknee {fknee} Hz, alpha {alpha}), {nlags}-lag Toeplitz N^-1 per {chunk}-sample chunk, "
                               f"mixed precision PCG to {tol:g}", "nsamples": e.nsamples},
        "solve": {"status": st, **info},
        "step_breakdown": fam,
        "fft_filter": fam_fft,
        "fp64_matvec_ms": fp64_mv_ms,
        "solve_only_ms": solve_only,
        "fma_peaks_tflops": {"fp32_measured": fp32_tf, "fp64_measured": fp64_tf,
                             "fp32_nominal": fp32_nominal_tflops(sm), "fp64_nominal": fp64_nominal_tflops(sm)},
        "roofline": {"bound": "alu", "kernel": f"toeplitz_fft_kernel ({dom}, {d.get('pipe')} pipe)",
                     "achieved": d.get("tflops"), "peak": d.get("peak_tflops"), "unit": "TFLOP/s",
                     "frac": d.get("flop_frac"), "traffic": None,
                     "peak_basis": ("measured FMA rate of this GPU (bm_measure_fma_peak); the double-float "
                                    "transform against the FP32 rate / 20")},
        "clocks": clocks, "input_generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ config 3
def run_config3(args):
    import torch
    L = _L()
    nside, ndet, ns, R = 512, 64, 2 ** 22, args.nrhs
    if args.ns != 2 ** 22:
        ns = args.ns
    tol = 1e-8
    t_gen = time.perf_counter()
    e, d_pix, d_c, d_s = pointing_on_device(nside, ndet, ns, args.seed + 2)
    gen = torch.Generator(device="cuda").manual_seed(args.seed + 2)
    nt = e.nsamples
    d_tod = torch.empty((R, nt), dtype=torch.float32, device="cuda")
    for r in range(R):
        sky = torch.randn((e.npix, 3), generator=gen, device="cuda", dtype=torch.float64)
        sky[:, 0] *= 100.0
        sky[:, 1:] *= 10.0
        device_signal(d_pix, d_c, d_s, sky, d_tod[r])
        device_white(d_tod[r], e.sigma, ns, gen)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    ctx = L.bm_context_create(0)
    fp32_tf, _ = measured_fma_tflops(L, ctx)
    inv_var = 1 / e.sigma ** 2
    out = torch.zeros(R * e.npix * 3, dtype=torch.float64, device="cuda")
    one = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")

    def make():
        p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, d_c, d_s, 3)
        n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, inv_var)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        return p, n, pc

    def free(h):
        L.bm_precond_destroy(h[2])
        L.bm_inv_noise_destroy(h[1])
        L.bm_pointing_destroy(h[0])

    h = make()
    # warm-up (includes the autotuner's one-time timing of the batched matvec variants)
    L.bm_pcg_solve(h[0], h[1], h[2], d_tod, R, out, tol, 100, L.BM_PREC_MIXED)
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    l0 = L.bm_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, infos = L.bm_pcg_solve(h[0], h[1], h[2], d_tod, R, out, tol, 100, L.BM_PREC_MIXED)
    torch.cuda.synchronize()
    batched_ms = (time.perf_counter() - t0) * 1000 / args.steps
    launches = (L.bm_kernel_launches() - l0) / args.steps
    clocks = sampler.stop()
    # one more solve with the library's kernel timing on, for the RHS and a
    # batched matvec timed on its own (kept out of the timed solves above:
    # the timing brackets kernels with events and times an extra matvec)
    L.bm_context_set_timing(ctx, True)
    L.bm_pcg_solve(h[0], h[1], h[2], d_tod, R, out, tol, 100, L.BM_PREC_MIXED)
    torch.cuda.synchronize()
    rhs_ms, _ = L.bm_context_kernel_time(ctx, "rhs_batched")
    mv_ms, mv_n = L.bm_context_kernel_time(ctx, "matvec_batched")
    L.bm_context_set_timing(ctx, False)
    # the batched matvec's algorithmic bytes: the weighted trig stream once
    # (8 B a kept sample) for all R right-hand sides, and per kept pixel the
    # R FP32 x values (12 B each) read and the R FP64 results (24 B) written
    hits = torch.empty(e.npix, dtype=torch.int32, device="cuda")
    mask = torch.empty(e.npix, dtype=torch.uint8, device="cuda")
    L.bm_precond_get_mask(h[2], mask, hits)
    kept = mask == 0
    n_kept_s, n_kept_p = int(hits[kept].sum().item()), int(kept.sum().item())
    mv_bytes = 8 * n_kept_s + n_kept_p * R * (12 + 24)
    mv_ms_l = mv_ms / max(mv_n, 1)
    # one right-hand side at a time, mixed and FP64 (timed on two RHS, scaled to R)
    t1 = time.perf_counter()
    for r in range(2):
        L.bm_pcg_solve(h[0], h[1], h[2], d_tod[r].contiguous(), 1, one, tol, 100, L.BM_PREC_MIXED)
    torch.cuda.synchronize()
    single_mixed_ms = (time.perf_counter() - t1) * 1000 / 2
    t1 = time.perf_counter()
    for r in range(2):
        L.bm_pcg_solve(h[0], h[1], h[2], d_tod[r].contiguous(), 1, one, tol, 100, L.BM_PREC_FP64)
    torch.cuda.synchronize()
    single_fp64_ms = (time.perf_counter() - t1) * 1000 / 2
    # agreement of the batched RHS 0 with its one-at-a-time FP64 solve
    L.bm_pcg_solve(h[0], h[1], h[2], d_tod[0].contiguous(), 1, one, 1e-10, 100, L.BM_PREC_FP64)
    a, b = out[:e.npix * 3].cpu().numpy(), one.cpu().numpy()
    keep = ~np.isnan(a)
    agree = float(np.linalg.norm(a[keep] - b[keep]) / np.linalg.norm(b[keep]))
    free(h)
    L.bm_context_destroy(ctx)
    line = {
        "workload": "config3", "metric": "time-to-solution of R right-hand sides sharing one pointing",
        "value": R * nt / (batched_ms * 1e-3), "unit": "TOD sample-RHS/s",
        "config": {"workload": f"nside {nside}, {ndet} det x {ns} samples, R = {R} white-noise realisations, "
                               f"mixed precision PCG to {tol:g}", "nsamples": nt, "nrhs": R},
        "batched_ms": batched_ms, "batched_rhs_ms_per_solve": rhs_ms,
        "one_at_a_time_mixed_ms": single_mixed_ms * R, "one_at_a_time_fp64_ms": single_fp64_ms * R,
        "speedup_vs_fp64_one_at_a_time": single_fp64_ms * R / batched_ms,
        "gpu_launches_per_solve": launches,
        "solve": {"status": st, "max_iterations": max(i["iterations"] for i in infos),
                  "max_rel_residual": max(i["rel_residual"] for i in infos)},
        "rhs0_rel_diff_vs_fp64_solve": agree,
        # the batched matvec streams little (one pointing read for all R) and
        # does ~11 FP32 flops per kept sample and right-hand side: its bound
        # is the FP32 pipe; the HBM fraction is given beside it
        "roofline": {"bound": "alu", "kernel": "batched_matvec_kernel (one pointing read for all R)",
                     "ms_per_launch": mv_ms_l, "flops_per_launch": 11.0 * n_kept_s * R,
                     "achieved": 11.0 * n_kept_s * R / (mv_ms_l * 1e-3) / 1e12 if mv_n else None,
                     "peak": fp32_tf, "unit": "TFLOP/s",
                     "frac": 11.0 * n_kept_s * R / (mv_ms_l * 1e-3) / 1e12 / fp32_tf if mv_n else None,
                     "peak_basis": "measured FP32 FMA rate (bm_measure_fma_peak)",
                     "bytes_per_launch": mv_bytes,
                     "hbm_frac": mv_bytes / (mv_ms_l * 1e-3) / 1e9 / hbm_peak() if mv_n else None,
                     "traffic": None},
        "clocks": clocks, "input_generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ config 4
def run_config4(args):
    import threading
    import torch
    L = _L()
    rng = np.random.default_rng(args.seed + 3)
    pool_ndet, pool_ns = 64, 2 ** 22
    # Per nside a pool of 64 detectors x 2^22 samples: pointing, and TODs
    # (signal of a seeded sky plus white noise, or plus 1/f noise at three
    # knee frequencies spanning [0.05, 0.5] Hz), made before the arrivals so
    # that building a request is a device gather, not a synthesis.
    fk_pool = (0.05, 0.158, 0.5)
    t_gen = time.perf_counter()
    gen = torch.Generator(device="cuda").manual_seed(args.seed + 3)
    pools = {}
    for ns_ in (64, 128, 256, 512):
        e0, pix0, c0, s0 = pointing_on_device(ns_, pool_ndet, pool_ns, args.seed + 3 + ns_)
        sky = torch.randn((e0.npix, 3), generator=gen, device="cuda", dtype=torch.float64)
        sky[:, 0] *= 100.0
        sky[:, 1:] *= 10.0
        sig = torch.empty(e0.nsamples, dtype=torch.float32, device="cuda")
        device_signal(pix0, c0, s0, sky, sig)
        tw = sig.clone()
        device_white(tw, e0.sigma, pool_ns, gen)
        t1f = {}
        for fk in fk_pool:
            t1f[fk] = sig.clone()
            device_one_over_f(t1f[fk], e0.sigma, pool_ns, 2 ** 20, fk, 1.0, 20.0, gen)
        del sig
        pools[ns_] = (e0, pix0, c0, s0, tw, t1f)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen

    # request list: Poisson arrivals; nside U{64..512}; ndet log-U[8, 512]; Ns = 2^U[18, 22]
    arrivals, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / args.rate)
        if t > args.horizon:
            break
        arrivals.append(t)
    # Shared observations (--shared-frac > 0): a few fixed pointings, each
    # drawn like a request but capped at 2^28 samples, whose requests are
    # white-noise Monte Carlo realisations: the observation's TOD (signal
    # plus white noise, gathered from the pool once) plus a fresh white-noise
    # draw per request, submitted with the observation's pointing_key.
    rng_obs = np.random.default_rng(args.seed + 5)
    observations = []
    for j in range(args.observations if args.shared_frac > 0 else 0):
        while True:
            nside = int(rng_obs.choice([64, 128, 256, 512]))
            ndet = int(round(math.exp(rng_obs.uniform(math.log(8), math.log(512)))))
            ns_ = int(2 ** rng_obs.uniform(18, 22)) // 1024 * 1024
            if ndet * ns_ <= 2 ** 28:
                break
        observations.append(dict(nside=nside, ndet=ndet, ns=ns_, key=j + 1))

    reqs = []
    for ta in arrivals:
        nside = int(rng.choice([64, 128, 256, 512]))
        ndet = int(round(math.exp(rng.uniform(math.log(8), math.log(512)))))
        ns_ = int(2 ** rng.uniform(18, 22)) // 1024 * 1024
        white = rng.random() < 0.5
        fknee = math.exp(rng.uniform(math.log(0.05), math.log(0.5)))
        obs = int(rng.integers(len(observations))) if observations and rng.random() < args.shared_frac else -1
        if obs >= 0:
            o = observations[obs]
            reqs.append(dict(t=ta, nside=o["nside"], ndet=o["ndet"], ns=o["ns"], white=True, fknee=fknee, obs=obs))
        else:
            reqs.append(dict(t=ta, nside=nside, ndet=ndet, ns=ns_, white=white, fknee=fknee, obs=-1))

    def gather_inputs(rq):
        e0, pix0, c0, s0, tw, t1f = pools[rq["nside"]]
        ndet, ns_ = rq["ndet"], rq["ns"]
        d = np.arange(ndet)
        src = d % pool_ndet
        off = ((d // pool_ndet) * 7919 + d * 131) % (pool_ns - ns_ + 1)
        starts = torch.from_numpy((src * pool_ns + off).astype(np.int32)).cuda()  # pool < 2^31 samples
        idx = (starts[:, None] + torch.arange(ns_, device="cuda", dtype=torch.int32)[None, :]).reshape(-1)
        if rq["white"]:
            tod_pool = tw
        else:  # the pool realisation nearest in log f_knee; N^-1 uses the request's own f_knee
            tod_pool = t1f[min(fk_pool, key=lambda f: abs(math.log(f / rq["fknee"])))]
        pix, c, s, tod = (torch.index_select(a, 0, idx) for a in (pix0, c0, s0, tod_pool))
        sigma = np.asarray(e0.sigma)[src]
        return e0, pix, c, s, tod, sigma

    obs_bufs = []
    for o in observations:
        e0, pix, c, s, tod, sigma = gather_inputs(dict(o, white=True))
        sig_t = torch.from_numpy(np.repeat(sigma, o["ns"]).astype(np.float32)).cuda()
        obs_bufs.append((e0, pix, c, s, tod, sigma, sig_t))
    obs_gen = torch.Generator(device="cuda").manual_seed(args.seed + 6)

    def build(rq):
        ndet, ns_ = rq["ndet"], rq["ns"]
        key = 0
        if rq["obs"] >= 0:
            e0, pix, c, s, tod0, sigma, sig_t = obs_bufs[rq["obs"]]
            tod = tod0 + sig_t * torch.randn(tod0.shape, generator=obs_gen, device="cuda", dtype=torch.float32)
            key = 0 if args.no_keys else observations[rq["obs"]]["key"]
        else:
            e0, pix, c, s, tod, sigma = gather_inputs(rq)
        chunk = min(2 ** 20, ns_)
        coeffs = None if rq["white"] else synth.toeplitz_band(sigma, rq["fknee"], 1.0, 20.0, chunk, 512)
        out = torch.empty(e0.npix * 3, dtype=torch.float64, device="cuda")
        det_off = np.arange(ndet + 1, dtype=np.int64) * ns_
        req, keep = L.make_request(e0.npix, pix, tod, out, det_off, 1 / sigma ** 2, cos2psi=c, sin2psi=s,
                                   coeffs=coeffs, chunk_len=chunk, tol=1e-6, maxiter=3000, pointing_key=key)
        return req, (keep, pix, c, s, tod, out)

    ctx = L.bm_context_create(0)
    srv = L.bm_serve_create(ctx, 120 * 2 ** 30, args.slots)
    done = []
    tickets = []
    lock = threading.Lock()
    sampler = ClockSampler(0)
    sampler.start()
    t_start = time.perf_counter()
    inflight_bytes = [0]
    cap = 40 * 2 ** 30  # caller-side input buffers outstanding at once

    def poller():
        while True:
            with lock:
                pending = [x for x in tickets if x["res"] is None]
                finished = len(tickets) == len(reqs) and not pending
            if finished:
                return
            for x in pending:
                st, res = L.bm_serve_poll(srv, x["ticket"], 0)
                if st == L.BM_OK:
                    x["res"] = res
                    x["t_done"] = time.perf_counter() - t_start
                    x["bufs"] = None
                    with lock:
                        inflight_bytes[0] -= x["bytes"]
            time.sleep(0.005)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    for rq in reqs:
        now = time.perf_counter() - t_start
        if rq["t"] > now:
            time.sleep(rq["t"] - now)
        nbytes = rq["ndet"] * rq["ns"] * (4 if rq["obs"] >= 0 else 16)
        while True:
            with lock:
                if inflight_bytes[0] + nbytes <= cap or inflight_bytes[0] == 0:
                    inflight_bytes[0] += nbytes
                    break
            time.sleep(0.01)
        req, bufs = build(rq)
        torch.cuda.synchronize()
        tk = L.bm_serve_submit(srv, req)
        with lock:
            tickets.append({"ticket": tk, "res": None, "t_arr": rq["t"], "bufs": bufs, "bytes": nbytes,
                            "white": rq["white"], "samples": rq["ndet"] * rq["ns"], "shared": rq["obs"] >= 0})
    th.join()
    wall = time.perf_counter() - t_start
    clocks = sampler.stop()
    stats = L.bm_serve_get_stats(srv)
    L.bm_serve_destroy(srv)
    for x in tickets:  # the requests' device buffers go back to the device
        x["bufs"] = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # The plain alternative: the same kind of requests solved one at a time in
    # FP64 (pointing, noise, preconditioner, FP64 PCG), on a seeded sample.
    def solve_alone(rq, prec):
        req, bufs = build(rq)
        keep, pix, c, s, tod, out = bufs
        e0 = pools[rq["nside"]][0]
        sigma = np.asarray(e0.sigma)[np.arange(rq["ndet"]) % pool_ndet]
        det_off = np.arange(rq["ndet"] + 1, dtype=np.int64) * rq["ns"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = L.bm_pointing_create_trig(ctx, e0.npix, pix, c, s, L.BM_SOLVER_IQU)
        chunk = min(2 ** 20, rq["ns"])
        if rq["white"]:
            n = L.bm_inv_noise_create_diag(ctx, det_off, 1 / sigma ** 2)
        else:
            n = L.bm_inv_noise_create_toeplitz(ctx, det_off, chunk,
                                               synth.toeplitz_band(sigma, rq["fknee"], 1.0, 20.0, chunk, 512),
                                               1 / sigma ** 2)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        st, info = L.bm_pcg_solve(p, n, pc, tod, 1, out, 1e-6, 3000, prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)
        return dt, rq["ndet"] * rq["ns"], st

    pick = np.random.default_rng(args.seed + 4).choice(len(reqs), size=min(args.alone_sample, len(reqs)),
                                                         replace=False)
    alone = {"fp64": [0.0, 0], "mixed": [0.0, 0]}
    for i in pick:
        for name, prec in (("fp64", L.BM_PREC_FP64), ("mixed", L.BM_PREC_MIXED)):
            dt, ns_tot, st = solve_alone(reqs[int(i)], prec)
            alone[name][0] += dt
            alone[name][1] += ns_tot
    L.bm_context_destroy(ctx)
    lat = np.array([x["t_done"] - x["t_arr"] for x in tickets]) * 1000
    ok = sum(1 for x in tickets if x["res"]["status"] == L.BM_OK)
    samples = sum(x["samples"] for x in tickets)
    lw = np.array([x["t_done"] - x["t_arr"] for x in tickets if x["white"]]) * 1000
    lt = np.array([x["t_done"] - x["t_arr"] for x in tickets if not x["white"]]) * 1000
    ls = np.array([x["t_done"] - x["t_arr"] for x in tickets if x["shared"]]) * 1000
    line = {
        "workload": "config4", "metric": "served map-making requests: latency from arrival and throughput",
        "value": samples / wall, "unit": "TOD samples/s",
        "config": {"workload": f"Poisson arrivals {args.rate}/s for {args.horizon} s, nside U{{64..512}}, "
                               f"ndet log-U[8,512], Ns 2^U[18,22], white or Toeplitz (p=1/2, fknee log-U[0.05,0.5]), "
                               f"tol 1e-6, budget 120 GB, {args.slots} slots"
                               + (f"; a fraction {args.shared_frac} of the requests are white-noise realisations "
                                  f"of {len(observations)} shared observations"
                                  + (" submitted without pointing_key" if args.no_keys else " (pointing_key)")
                                  if observations else ""),
                   "requests": len(reqs), "shared_frac": args.shared_frac,
                   "observations": observations},
        "completed_ok": ok,
        "failed": [{"status": x["res"]["status"], "message": x["res"]["message"], "samples": x["samples"],
                    "white": x["white"], "iterations": x["res"]["iterations"],
                    "rel_residual": x["res"]["rel_residual"]}
                   for x in tickets if x["res"]["status"] != L.BM_OK][:20],
        "wall_s": wall, "offered_samples_per_s": samples / args.horizon,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "p50_white": float(np.percentile(lw, 50)) if lw.size else None,
                       "p50_toeplitz": float(np.percentile(lt, 50)) if lt.size else None,
                       "p50_shared": float(np.percentile(ls, 50)) if ls.size else None},
        "one_at_a_time": {"sample_requests": len(pick),
                          "fp64_samples_per_s": alone["fp64"][1] / alone["fp64"][0],
                          "mixed_samples_per_s": alone["mixed"][1] / alone["mixed"][0]},
        "served_vs_fp64_one_at_a_time": (samples / wall) / (alone["fp64"][1] / alone["fp64"][0]),
        "served_vs_mixed_one_at_a_time": (samples / wall) / (alone["mixed"][1] / alone["mixed"][0]),
        "server_stats": stats, "clocks": clocks, "pool_generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ hwp
def run_hwp(args):
    """Config 1's scan and white noise with the angle of every sample rebuilt
    from the half-wave-plate model theta = psi_d + 2 (2 pi nu k + phi0),
    nu = 1 Hz / 20 Hz (the scan generator's own model): one step is the
    ingest (angles from the model), the preconditioner, the RHS and the mixed
    solve.  The matvec alone is timed for this pointing (it reads the sorted
    time index, 4 B a sample, and rebuilds the angle) and for the stored-trig
    pointing of the same samples (8 B a sample of weighted trig)."""
    import torch
    L = _L()
    nside, ndet, ns = args.nside, args.ndet, args.ns
    tol = args.tol
    t_gen = time.perf_counter()
    e, d_pix, d_c, d_s = pointing_on_device(nside, ndet, ns, args.seed)
    sky = torch.from_numpy(synth.sky_map(e.npix, args.seed)).cuda()
    d_tod = torch.empty(e.nsamples, dtype=torch.float32, device="cuda")
    device_signal(d_pix, d_c, d_s, sky, d_tod)
    gen = torch.Generator(device="cuda").manual_seed(args.seed)
    device_white(d_tod, e.sigma, ns, gen)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    nu, phi0 = e.scan.hwp_hz / e.scan.fsamp, e.hwp_phase0
    ctx = L.bm_context_create(0)
    out = torch.zeros(e.npix * 3, dtype=torch.float64, device="cuda")
    inv_var = 1 / e.sigma ** 2
    infos = []

    def step():
        p = L.bm_pointing_create_hwp(ctx, e.npix, d_pix, e.det_offsets, e.psi_det, nu, phi0, 3)
        n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, inv_var)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        st, info = L.bm_pcg_solve(p, n, pc, d_tod, 1, out, tol, 200, L.BM_PREC_MIXED)
        infos.append((st, info[0]))
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(0)
    sampler.start()
    L.bm_context_set_timing(ctx, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000 / args.steps
    clocks = sampler.stop()
    fam = {}
    for name in ("ingest", "ingest_validate", "ingest_hist", "ingest_scatter", "blocks", "rhs",
                 "matvec_white_hwp"):
        tot, cnt = L.bm_context_kernel_time(ctx, name)
        if cnt:
            fam[name] = {"ms_per_launch": tot / cnt, "launches_per_step": cnt / args.steps}
    # the matvec alone: this pointing against the stored-trig one
    x = torch.nan_to_num(out)
    q = torch.empty_like(x)
    mv = {}
    for name in ("hwp", "stored"):
        if name == "hwp":
            p = L.bm_pointing_create_hwp(ctx, e.npix, d_pix, e.det_offsets, e.psi_det, nu, phi0, 3)
        else:
            p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, d_c, d_s, 3)
        n = L.bm_inv_noise_create_diag(ctx, e.det_offsets, inv_var)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        hits = torch.empty(e.npix, dtype=torch.int32, device="cuda")
        mask = torch.empty(e.npix, dtype=torch.uint8, device="cuda")
        L.bm_precond_get_mask(pc, mask, hits)
        kept = mask == 0
        n_kept_s, n_kept_p = int(hits[kept].sum().item()), int(kept.sum().item())
        for _ in range(3):
            L.bm_matvec(p, n, pc, x, q, L.BM_PREC_MIXED)
        fam_name = "matvec_white_hwp" if name == "hwp" else "matvec_white_f32"
        L.bm_context_kernel_time(ctx, fam_name)  # reset
        for _ in range(args.matvec_reps):
            L.bm_matvec(p, n, pc, x, q, L.BM_PREC_MIXED)
        tot, cnt = L.bm_context_kernel_time(ctx, fam_name)
        k_ms = tot / max(cnt, 1)
        bps = 4 if name == "hwp" else 8  # sorted time index | weighted trig pair
        nitems = n_kept_p + n_kept_s // 4096
        alg = bps * n_kept_s + 12 * n_kept_p + 24 * nitems
        gbs = alg / (k_ms * 1e-3) / 1e9
        mv[name] = {"kernel_ms": k_ms, "kept_samples_per_s": n_kept_s / (k_ms * 1e-3),
                    "bytes_per_kept_sample": bps, "algorithmic_bytes": alg, "achieved_gbs": gbs,
                    "hbm_frac": gbs / hbm_peak()}
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)
    L.bm_context_set_timing(ctx, False)
    L.bm_context_destroy(ctx)
    st, info = infos[-1]
    h = mv["hwp"]
    line = {
        "workload": "hwp", "metric": METRIC, "value": e.nsamples / (ms * 1e-3), "unit": "TOD samples/s",
        "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": f"GLS map-making, nside {nside}, {ndet} det x {ns} samples, white noise, IQU, "
                               f"angle rebuilt from the half-wave-plate model (nu = {nu:g} turns a sample), "
                               f"mixed precision PCG to {tol:g}", "nsamples": e.nsamples},
        "solve": {"status": st, **info},
        "step_breakdown": fam,
        "matvec": mv,
        "roofline": {"bound": "hbm", "kernel": "white_matvec_hwp_kernel (sorted time index: 4 B a kept sample)",
                     "achieved": h["achieved_gbs"], "peak": hbm_peak(), "unit": "GB/s", "frac": h["hbm_frac"],
                     "traffic": None},
        "clocks": clocks, "input_generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)


def run(args, rank, world, local_rank):
    if rank != 0:
        return
    if args.workload == "offsets":
        run_config2(args, noise="offsets")
        return
    {"config0": run_config0, "config2": run_config2, "config3": run_config3, "config4": run_config4,
     "hwp": run_hwp}[args.workload](args)
