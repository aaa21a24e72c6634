#!/usr/bin/env python3
"""Benchmark of the GLS map-making hot path (BrahMap, arXiv 2501.16122) on GB300.

Workload (default): HEALPix nside 256 (786,432 pixels), 256 detectors x 2^22
samples (1,073,741,824 samples) from the seeded spin + precession scan, FP32
TOD, int32 pixel indices, FP32 precomputed cos 2psi / sin 2psi, diagonal white noise
(sigma_d in [1, 2] uK), IQU, pixels with hits < 3 or cond > 1e3 masked, PCG
to 1e-8 in mixed precision (FP32 per-sample products, FP64 accumulation,
FP64 iterative refinement).

One step = one pass of the whole hot path over the resident inputs:
pointing ingest (trig, pixel sort) -> block preconditioner + mask -> RHS ->
PCG with refinement -> map.  `value` is TOD samples per second of whole
steps (all ranks); `matvec` gives the P^T N^-1 P matvec throughput alone.
`e2e` repeats the step through host (pinned) buffers with the host->device
copies of pix/cos/sin/tod and the device->host copy of the map inside the timed
region.  `--impl reference` times the FP64 CPU oracle on a bounded sample.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run (one rank per GPU) the same workload is sharded by
detector (the paper's data distribution): each rank ingests and solves over
its own detectors, and the library sums the per-pixel partial blocks, RHS and
A x over the ranks with an NCCL all-reduce (bm_context_set_allreduce); the
slowest rank's time counts and `value` is the whole workload's samples per
second (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TOD samples/s per PᵀN⁻¹P matvec (%HBM peak); PCG time-to-map at 1e-6 rel err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--nside", type=int, default=256)
    ap.add_argument("--ndet", type=int, default=256)
    ap.add_argument("--ns", type=int, default=2 ** 22, help="samples per detector")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--seed", type=int, default=1001)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=-1,
                    help="host processes of the multi-core oracle figure (-1: every core, 0: skip)")
    ap.add_argument("--matvec-reps", type=int, default=20)
    ap.add_argument("--profile", action="store_true", help="short run for ncu: no e2e, cpu, clocks")
    ap.add_argument("--workload", default="config1",
                    choices=["config0", "config1", "config2", "config3", "config4", "offsets", "hwp"],
                    help="config1 (default): nside 256 white-noise solve; config0: small FP64 solve; "
                         "config2: 512-lag Toeplitz noise; config3: 64 right-hand sides batched; "
                         "config4: Poisson request stream through the server; offsets: config2's 1/f TOD "
                         "with a baseline offset per 60 s marginalised out instead of the Toeplitz N^-1")
    ap.add_argument("--horizon", type=float, default=20.0, help="config4: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=20.0, help="config4: mean arrivals per second")
    ap.add_argument("--nrhs", type=int, default=64, help="config3: right-hand sides")
    ap.add_argument("--slots", type=int, default=2, help="config4: requests the server runs at once")
    ap.add_argument("--shared-frac", type=float, default=0.0,
                    help="config4: fraction of requests that are white-noise realisations of a few shared "
                         "observations (same pointing, pointing_key set)")
    ap.add_argument("--observations", type=int, default=4, help="config4: shared observations")
    ap.add_argument("--no-keys", action="store_true",
                    help="config4: submit the shared observations' requests without pointing_key (each solved "
                         "from scratch: the serial comparison for the same arrivals)")
    ap.add_argument("--alone-sample", type=int, default=24,
                    help="config4: requests re-solved one at a time for the serial comparison")
    ap.add_argument("--no-fp64-solve", action="store_true", help="config2: skip the timed plain FP64 solve")
    ap.add_argument("--rhs-path", choices=["carried", "gather"], default="carried",
                    help="config1: the TOD sorted along with the pointing (carried, default) or "
                         "gathered through the permutation by the solve (gather)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.lines = gpu, None, []
        self.window = None  # (t0, t1) monotonic seconds of the timed region, when marked

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, t0: float, t1: float):
        """Keep only the samples taken between t0 and t1 (time.monotonic())."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.window is not None:
            lines = [(ts, ln) for ts, ln in lines if self.window[0] <= ts <= self.window[1]]
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ inputs
def make_inputs(args, seed):
    """Config-1 inputs: int32 pixels, FP32 precomputed cos 2psi / sin 2psi, FP32 TOD."""
    import synth
    e = synth.make_experiment(args.nside, args.ndet, args.ns, seed)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    sky = synth.sky_map(e.npix, seed)
    tod = synth.tod(e, pt["pix"], pt["psi"], sky, dtype=np.float32, trig=(c32, s32))
    return e, pt["pix"], c32, s32, tod


def cpu_oracle_run(nside, ndet, ns, seed, tol):
    """One oracle map-making pass (system set-up, RHS, PCG) on a sample; returns (samples, seconds)."""
    import synth
    from oracle import gls
    e = synth.make_experiment(nside, ndet, ns, seed)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    tod = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, seed), dtype=np.float32,
                    trig=(c32, s32)).astype(np.float64)
    t0 = time.perf_counter()
    S = gls.System(pt["pix"], None, 3, e.npix, gls.WhiteNoise(1.0 / e.sigma ** 2, e.det_offsets),
                   trig=(c32, s32))
    x, info = gls.pcg(S, S.rhs(tod), tol, 100)
    dt = time.perf_counter() - t0
    return e.nsamples, dt


CPU_SAMPLE = dict(ndet=8, ns=2 ** 19)  # 4.2M samples of the same scan: ~10 s of oracle work


def _oracle_slice_worker(k, nside, ndet, ns, seed, ready, start, out):
    """One host process of the multi-core oracle run: generates its own
    detectors' samples (untimed), waits for the common start, then computes
    its partial sums with the oracle's functions: the blocks of Eq. 7, the hit
    counts and b = P^T N^-1 d of its samples (white noise)."""
    import synth
    from oracle import gls
    e = synth.make_experiment(nside, ndet, ns, seed)
    pt = synth.pointing(e)
    c32, s32 = synth.trig32(pt["psi"])
    d = synth.tod(e, pt["pix"], pt["psi"], synth.sky_map(e.npix, seed), dtype=np.float32,
                  trig=(c32, s32)).astype(np.float64)
    ready.put(k)
    start.wait()
    t0 = time.perf_counter()
    pix = pt["pix"].astype(np.int64)
    v = gls.pointing_weights_trig(c32, s32, 3)
    w = (1.0 / e.sigma ** 2)[gls.sample_detector(e.det_offsets)]
    B = gls.block_matrices(pix, v, w, e.npix)
    h = gls.hits(pix, e.npix)
    b = gls.apply_PT(pix, v, w * d, e.npix)
    out.put((k, e.nsamples, B, h, b, t0, time.perf_counter()))


def cpu_oracle_multicore(nside, nproc, seed):
    """The oracle over nproc host processes, split by detector (each process
    a slice of CPU_SAMPLE's size with detectors of its own): partial blocks,
    hits and RHS per process, summed in process order (a fixed order), then
    the mask, the block inverse and the white-noise GLS map x = M b (the PCG's
    one-iteration solution).  Returns (samples, seconds from the common start
    to the map)."""
    import multiprocessing as mp
    from oracle import gls
    ctx = mp.get_context("spawn")  # GPU work already ran in this process: no fork
    ready, start, out = ctx.Queue(), ctx.Event(), ctx.Queue()
    procs = [ctx.Process(target=_oracle_slice_worker,
                         args=(k, nside, CPU_SAMPLE["ndet"], CPU_SAMPLE["ns"], seed + 7919 * (k + 1), ready, start,
                               out))
             for k in range(nproc)]
    for pr in procs:
        pr.start()
    for _ in procs:  # every process has generated its inputs
        ready.get(timeout=600)
    start.set()
    parts = sorted((out.get(timeout=600) for _ in procs), key=lambda p_: p_[0])
    for pr in procs:
        pr.join()
    t_parts = max(p_[6] for p_ in parts)
    tc = time.perf_counter()
    n = sum(p_[1] for p_ in parts)
    B, h, b = parts[0][2].copy(), parts[0][3].copy(), parts[0][4].copy()
    for p_ in parts[1:]:  # fixed order: process 0, 1, ...
        B += p_[2]
        h += p_[3]
        b += p_[4]
    mask = gls.pixel_mask(h, B, 3, 1e3)
    M = gls.block_inverse(B, mask)
    b[mask] = 0.0
    gls.precond_apply(M, b)
    combine = time.perf_counter() - tc
    t0 = min(p_[5] for p_ in parts)
    return n, (t_parts - t0) + combine


# Kernel of each timed family, and the DRAM traffic per launch measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the small case of
# profiles/ scaled to the full launch by the samples processed; None when the
# kernel has changed since the counters were taken.
KERNELS = {"ingest_validate": "validate_kernel", "ingest_hist": "rs_hist_kernel",
           "ingest_scatter": "rs_scatter_kernel", "blocks": "blocks_kernel", "rhs": "gather_reduce_kernel",
           "matvec_white_f32": "white_matvec_f32_kernel"}
TRAFFIC = {
    # ncu on the 67M-sample case of the same scan (256 detectors x 262,144
    # samples): 39.1 and 41.9 DRAM bytes per sample for the two scatter
    # passes (mean 40.5); the traffic grows in proportion to the samples
    "ingest_scatter": lambda n: 40.5 * n,
}


def n_valid_kept(hits, kept):
    return int(hits[kept].sum().item())


# ------------------------------------------------------------- reference
def run_reference(args, rank):
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        n, dt = cpu_oracle_run(args.nside, CPU_SAMPLE["ndet"], CPU_SAMPLE["ns"], args.seed, args.tol)
        if i >= args.warmup:
            steps.append((n, dt))
    n = sum(s[0] for s in steps)
    t = sum(s[1] for s in steps)
    v = n / t
    sample = (f"{CPU_SAMPLE['ndet']} detectors x {CPU_SAMPLE['ns']} samples of the nside-{args.nside} scan "
              f"(one oracle set-up + RHS + PCG per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TOD samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / len(steps),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded scan, Gaussian sky, white noise)",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "TOD samples/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "TOD samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"GLS map-making, nside {args.nside}, {args.ndet} det x {args.ns} samples, "
                        f"white noise, IQU, mixed precision PCG to {args.tol:g}",
            "nside": args.nside, "npix": 12 * args.nside ** 2, "ndet": args.ndet, "samples_per_det": args.ns,
            "nsamples": args.ndet * args.ns, "solver": "IQU", "noise": "white", "tod_dtype": "f32",
            "trig_dtype": "f32 (precomputed cos 2psi, sin 2psi)", "tol": args.tol, "min_hits": 3, "max_cond": 1e3,
            "parallelism": (f"detector-sharded x{args.gpus} (NCCL all-reduce of per-pixel partial sums)"
                            if args.gpus > 1 else "1 GPU"),
            "tod_path": ("sorted along with the pointing, read in pixel order by the RHS"
                         if args.rhs_path == "carried" else "gathered through the sort permutation by the RHS"),
            "l2": "inputs (17 GB) larger than L2 (129 MB); no flush needed"}


# ------------------------------------------------------------------ gb300
def run_gb300(args, rank, world, local_rank):
    import torch
    from paper_2501_16122_gb300 import _lib as L

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    t_gen = time.perf_counter()
    e, pix, c32, s32, tod = make_inputs(args, args.seed)
    t_gen = time.perf_counter() - t_gen
    nt_total = e.nsamples
    det_offsets, inv_var = e.det_offsets, 1.0 / e.sigma ** 2
    if world > 1:  # this rank's detectors only
        d0, d1, det_offsets = L.detector_shard(e.det_offsets, rank, world)
        s0, s1 = int(e.det_offsets[d0]), int(e.det_offsets[d1])
        pix, c32, s32, tod = pix[s0:s1], c32[s0:s1], s32[s0:s1], tod[s0:s1]
        inv_var = inv_var[d0:d1]
    nt = pix.size
    stream = torch.cuda.current_stream()
    d_pix = torch.from_numpy(pix).cuda()
    d_trig = (torch.from_numpy(c32).cuda(), torch.from_numpy(s32).cuda())
    d_tod = torch.from_numpy(tod).cuda()
    ctx = L.bm_context_create(local_rank, stream)
    if world > 1:  # partial per-pixel sums over the ranks: NCCL all-reduce
        L.bm_context_set_allreduce(ctx, L.torch_allreduce())
    out = torch.empty(e.npix * 3, dtype=torch.float64, device="cuda")
    infos = []

    carried = args.rhs_path == "carried"

    def step(src_pix, src_trig, src_tod, tod_ready=None):
        if carried:  # the TOD rides through the pixel sort; the solve reads it in sorted order
            p = L.bm_pointing_create_with_tod(ctx, e.npix, src_pix, src_tod, cos2psi=src_trig[0],
                                              sin2psi=src_trig[1])
        else:
            p = L.bm_pointing_create_trig(ctx, e.npix, src_pix, src_trig[0], src_trig[1], L.BM_SOLVER_IQU)
        n = L.bm_inv_noise_create_diag(ctx, det_offsets, inv_var)
        pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
        if tod_ready is not None:  # the TOD upload ran beside the ingest and the preconditioner
            stream.wait_event(tod_ready)
        st, info = L.bm_pcg_solve(p, n, pc, None if carried else src_tod, 1, out, args.tol, 200,
                                  L.BM_PREC_MIXED)
        infos.append((st, info[0]))
        L.bm_precond_destroy(pc)
        L.bm_inv_noise_destroy(n)
        L.bm_pointing_destroy(p)

    # clocks are sampled from before the warm-up (nvidia-smi takes a moment to
    # start) and kept for the timed region only
    sampler = ClockSampler(local_rank)
    if not args.profile:
        sampler.start()
    for _ in range(args.warmup):
        step(d_pix, d_trig, d_tod)
    # --- timed region (device-resident inputs)
    L.bm_context_set_timing(ctx, True)
    launches0 = L.bm_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.monotonic()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(d_pix, d_trig, d_tod)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_wall0, time.monotonic())
    barrier()
    launches = L.bm_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop() if not args.profile else None
    fam = {}
    for name in ("ingest", "ingest_validate", "ingest_hist", "ingest_scatter", "blocks", "rhs",
                 "matvec_white_f32", "matvec_white_f64"):
        tot, cnt = L.bm_context_kernel_time(ctx, name)
        if cnt:
            fam[name] = {"ms_per_launch": tot / cnt, "launches": cnt, "ms_per_step": tot / args.steps}
    L.bm_context_set_timing(ctx, False)

    # --- matvec alone (the metric's kernel), x = the solved map
    p = L.bm_pointing_create_trig(ctx, e.npix, d_pix, d_trig[0], d_trig[1], L.BM_SOLVER_IQU)
    n = L.bm_inv_noise_create_diag(ctx, det_offsets, inv_var)
    pc = L.bm_blockdiag_precond_create(p, n, 3, 1e3)
    mask = torch.empty(e.npix, dtype=torch.uint8, device="cuda")
    hits = torch.empty(e.npix, dtype=torch.int32, device="cuda")
    L.bm_precond_get_mask(pc, mask, None)
    L.bm_pointing_get_hits(p, hits)  # this rank's samples (all of them at N = 1)
    kept = mask == 0
    n_kept_samples = int(hits[kept].sum().item())
    n_kept_pix = int(kept.sum().item())
    x = torch.nan_to_num(out)
    q = torch.empty_like(x)
    for _ in range(3):
        L.bm_matvec(p, n, pc, x, q, L.BM_PREC_MIXED)
    L.bm_context_set_timing(ctx, True)
    torch.cuda.synchronize()
    mv0, mv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mv0.record(stream)
    for _ in range(args.matvec_reps):
        L.bm_matvec(p, n, pc, x, q, L.BM_PREC_MIXED)
    mv1.record(stream)
    torch.cuda.synchronize()
    mv_call_ms = mv0.elapsed_time(mv1) / args.matvec_reps
    k_tot, k_cnt = L.bm_context_kernel_time(ctx, "matvec_white_f32")
    L.bm_context_set_timing(ctx, False)
    k_ms = k_tot / max(k_cnt, 1)
    # the plain FP64 path on the same system, beside the refined one (solve
    # only: pointing, noise model and preconditioner already built)
    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    out_alt = torch.empty_like(out)
    fp64_path = {
        "matvec_ms": timed(lambda: L.bm_matvec(p, n, pc, x, q, L.BM_PREC_FP64)),
        "solve_ms": timed(lambda: L.bm_pcg_solve(p, n, pc, d_tod, 1, out_alt, args.tol, 200, L.BM_PREC_FP64)),
        "mixed_solve_ms": timed(lambda: L.bm_pcg_solve(p, n, pc, d_tod, 1, out_alt, args.tol, 200, L.BM_PREC_MIXED)),
    }
    nitems_est = sum(math.ceil(h / 4096) for h in hits[kept].tolist()) if n_kept_pix < 5_000_000 else 0
    alg_bytes = 8 * n_kept_samples + 12 * n_kept_pix + 24 * nitems_est  # trig pair + x + item partials
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    L.bm_precond_destroy(pc)
    L.bm_inv_noise_destroy(n)
    L.bm_pointing_destroy(p)

    # --- roofline of every timed kernel family of the step (algorithmic bytes
    # per step / device time per step); the dominant family is the headline
    nbits = 1
    while (1 << nbits) <= e.npix:
        nbits += 1
    passes = -(-nbits // 10)
    bits = -(-nbits // passes)
    kb = 2 if nbits - bits <= 16 else 4  # bytes of a key stored between passes
    n_valid = int(hits.sum().item())
    scatter_bytes = 0
    hist_bytes = 0
    # The timed step passes cos/sin as 16-byte-aligned device arrays: the
    # first sort pass reads them itself and the validation reads and copies
    # the pixels alone; with the TOD carried, the time-ordered pairs are left
    # to the first time-ordered operator (none in a white-noise step), else
    # the first pass writes them (8 bytes a sample).
    for ps in range(passes):
        last = ps == passes - 1
        # keys + records, or pixel keys + cos + sin (+ TOD) in time order
        rd = (kb + 16) if ps > 0 else (4 + (12 if carried else 8))
        # perm + trig (+ TOD) of kept samples, or records + keys
        wr = ((16 if carried else 12) * n_valid / nt) if last else 16 + kb
        if ps == 0 and not carried:
            wr += 8                                        # the time-ordered trig pairs
        scatter_bytes += (rd + wr) * nt
        if ps > 0:                                         # (the first pass's counts come from validation)
            hist_bytes += kb * nt                          # keys
    step_bytes = {
        # pix in (with the first pass's digit counts); pix out unless the TOD is
        # carried (then the time-ordered copy waits for a time-ordered operator)
        "ingest_validate": (4 if carried else 8) * nt,
        "ingest_hist": hist_bytes,
        "ingest_scatter": scatter_bytes,
        # perm + trig pair (+ the carried TOD, whose RHS this pass also sums) in, weighted pair out
        "blocks": (24 if carried else 20) * n_valid_kept(hits, kept),
        # perm + gathered d + trig pair; with the carried TOD the RHS was summed
        # with the blocks and the solve copies it (read + write of the map-sized b)
        "rhs": 16 * n_valid_kept(hits, kept) if not carried else 2 * 8 * 3 * e.npix,
        "matvec_white_f32": alg_bytes * fam.get("matvec_white_f32", {}).get("launches", 0) / max(args.steps, 1),
    }
    rooflines = {}
    for name, b in step_bytes.items():
        f = fam.get(name)
        if not f or f["ms_per_step"] <= 0:
            continue
        gbs = b / (f["ms_per_step"] * 1e-3) / 1e9
        rooflines[name] = {"ms_per_step": f["ms_per_step"], "bytes_per_step": b, "achieved_gbs": gbs,
                           "frac": gbs / hbm, "bytes_per_sample": b / nt}
    dom = max(rooflines, key=lambda k: rooflines[k]["ms_per_step"]) if rooflines else None

    # --- end to end from pinned host buffers
    e2e = None
    if not args.no_e2e and not args.profile:
        h_pix = torch.from_numpy(pix).pin_memory()
        h_c = torch.from_numpy(c32).pin_memory()
        h_s = torch.from_numpy(s32).pin_memory()
        h_tod = torch.from_numpy(tod).pin_memory()
        h_out = torch.empty(e.npix * 3, dtype=torch.float64).pin_memory()

        upload = torch.cuda.Stream()

        def e2e_step():
            # The pointing goes to the library as page-locked host buffers: its
            # ingest reads them once over the host link, with no staging copy.
            # A carried TOD is read the same way by the ingest; otherwise it is
            # needed only by the solve and is uploaded on a second stream while
            # the pointing is ingested.
            if carried:
                step(h_pix, (h_c, h_s), h_tod)
                h_out.copy_(out, non_blocking=True)
                torch.cuda.current_stream().synchronize()
                return
            with torch.cuda.stream(upload):
                c = h_tod.to("cuda", non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(upload)
            c.record_stream(stream)
            step(h_pix, (h_c, h_s), c, ready)
            h_out.copy_(out, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        e2e_step()
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(max(1, args.steps // 2)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e2e_ms = (time.perf_counter() - w0) * 1000 / max(1, args.steps // 2)
        e2e = {"ms_per_step": e2e_ms, "h2d_bytes_per_step": int(pix.nbytes + c32.nbytes + s32.nbytes + tod.nbytes),
               "d2h_bytes_per_step": int(h_out.numel() * 8)}

    # --- max over ranks
    vals = torch.tensor([ms, e2e["ms_per_step"] if e2e else 0.0], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    ms_max, e2e_max = vals.tolist()

    # --- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.profile:
        n_s, dt = cpu_oracle_run(args.nside, CPU_SAMPLE["ndet"], CPU_SAMPLE["ns"], args.seed, args.tol)
        cpu = {"value": n_s / dt, "unit": "TOD samples/s", "cores": 1, "kind": "oracle",
               "sample": f"{CPU_SAMPLE['ndet']} det x {CPU_SAMPLE['ns']} samples of the same scan "
                         f"(oracle set-up + RHS + PCG, {dt:.1f} s)"}
        if args.cpu_procs != 0:
            nproc = args.cpu_procs if args.cpu_procs > 0 else (os.cpu_count() or 1)
            n_m, dt_m = cpu_oracle_multicore(args.nside, nproc, args.seed)
            cpu["multi_core"] = {
                "value": n_m / dt_m, "unit": "TOD samples/s", "cores": nproc, "kind": "oracle",
                "sample": (f"{nproc} host processes, each {CPU_SAMPLE['ndet']} det x {CPU_SAMPLE['ns']} samples of "
                           f"the same scan (detectors of its own): the oracle's blocks, hits and RHS per process, "
                           f"summed in process order, then mask, inverse and x = M b ({dt_m:.1f} s)")}

    if rank == 0:
        st_ok = all(s == L.BM_OK for s, _ in infos)
        last = infos[-1][1]
        line = {
            "metric": METRIC, "value": nt_total / (ms_max * 1e-3), "unit": "TOD samples/s",
            "value_basis": ("the step's TOD samples / the whole step's time (ingest + preconditioner + RHS + "
                            "PCG to tol); the PᵀN⁻¹P matvec alone is under 'matvec', the time-to-map without "
                            "the ingest under 'time_to_map_ms'"),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32",
            "precision": "f32 per-sample products; double-float / f64 accumulation; f64 blocks, CG scalars and refinement",
            "data": "synthetic (seeded spin+precession scan, Gaussian IQU sky, white noise)",
            "config": workload_config(args),
            "matvec": {"samples_per_s": nt / (k_ms * 1e-3), "kept_samples_per_s": n_kept_samples / (k_ms * 1e-3),
                       "kernel_ms": k_ms, "call_ms": mv_call_ms, "kept_samples": n_kept_samples,
                       "hbm_frac": achieved / hbm,
                       "note": ("this rank's samples; the call includes the all-reduce of A x" if world > 1
                                else "samples of the step's TOD (kept: in unmasked pixels)")},
            "time_to_map_ms": ms_max - fam.get("ingest", {}).get("ms_per_step", 0.0),
            "solve_only_ms": fp64_path,
            "step_breakdown_ms": {k: v["ms_per_step"] for k, v in fam.items()},
            "solve": {"status_ok": st_ok, "iterations": last["iterations"],
                      "outer_iterations": last["outer_iterations"], "rel_residual": last["rel_residual"]},
            "roofline": ({"bound": "hbm", "achieved": rooflines[dom]["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                          "frac": rooflines[dom]["frac"], "traffic": (TRAFFIC.get(dom) or (lambda n: None))(nt),
                          "kernel": KERNELS[dom], "family": dom, "peak_kind": peak_kind,
                          "launches_per_step": fam[dom]["launches"] / args.steps,
                          "bytes_per_launch": rooflines[dom]["bytes_per_step"] / (fam[dom]["launches"] / args.steps),
                          "ms_per_launch": fam[dom]["ms_per_launch"]} if dom else None),
            "rooflines": rooflines,
            "matvec_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                "frac": achieved / hbm, "kernel": "white_matvec_f32_kernel",
                                "peak_kind": peak_kind, "bytes_per_launch": alg_bytes},
            "gpu_launches": int(launches),
            "input_generation_s": t_gen,
        }
        if e2e:
            line["e2e"] = {"value": nt_total / (e2e_max * 1e-3), "unit": "TOD samples/s",
                           "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                           "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "ms_per_step": e2e_max}
        if clocks:
            line["clocks"] = clocks
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    L.bm_context_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "config4":
        # the caller's request buffers come and go in many sizes: expandable
        # segments keep torch's cache from fragmenting next to the server's
        # own allocations
        os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    if args.workload != "config1":
        import bench_workloads
        bench_workloads.run(args, rank, world, local_rank)
        return
    run_gb300(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
