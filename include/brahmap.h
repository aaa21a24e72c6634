/*
 * brahmap.h — C-ABI of the GB300 GLS map-making library.
 *
 * The library solves the generalized-least-squares map-making problem of
 * BrahMap (Anand & Puglisi, arXiv 2501.16122, Sec. II):
 *
 *     d = P s + n                      (Eq. 3)
 *     A x = b,  A = P^T N^-1 P,  b = P^T N^-1 d     (Eq. 5-6)
 *     M = (P^T diag(N)^-1 P)^-1        (Eq. 7, the block-diagonal preconditioner)
 *
 * where P (Eq. 8) has, for every time sample t, the entries
 * [1, cos 2psi_t, sin 2psi_t] in the columns (I, Q, U) of the pixel p_t hit
 * at time t (QU solves use [cos 2psi, sin 2psi], I solves [1]).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers marked "device" are CUDA device pointers on the context's device;
 *    pointers marked "host" are ordinary host memory.  The caller allocates and
 *    frees every user array (the ownership rule the paper's Python layer
 *    adopts, Sec. III-A item 3); handles own the device copies they make, so a
 *    caller may free its inputs as soon as a *_create call returns.
 *  - Time samples are laid out detector by detector: samples of detector d
 *    are [det_offsets[d], det_offsets[d+1]).  Maps are pixel-major with the
 *    Stokes components interleaved, [npix][ncomp] (Eq. 8's sky vector), FP64.
 *  - Pixel indices are int32 in [0, npix); -1 marks a flagged sample, which
 *    contributes nothing (its row of P is zero).
 *  - Every call is stream-ordered on the context's stream and returns after
 *    the work it enqueued has completed, unless documented otherwise.
 *  - Errors: every call returns a bm_status; no exception crosses the ABI.
 *    bm_last_error() returns a thread-local message for the last failure on
 *    the calling thread.  On failure, outputs are unspecified and no memory
 *    is leaked.  An out-of-range argument (size, enum, NULL pointer) returns
 *    BM_ERR_INVALID before any device work is enqueued.
 *  - A handle is used by one host thread at a time; the server (bm_serve_*)
 *    is thread-safe.
 */
#ifndef BRAHMAP_H
#define BRAHMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BM_OK = 0,
    BM_ERR_INVALID = 1,        /* bad argument */
    BM_ERR_OOM = 2,            /* device allocation failed (nothing leaked) */
    BM_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    BM_ERR_NOT_CONVERGED = 4,  /* maxiter reached before tol */
    BM_ERR_BREAKDOWN = 5,      /* p^T A p <= 0 or a non-finite CG scalar */
    BM_ERR_TIMEOUT = 6,        /* a bounded wait expired */
    BM_ERR_BUSY = 7,           /* server admission refused (budget or slots) */
    BM_ERR_NOT_FOUND = 8       /* unknown server ticket */
} bm_status;

typedef enum { BM_SOLVER_I = 1, BM_SOLVER_QU = 2, BM_SOLVER_IQU = 3 } bm_solver_type;
typedef enum { BM_F32 = 0, BM_F64 = 1 } bm_dtype;

/* BM_PREC_FP64: every per-sample product and sum in FP64 (the plain path).
 * BM_PREC_MIXED: FP32 per-sample products inside an FP64 iterative
 * refinement loop whose residual r = b - A x uses the FP64 operator. */
typedef enum { BM_PREC_FP64 = 0, BM_PREC_MIXED = 1 } bm_precision;

typedef struct bm_context bm_context;
typedef struct bm_pointing bm_pointing;
typedef struct bm_inv_noise bm_inv_noise;
typedef struct bm_precond bm_precond;

/* Per right-hand-side outcome of bm_pcg_solve. */
typedef struct {
    int32_t status;            /* bm_status of this RHS */
    int32_t iterations;        /* PCG iterations (inner iterations summed in mixed mode) */
    int32_t outer_iterations;  /* refinement steps (mixed mode; 0 for FP64) */
    int32_t reserved;
    double rel_residual;       /* ||b - A x||_2 / ||b||_2, recomputed with the FP64 operator */
} bm_solve_info;

/* ---------------------------------------------------------------- errors */

/* Static text of a status code. */
const char* bm_status_string(bm_status s);
/* Message of the last failed call on this thread ("" if none). */
const char* bm_last_error(void);
/* Library version string. */
const char* bm_version(void);

/* --------------------------------------------------------------- context */

/* Bind the library to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is
 * borrowed: the caller keeps it alive until bm_context_destroy.  The context
 * keeps its scratch buffers (the pixel sort's ping-pong buffers, up to
 * 20-28 bytes a sample, and the solver's vectors) in a device memory pool of
 * its own for reuse by later calls; bm_context_destroy releases them. */
bm_status bm_context_create(int device, void* cuda_stream, bm_context** out);
void bm_context_destroy(bm_context* ctx);

/* Detector-sharded solve (paper Sec. III-A item 1: every process owns a
 * subset of the samples and its own operator instances; Sec. III-B: the
 * pointing operator's transpose sums its partial map over the processes).
 * A reduction callback: sum the FP64 array buf (device memory of the
 * context's GPU, count values) over every rank, in place, so that every rank
 * holds the same bits; return BM_OK, or another status to fail the calling
 * entry point with it.  For example ncclAllReduce followed by a stream
 * synchronize, or a copy to the host, an MPI or gloo allreduce and a copy
 * back.  The library calls it from the calling thread after synchronising the
 * context stream, and uses buf again only after it returns. */
typedef bm_status (*bm_allreduce_fn)(double* buf, int64_t count, void* user);
/* Make ctx one rank of a detector-sharded solve (fn = NULL: unsharded again).
 * Every pointing and noise handle built on it then holds this rank's
 * samples only (its own detectors, with det_offsets of its own layout), and
 * the library sums over the ranks, through fn, exactly the per-pixel
 * quantities that need it: the hit counts and blocks of
 * bm_blockdiag_precond_create (before the mask, the condition numbers and
 * the inverse, which every rank then computes from the same sums), the
 * right-hand side b of bm_rhs / bm_pcg_solve, A x of bm_matvec and of every
 * PCG iteration, and P^T y of bm_pointing_apply_transpose.  Everything else
 * (CG vectors and scalars, map) is replicated: every rank computes the same
 * values.  All ranks must therefore make the same sequence of these calls
 * with the same npix, solver, min_hits, max_cond, tol and maxiter; a Toeplitz
 * chunk or an offset interval never spans two ranks, since both stay within
 * a detector.  bm_matvec_white_static and bm_pointing_get_hits return this
 * rank's partial values (no reduction); bm_precond_get_mask returns the hit
 * counts summed over the ranks.  Several right-hand sides of a sharded solve
 * are solved one after another. */
bm_status bm_context_set_allreduce(bm_context* ctx, bm_allreduce_fn fn, void* user);

/* Kernel timing: when enabled, the library brackets its main kernels with
 * CUDA events on the context stream and accumulates per-kernel device time.
 * bm_context_kernel_time returns the accumulated milliseconds and launch
 * count of the kernel family `name` ("matvec_white_f32", "matvec_white_f64",
 * "toeplitz_f32", "toeplitz_f64", "rhs", "ingest", "blocks") and resets it. */
bm_status bm_context_set_timing(bm_context* ctx, int enable);

/* CUDA graphs (on by default): bm_pcg_solve runs its PCG iterations as one
 * CUDA graph per solve whose conditional WHILE node ends the loop on the
 * device, captured on a stream of the context.  While a capture is in
 * progress, a device-wide synchronisation (cudaDeviceSynchronize,
 * torch.cuda.synchronize) by any other thread of the process fails with
 * cudaErrorStreamCaptureUnsupported; a context used while other threads
 * synchronise the device can turn the graphs off (the iterations are then
 * driven from the host: the same results, bit for bit).  The server's
 * contexts have them off. */
bm_status bm_context_set_graphs(bm_context* ctx, int enable);
bm_status bm_context_kernel_time(bm_context* ctx, const char* name, double* total_ms,
                                 int64_t* launches);
/* Number of CUDA kernels the library has launched in this process so far
 * (all contexts and threads). */
int64_t bm_kernel_launches(void);

/* Measured FP32 (dtype BM_F32) or FP64 (BM_F64) fused multiply-add rate of
 * the context's GPU in flop/s (2 per FMA): independent FMA chains on every
 * SM, timed with CUDA events on the context stream (best of three after a
 * warm-up, a few ms each).  The denominator of the rooflines of the
 * arithmetic-bound kernels.  A measurement helper with no counterpart in the
 * paper. */
bm_status bm_measure_fma_peak(bm_context* ctx, bm_dtype dtype, double* flops_per_s);

/* ------------------------------------------------------------- pixelisation */

/* HEALPix RING index of n directions (Gorski et al. 2005; the paper's "sky
 * pixel", Sec. II): z = cos(theta) in [-1, 1], phi in [0, 2 pi), both device
 * FP64 [n]; pix device int32 [n].  Computed with correctly rounded FP64
 * operations in a fixed order (no fused multiply-add), so the integers match
 * any other implementation of the same steps bit for bit.  nside in
 * [1, 8192]. */
bm_status bm_ang2pix_ring(bm_context* ctx, int64_t nside, int64_t n, const double* z,
                          const double* phi, int32_t* pix);

/* -------------------------------------------------------------- pointing */

/* Pointing matrix P (Eq. 8) and its precomputed elements (the paper's
 * ProcessTimeSamples, Sec. III-A item 1): pix int32 [nsamples]
 * (-1 = flagged), psi [nsamples] of dtype psi_dtype (the polarisation
 * angle theta of Eq. 2, radians).  Both may be device memory of the
 * context's GPU or page-locked host memory (cudaHostAlloc /
 * cudaHostRegister), which the ingest reads once, directly over the host
 * link, without a staging copy; other host memory returns BM_ERR_INVALID.
 * The handle keeps the pixel-sorted sample
 * permutation, CSR offsets, hit counts and cos/sin 2psi stored as FP32
 * (hi, lo) pairs whose sum carries the FP64 value to 2^-48.
 * Requires 1 <= npix <= 2^28, 1 <= nsamples < 2^32.  A pixel index outside
 * [-1, npix) returns BM_ERR_INVALID. */
bm_status bm_pointing_create(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                             const void* psi, bm_dtype psi_dtype, bm_solver_type solver,
                             bm_pointing** out);
/* The same operator from precomputed FP32 cos 2psi and sin 2psi ([nsamples]
 * each, |values| <= 1; device or page-locked host memory, as pix): the FP32
 * numbers are the entries of P
 * (Eq. 8) exactly, so no extra precision is kept and every FP64 result is
 * computed from them.  Requirements and errors as bm_pointing_create. */
bm_status bm_pointing_create_trig(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                  const float* cos2psi, const float* sin2psi, bm_solver_type solver,
                                  bm_pointing** out);
/* bm_pointing_create (psi given, cos2psi = sin2psi = NULL) or
 * bm_pointing_create_trig (cos2psi and sin2psi given, psi = NULL) that also
 * sorts one FP32 TOD d [nsamples] (device or page-locked host memory) along
 * with the samples: the handle keeps d of the kept samples in pixel-sorted
 * order (4 bytes a sample), and bm_rhs / bm_pcg_solve called with tod = NULL
 * read it as a stream instead of gathering d through the permutation.  The
 * operator is the one the other constructors build; d is copied, so the
 * caller's array may be freed on return.  The carried TOD serves one
 * right-hand side of a white-noise system (a Toeplitz N^-1 filters in time
 * order).  With the trig pair in 16-byte-aligned device memory the handle
 * keeps only the pixel-sorted pairs at first (and, with pix there too, no
 * time-ordered pixel copy); the first time-ordered operator
 * (bm_pointing_apply, a Toeplitz or offset-template matvec or solve) builds
 * the time-ordered ones from the sorted order (8 + 4 bytes a sample, memory
 * allocated then; that call must not be inside a stream capture, else
 * BM_ERR_INVALID).  This entry point has no counterpart in the paper.  Errors as
 * bm_pointing_create; BM_ERR_INVALID when both or neither of psi and the trig
 * pair are given, or tod is NULL. */
bm_status bm_pointing_create_with_tod(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                      const void* psi, bm_dtype psi_dtype, const float* cos2psi,
                                      const float* sin2psi, const float* tod, bm_solver_type solver,
                                      bm_pointing** out);
/* Pointing whose polarisation angle is rebuilt on the device from a rotating
 * half-wave plate instead of being read per sample (Eq. 2: the angle theta
 * includes the optics).  Sample k of detector d (k counted from the
 * detector's first sample, samples laid out detector by detector) has
 *     theta = psi_det[d] + 2 phi_hwp(k),
 *     phi_hwp(k) = 2 pi hwp_turns_per_sample k + hwp_phase0,
 * hwp_turns_per_sample = f_hwp / f_samp (taken modulo 1 and to 2^-64 of a
 * turn: exact for every FP64 value of at least 2^-11), hwp_phase0 in radians.
 * The phase is reduced exactly in 64-bit fixed point, so the angle keeps
 * FP64 accuracy however long the detector.  pix as for bm_pointing_create
 * (device or page-locked host int32 [nsamples]); det_offsets host int64
 * [ndet + 1] (det_offsets[0] = 0, increasing, det_offsets[ndet] =
 * nsamples); psi_det host FP64 [ndet].  The handle keeps what
 * bm_pointing_create keeps for the FP64 angles of this model (the FP64
 * operator, blocks and right-hand sides read them), and the mixed-precision
 * white-noise matvec with a per-detector N^-1 rebuilds (cos 2 theta,
 * sin 2 theta) in FP32 from each pixel-sorted sample's time index (4 bytes a
 * sample) instead of streaming a stored weighted pair (8 bytes a sample).
 * Errors as bm_pointing_create, and BM_ERR_INVALID for bad det_offsets or a
 * non-finite angle or rate.  This entry point has no counterpart in the
 * paper. */
bm_status bm_pointing_create_hwp(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                 int32_t ndet, const int64_t* det_offsets, const double* psi_det,
                                 double hwp_turns_per_sample, double hwp_phase0, bm_solver_type solver,
                                 bm_pointing** out);
void bm_pointing_destroy(bm_pointing* p);
/* hits device int32 [npix]: samples per pixel (flagged samples excluded). */
bm_status bm_pointing_get_hits(const bm_pointing* p, int32_t* hits);
/* The pixel-sorted sample order the operators run in (the precomputation
 * of Sec. III-A item 1, which groups the samples of each pixel for P^T):
 * *nvalid (host, may be NULL) receives the number of non-flagged samples,
 * and order (device uint32 [nvalid], caller-owned; may be NULL to ask for
 * the count alone) their time indices in increasing pixel, samples of one
 * pixel in time order (the stable sort by pixel).  Synchronous.
 * BM_ERR_INVALID for a NULL handle. */
bm_status bm_pointing_get_order(const bm_pointing* p, uint32_t* order, int64_t* nvalid);
/* y = P x (the paper's PointingLO): x device FP64 [npix][ncomp], y device
 * FP64 [nsamples]; every non-flagged sample, no mask.  FP64 arithmetic. */
bm_status bm_pointing_apply(bm_pointing* p, const double* x, double* y);
/* x = P^T y (PointingLO.T): y device FP64 [nsamples], x device FP64
 * [npix][ncomp].  Deterministic (pixel-sorted segmented sums, no atomics). */
bm_status bm_pointing_apply_transpose(bm_pointing* p, const double* y, double* x);

/* ---------------------------------------------------------- inverse noise */

/* Diagonal white N^-1 (the paper's InvNoiseCovUnCorr): inv_var host FP64
 * [ndet] = 1/sigma_d^2 > 0, det_offsets host int64 [ndet+1], increasing,
 * det_offsets[0] = 0. */
bm_status bm_inv_noise_create_diag(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                   const double* inv_var, bm_inv_noise** out);
/* Banded symmetric Toeplitz N^-1 applied chunk by chunk: each detector's
 * samples are cut into chunks of chunk_len (the last one may be shorter) and
 *   z_t = c_0 y_t + sum_{k=1}^{nlags-1} c_k (y_{t-k} + y_{t+k}),
 * with y = 0 outside the chunk.  coeffs host FP64 [ndet][nlags];
 * white_inv_var host FP64 [ndet] is diag(N)^-1 of Eq. 7 for the
 * preconditioner.  1 <= nlags <= 1024, chunk_len >= 1. */
bm_status bm_inv_noise_create_toeplitz(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                       int64_t chunk_len, int32_t nlags, const double* coeffs,
                                       const double* white_inv_var, bm_inv_noise** out);
/* Diagonal N^-1 = W with a weight per sample: the general weighting of
 * Eq. 4 restricted to a diagonal W (s = (P^T W P)^-1 P^T W d), which covers
 * gap treatment (weight 0 for samples to ignore) and sample-dependent noise
 * levels.  weights FP64 [nsamples], each >= 0 and finite, in device or
 * page-locked host memory; copied, so the caller may free them on return.
 * The preconditioner of Eq. 7 is then exact per pixel (A is block diagonal),
 * as for white noise; bm_blockdiag_precond_create gathers the weights into
 * pixel-sorted order once (20 bytes a kept sample on the device).  Errors:
 * BM_ERR_INVALID for nsamples outside [1, 2^32) or a negative or non-finite
 * weight. */
bm_status bm_inv_noise_create_sample_weights(bm_context* ctx, int64_t nsamples, const double* weights,
                                             bm_inv_noise** out);
/* White N^-1 with one baseline offset per interval marginalised out: the
 * general weighting of Eq. 4 with the offsets as a filtering template
 * (Sec. IV names filtering templates among the needs of real data),
 *   W = Nk - Nk F (F^T Nk F)^-1 F^T Nk,
 * F the indicator matrix of the intervals (each detector's samples cut into
 * intervals of baseline_len, the last one possibly shorter), Nk the white N^-1
 * (inv_var host FP64 [ndet], as for bm_inv_noise_create_diag) restricted to
 * the kept samples of the system (not flagged, pixel not masked).  On a kept
 * sample of interval I, (W y)_t = w_d (y_t - mean of y over I's kept samples).
 * A constant I map is an offset on every interval, so the I monopole is in
 * the null space of A: the solve converges to one solution of a consistent
 * system, defined up to that monopole.  The preconditioner of Eq. 7 uses
 * diag(N)^-1 = w_d; it must be built from this noise handle (it also counts
 * each interval's kept samples).  bm_inv_noise_apply takes every sample as
 * kept.  Errors: BM_ERR_INVALID for baseline_len < 1 or the det_offsets /
 * inv_var rules of bm_inv_noise_create_diag; at solve time for a
 * preconditioner built from another noise handle. */
bm_status bm_inv_noise_create_offset_filter(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                            const double* inv_var, int64_t baseline_len, bm_inv_noise** out);
void bm_inv_noise_destroy(bm_inv_noise* n);
/* z = N^-1 y in FP64: y, z device FP64 [nsamples]. */
bm_status bm_inv_noise_apply(bm_inv_noise* n, const double* y, double* z);

/* --------------------------------------------------------- preconditioner */

/* Block-diagonal preconditioner of Eq. 7 with the pixel mask: the blocks
 * B_p = sum_{t in p} w_d(t) v_t v_t^T (w = the noise's white level) are
 * accumulated in FP64; a pixel is masked when hits < min_hits, or, for QU
 * and IQU, when lambda_min(B_p) <= 0 or lambda_max/lambda_min > max_cond
 * (strict); M_p = B_p^-1 on kept pixels.  Masked pixels leave the solve.
 * p and n must describe the same samples (same context). */
bm_status bm_blockdiag_precond_create(bm_pointing* p, bm_inv_noise* n, int32_t min_hits,
                                      double max_cond, bm_precond** out);
void bm_precond_destroy(bm_precond* pc);
/* mask device uint8 [npix] (1 = masked), hits device int32 [npix]; either may be NULL. */
bm_status bm_precond_get_mask(const bm_precond* pc, uint8_t* mask, int32_t* hits);
/* blocks device FP64 [npix][ncomp][ncomp]: B_p (not inverted); cond device
 * FP64 [npix] (inf where lambda_min <= 0, 0 for empty pixels).  Either may be NULL. */
bm_status bm_precond_get_blocks(const bm_precond* pc, double* blocks, double* cond);
/* z = M r per pixel (zero on masked pixels): r, z device FP64 [npix][ncomp]. */
bm_status bm_precond_apply(bm_precond* pc, const double* r, double* z);

/* ------------------------------------------------------------ the system */

/* b = P^T N^-1 d_m (Eq. 6) where d_m is d with the samples of flagged or
 * masked pixels set to 0: tod device [nrhs][nsamples] of dtype tod_dtype,
 * b device FP64 [nrhs][npix][ncomp].  FP64 arithmetic, deterministic.
 * tod = NULL uses the TOD the pointing was created with
 * (bm_pointing_create_with_tod; nrhs = 1, white noise, tod_dtype unused but
 * checked); else BM_ERR_INVALID. */
bm_status bm_rhs(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod,
                 bm_dtype tod_dtype, int32_t nrhs, double* b);

/* q = A x = P^T N^-1 P x on kept pixels (zero on masked ones): x, q device
 * FP64 [npix][ncomp].  BM_PREC_FP64: FP64 products and sums.  BM_PREC_MIXED:
 * FP32 per-sample products and filter, FP64 per-pixel accumulation (the
 * operator the inner solve of the mixed path uses).  White noise streams the
 * samples in pixel-sorted order; Toeplitz noise gathers in time order,
 * filters each chunk, and reduces in pixel-sorted order.  Deterministic. */
bm_status bm_matvec(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q,
                    bm_precision prec);

/* q = A x for white noise with FP32 per-sample products -- the same operator
 * and the same result as bm_matvec(p, n, pc, x, q, BM_PREC_MIXED) -- for
 * callers that cannot allocate device memory during the call (a process
 * whose free device memory belongs to another allocator, or a pipeline that
 * fixes its memory budget before it starts).  This entry point has no
 * counterpart in the paper.  It allocates nothing: its scratch is a 16 MiB
 * array built into the library, present on every GPU that loads the library
 * until the process exits.  The array holds one FP64 value per work item and
 * Stokes component; a problem needing more than 2^21 values is rejected
 * with BM_ERR_INVALID (use bm_matvec).  x, q device FP64 [npix][ncomp]; n
 * must be the diagonal noise pc was built from (a weight per detector or
 * per sample).  bm_context_create looks the array's address up and loads
 * the kernels' code, so no call maps memory, not even the first.  The call
 * synchronises the context stream before it returns (so it cannot be
 * captured into a CUDA graph).  All calls share the array: calls that
 * overlap on the GPU race, so serialise them. */
bm_status bm_matvec_white_static(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x,
                                 double* q);

/* GLS maps by block-preconditioned CG (Eq. 5-7): tod [nrhs][nsamples]
 * (tod_dtype) in device memory, or in page-locked host memory, which is then
 * uploaded into a library workspace first, or NULL for the TOD the pointing
 * was created with (as bm_rhs); map_out device FP64
 * [nrhs][npix][ncomp] (NaN on masked
 * pixels).  x0 = 0; stops when ||b - A x||_2 <= tol ||b||_2 (per RHS) or
 * after maxiter PCG iterations (maxiter counts inner iterations in mixed
 * mode).  info host [nrhs] (may be NULL).  Returns BM_OK when every RHS
 * converged, otherwise the first non-OK per-RHS status. */
bm_status bm_pcg_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod,
                       bm_dtype tod_dtype, int32_t nrhs, double* map_out, double tol,
                       int32_t maxiter, bm_precision prec, bm_solve_info* info);

/* --------------------------------------------------------------- serving */

/* A request loop that runs map-making solves as they arrive (continuous
 * batching): up to max_slots requests run at once, each in its own slot with
 * its own CUDA stream, so their device work overlaps; a request is admitted
 * when a slot is free and its estimated device memory fits in what is left of
 * hbm_budget_bytes (first come, first served; the head of the queue waits for
 * memory rather than being overtaken, except by requests that wait for a
 * resident pointing in use).  A request that fails to allocate while other
 * requests hold memory is queued again (at most three times) and runs after
 * one of them has finished.
 *
 * Resident pointings: requests that carry the same nonzero pointing_key
 * share one pointing (the caller promises equal npix, nsamples, solver,
 * det_offsets and pixel and angle values, in whatever buffers).  The first
 * such request leaves the ingested pointing, its noise model and its
 * preconditioner resident on the device after it completes; later requests
 * with the key reuse them (the noise model and preconditioner are rebuilt
 * when the noise levels, min_hits or max_cond differ), so their cost is the
 * RHS and the PCG alone.  Resident pointings count against the budget and
 * the least recently used one that no request is using is released when an
 * admitted request needs its memory.
 *
 * Batching: when a slot takes a white-noise mixed-precision request with a
 * pointing_key, every queued request with the same key, noise levels,
 * min_hits, max_cond, tol, maxiter and TOD dtype joins it (as many as the
 * memory left allows, at most 256), and they are solved together by the
 * multi-RHS PCG of bm_pcg_solve (one pass over the pointing for all of
 * them).  A request's map from a batch agrees with its map solved alone to
 * the rounding of the per-RHS CG scalars (their reduction tree depends on the
 * batch size); a request without a key, or that is not batched, is exactly
 * the computation of bm_pointing_create(_trig) + bm_inv_noise_create_* +
 * bm_blockdiag_precond_create + bm_pcg_solve, so its map does not depend on
 * what else is running.  All bm_serve_* calls are thread-safe.  This loop has
 * no counterpart in the paper. */
typedef struct bm_server bm_server;
typedef enum { BM_NOISE_WHITE = 0, BM_NOISE_TOEPLITZ = 1 } bm_noise_kind;

/* One map-making request.  Device arrays are the caller's and must stay
 * valid until bm_serve_poll reports the request finished; host arrays are
 * copied by bm_serve_submit. */
typedef struct {
    int64_t npix, nsamples;
    bm_solver_type solver;
    const int32_t* pix;          /* device [nsamples], -1 = flagged */
    const float* cos2psi;        /* device [nsamples] FP32 trig, or NULL to use psi */
    const float* sin2psi;        /* device [nsamples] */
    const void* psi;             /* device [nsamples] (when cos2psi is NULL) */
    bm_dtype psi_dtype;
    int32_t ndet;
    const int64_t* det_offsets;  /* host [ndet + 1] */
    bm_noise_kind noise;
    const double* inv_var;       /* host [ndet]: white level 1/sigma_d^2 */
    int64_t chunk_len;           /* Toeplitz: chunk length */
    int32_t nlags;               /* Toeplitz: band length */
    const double* coeffs;        /* host [ndet][nlags] (Toeplitz) */
    const void* tod;             /* device [nsamples] */
    bm_dtype tod_dtype;
    int32_t min_hits;
    double max_cond;
    double tol;
    int32_t maxiter;
    bm_precision precision;
    double* map_out;             /* device [npix][ncomp], written by the solve */
    uint64_t pointing_key;       /* 0, or the caller's name of a shared pointing (see above) */
} bm_request;

typedef struct {
    int32_t status;              /* bm_status of the solve */
    int32_t iterations, outer_iterations, slot;
    double rel_residual;
    double queue_ms;             /* submit -> start */
    double run_ms;               /* start -> finish */
    double latency_ms;           /* submit -> finish */
    int64_t device_bytes;        /* memory reserved for the request */
    char message[256];           /* bm_last_error() of a failed solve, else "" */
    int32_t batch_size;          /* right-hand sides solved together with this one (1 = alone) */
    int32_t resident;            /* 1 when the request reused a resident pointing */
} bm_result;

typedef struct {
    int64_t submitted, completed, rejected, cancelled, running, queued;
    double p50_ms, p99_ms, mean_ms;   /* latency over completed requests */
    double samples_per_s;             /* samples of completed requests / wall time since creation */
    int64_t budget_bytes, reserved_bytes, peak_reserved_bytes;
    int64_t resident_bytes;           /* estimated memory of the resident pointings */
    int64_t resident_hits;            /* requests that reused a resident pointing */
    int64_t batches, batched_requests;/* multi-RHS solves run, and the requests in them */
    int64_t evictions, oom_requeues;  /* resident pointings released; requests queued again */
} bm_serve_stats;

/* Server on ctx's device with max_slots in [1, 64] slots. */
bm_status bm_serve_create(bm_context* ctx, size_t hbm_budget_bytes, int32_t max_slots, bm_server** out);
/* Queue a request; *ticket identifies it.  BM_ERR_BUSY if its estimated
 * device memory exceeds the whole budget (it could never run). */
bm_status bm_serve_submit(bm_server* s, const bm_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (0 = just check) for the request to finish:
 * BM_OK and *out filled when finished (the ticket is then released),
 * BM_ERR_TIMEOUT if still queued or running, BM_ERR_NOT_FOUND for an
 * unknown or released ticket. */
bm_status bm_serve_poll(bm_server* s, uint64_t ticket, int32_t timeout_ms, bm_result* out);
/* Cancel a queued request (BM_OK); BM_ERR_BUSY if it is already running,
 * BM_ERR_NOT_FOUND if unknown.  A cancelled request reports BM_ERR_NOT_FOUND
 * in its result status. */
bm_status bm_serve_cancel(bm_server* s, uint64_t ticket);
bm_status bm_serve_get_stats(bm_server* s, bm_serve_stats* out);
/* Stop accepting, cancel queued requests, wait for running ones, release. */
void bm_serve_destroy(bm_server* s);

#ifdef __cplusplus
}
#endif

#endif /* BRAHMAP_H */
