// Internal declarations of the GB300 GLS map-making library: handle layouts,
// error plumbing, device helpers and the launch wrappers shared between
// translation units.  Nothing here is part of the C-ABI (include/brahmap.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/brahmap.h"

namespace bm {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

struct Error {
    bm_status status;
};

#define BM_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::bm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                            __LINE__);                                                      \
            throw ::bm::Error{e_ == cudaErrorMemoryAllocation ? BM_ERR_OOM : BM_ERR_CUDA};  \
        }                                                                                   \
    } while (0)

#define BM_REQUIRE(cond, ...)                 \
    do {                                      \
        if (!(cond)) {                        \
            ::bm::set_error(__VA_ARGS__);     \
            throw ::bm::Error{BM_ERR_INVALID}; \
        }                                     \
    } while (0)

// Every kernel launch of the library goes through BM_LAUNCH_CHECK, which
// also counts it (bm_kernel_launches()).
void count_launch();
#define BM_LAUNCH_CHECK()              \
    do {                               \
        ::bm::count_launch();          \
        BM_CUDA(cudaGetLastError());   \
    } while (0)

// Stream of the context whose entry point is running on this thread; device
// buffers are allocated and freed stream-ordered on it (cudaMallocAsync from
// the device's memory pool, which keeps freed memory for reuse).
extern thread_local cudaStream_t tl_stream;

// Device allocation that throws BM_ERR_OOM and is released by DevBuf's destructor.
template <typename T>
struct DevBuf {
    T* ptr = nullptr;
    size_t n = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), n(o.n), stream(o.stream) { o.ptr = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr; n = o.n; stream = o.stream;
            o.ptr = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        void* p = nullptr;
        stream = tl_stream;
        cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), stream);
        if (e == cudaErrorMemoryAllocation) {
            // the pool may hold memory freed by finished work: release it to
            // the device once and retry
            (void)cudaGetLastError();
            int dev = 0;
            cudaMemPool_t pool = nullptr;
            if (cudaStreamSynchronize(stream) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
                cudaMemPoolTrimTo(pool, 0);
            e = cudaMallocAsync(&p, count * sizeof(T), stream);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
            throw Error{BM_ERR_OOM};
        }
        ptr = static_cast<T*>(p);
        n = count;
    }
    // The same from a given memory pool (NULL: the device's default pool).
    void alloc_from(cudaMemPool_t pool, size_t count) {
        if (!pool) {
            alloc(count);
            return;
        }
        release();
        if (count == 0) return;
        void* p = nullptr;
        stream = tl_stream;
        cudaError_t e = cudaMallocFromPoolAsync(&p, count * sizeof(T), pool, stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
            throw Error{BM_ERR_OOM};
        }
        ptr = static_cast<T*>(p);
        n = count;
    }
    void release() {
        if (ptr) cudaFreeAsync(ptr, stream);
        ptr = nullptr;
        n = 0;
    }
    T* get() const { return ptr; }
};

// Per-kernel-family device time, measured with events on the context stream.
struct KernelTimer {
    double total_ms = 0.0;
    int64_t launches = 0;
};

}  // namespace bm

// ----------------------------------------------------------------- handles
struct bm_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    bool timing = false;
    std::map<std::string, bm::KernelTimer> timers;
    // Event pairs recorded around timed kernels; resolved when queried, so
    // timing never blocks the host inside a solve.
    struct Pending { std::string name; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double* h_pinned = nullptr;  // small pinned host buffer for scalar reads
    // Named grow-only scratch buffers, from a pool of their own: long-lived
    // workspaces taken between the allocations of short-lived handles would
    // split the default pool's blocks and make later large allocations map
    // new memory.
    cudaMemPool_t ws_pool = nullptr;
    std::map<std::string, bm::DevBuf<char>> ws;
    uint64_t ws_generation = 0;  // bumped when a workspace is (re)allocated: graphs holding its address are stale
    // Library-owned stream for CUDA-graph capture and replay (the caller's
    // stream may be the legacy default stream, which cannot be captured),
    // ordered against `stream` with side_ev.
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev = nullptr;
    // Whether solves may capture their iterations into CUDA graphs.  Off for
    // the server's contexts: while a stream captures, a device-wide
    // synchronisation by any other thread of the process fails, and the
    // server runs next to the caller's own threads.
    bool graphs = true;
    // Device address of the allocation-free matvec's static scratch array on
    // this context's device (looked up when the context is created).
    double* static_scratch = nullptr;
    // Detector-sharded solve (bm_context_set_allreduce): the caller's sum of
    // per-pixel partial results over the ranks; NULL on an unsharded context.
    bm_allreduce_fn allreduce = nullptr;
    void* allreduce_user = nullptr;
};

namespace bm {
// The angle model of a half-wave-plate pointing (bm_pointing_create_hwp): the
// angle 2 theta of sample k of detector d, in turns, is
// turn0[d] + 4 frac(nu k) (mod 1), all as 64-bit fixed-point fractions of a
// turn, so the phase is reduced exactly.
struct HwpModel {
    const uint32_t* off = nullptr;            // [ndet + 1] sample offsets
    const unsigned long long* turn0 = nullptr;  // [ndet] (2 psi_d + 4 phi0) / (2 pi) mod 1
    unsigned long long nu = 0;                // turns per sample mod 1
    int ndet = 0;
    uint32_t ns = 0;                          // samples per detector when all are equal, else 0
    float inv_ns = 0.f;
    const float4* tabdf = nullptr;            // [kHwpTab] (cos, sin)(2 pi j / kHwpTab) as double-float
                                              // pairs: (cos hi, sin hi, cos lo, sin lo)
};
}  // namespace bm

struct bm_pointing {
    bm_context* ctx = nullptr;
    int64_t npix = 0, nsamples = 0, nvalid = 0;
    int ncomp = 3;
    bm::DevBuf<int32_t> pix;       // [nsamples] time order, -1 = flagged; read through bm::time_pix,
                                   //   which builds it on first use when deferred
    bool pix_deferred = false;     // pix not built yet (a pointing carrying a TOD, pixels in device memory)
    bm::DevBuf<float2> cs_hi_t;    // [nsamples] (cos 2psi, sin 2psi) rounded to FP32; read through
                                   //   bm::time_trig, which builds it on first use when deferred
    bool trig_t_deferred = false;  // cs_hi_t not built yet (a pointing carrying a TOD, given cos/sin)
    bm::DevBuf<float2> cs_lo_t;    // [nsamples] FP64 value minus hi, rounded to FP32
    bm::DevBuf<uint32_t> perm;     // [nvalid] sample index, pixel-sorted (stable)
    bm::DevBuf<int64_t> off;       // [npix + 1] CSR offsets into perm
    bm::DevBuf<int32_t> hits;      // [npix]
    bm::DevBuf<float2> cs_hi_s;    // [nvalid] trig in pixel-sorted order
    bm::DevBuf<float2> cs_lo_s;
    bm::DevBuf<float> tod_s;       // [nvalid] a TOD sorted along with the samples, or empty
    // Half-wave-plate angle model (bm_pointing_create_hwp), else hwp = false.
    bool hwp = false;
    bm::HwpModel hwp_model;                 // device pointers into the buffers below
    bm::DevBuf<uint32_t> hwp_off;           // [ndet + 1]
    bm::DevBuf<unsigned long long> hwp_turn0;  // [ndet]
    bm::DevBuf<float2> hwp_tab;             // [kHwpTab] (cos, sin)(2 pi j / kHwpTab) in FP32
    bm::DevBuf<float4> hwp_tab_df;          // [kHwpTab] the same as double-float pairs
};

struct bm_inv_noise {
    bm_context* ctx = nullptr;
    int kind = 0;  // 0 = diagonal white (a weight per detector), 1 = banded Toeplitz,
                   // 2 = diagonal with a weight per sample (wsamp), 3 = white with a
                   // baseline offset per interval marginalised out
    int ndet = 0;
    int64_t nsamples = 0;
    std::vector<int64_t> h_det_off;
    std::vector<double> h_white;   // diag(N)^-1 per detector (the white level)
    bm::DevBuf<int64_t> det_off;   // [ndet + 1]
    bm::DevBuf<double> white;      // [ndet]
    bm::DevBuf<double> wsamp;      // kind 2: [nsamples] weight of every sample, time order
    bm::DevBuf<uint32_t> det_off32;  // [ndet + 1] (nsamples < 2^32)
    bm::DevBuf<float2> wdf;          // [ndet] white level as double-float (hi, lo)
    bm::DevBuf<float> wsqrt;         // [ndet] sqrt of the white level, FP32
    // Offset filter: each detector's samples cut into intervals of
    // baseline_len (the last one may be shorter); int_start[d] = the index of
    // detector d's first interval, int_start[ndet] = nint.
    int64_t baseline_len = 0;
    int64_t nint = 0;
    bm::DevBuf<int64_t> int_start;  // [ndet + 1]
    // Toeplitz
    int64_t chunk_len = 0;
    int nlags = 0;
    bm::DevBuf<double> coeffs64;   // [ndet][nlags]
    bm::DevBuf<float> coeffs32;    // [ndet][nlags]
    // FFT overlap-save form of the band (sizes 0 = use the direct filter).
    uint32_t ns_uniform = 0;       // samples per detector when all are equal (and < 2^20 detectors), else 0
    float inv_ns = 0.f;
    int fft_n32 = 0, fft_n64 = 0;
    bm::DevBuf<float> spec32;      // [ndet][fft_n32/2 + 1] real band spectrum
    bm::DevBuf<double> spec64;     // [ndet][fft_n64/2 + 1]
    bm::DevBuf<float2> spec_df;    // the same as double-float (hi, lo) pairs
    bm::DevBuf<float2> tw32;       // [fft_n32] exp(-2 pi i e / N)
    bm::DevBuf<double2> tw64;      // [fft_n64]
    // Filter tiling per tile length: [ndet + 1] prefix of tiles per detector
    // on the device, built on first use.
    struct TilePlan {
        bm::DevBuf<int64_t> tile_start;
        int64_t tiles_per_chunk = 0, ntiles = 0;
    };
    std::map<int, TilePlan> tile_plans;
};

struct bm_precond {
    bm_context* ctx = nullptr;
    bm_pointing* p = nullptr;
    bm_inv_noise* n = nullptr;
    int ncomp = 3, nsym = 6;
    int32_t min_hits = 3;
    double max_cond = 1e3;
    int64_t nkept = 0;
    bm::DevBuf<double> B;          // [npix][ncomp*ncomp] full symmetric block
    bm::DevBuf<double> Minv;       // [npix][ncomp*ncomp]
    bm::DevBuf<double> cond;       // [npix]
    bm::DevBuf<uint8_t> mask;      // [npix]
    bm::DevBuf<int32_t> hits_global;  // [npix] hit counts over all ranks (sharded context), else empty
    // Work items: pieces (<= item_max samples) of kept pixels' sorted segments.
    int64_t nitems = 0;
    bm::DevBuf<int32_t> item_pix;  // [nitems]
    bm::DevBuf<int64_t> item_beg;  // [nitems]
    bm::DevBuf<int32_t> item_len;  // [nitems]
    bm::DevBuf<int64_t> pitem;     // [npix + 1] CSR: items of pixel p
    // White noise: weighted sorted stream sqrt(w) (cos, sin) (or w for I-only).
    bm::DevBuf<float2> wcs;        // [nvalid]
    bm::DevBuf<float> w1;          // [nvalid] (I-only)
    // White noise and a TOD carried by the pointing: b = P^T N^-1 d_m of that
    // TOD in double-float (the mixed solve's RHS), zero on masked pixels.
    bm::DevBuf<double> b_tod;      // [npix][ncomp] or empty
    // Noise with a weight per sample: the weights in pixel-sorted order.
    bm::DevBuf<float2> ws_df;      // [nvalid] double-float
    bm::DevBuf<float> ws_sqrt;     // [nvalid] sqrt(w) in FP32
    bm::DevBuf<double> ws64;       // [nvalid] FP64
    // Toeplitz noise, inner operator's transpose by time chunks (built on
    // first use; pt_nch = 0 not built yet, -1 not used): the kept samples'
    // time index and trig pair in (time chunk, pixel, time) order, and the
    // segments of that order (one per chunk and pixel with samples there),
    // chunk by chunk.
    int pt_nch = 0;
    bm::DevBuf<uint32_t> cm_t;     // [kept samples] time index
    bm::DevBuf<float2> cm_cs;      // [kept samples] trig pair (FP32 hi)
    bm::DevBuf<int32_t> seg_pix;   // [segments] pixel
    bm::DevBuf<uint32_t> seg_beg;  // [segments] first position in cm_t / cm_cs
    bm::DevBuf<int32_t> seg_len;   // [segments] samples
    bm::DevBuf<int32_t> seg_mid;   // [segments] samples in the first half of the segment's chunk
    std::vector<int64_t> cseg;     // [pt_nch + 1] first segment of each chunk (host)
    // Offset filter: 1 / (the kept samples of each interval), 0 where none;
    // the interval of every sample in pixel-sorted order.
    bm::DevBuf<double> ofs_inv;    // [nint]
    bm::DevBuf<uint32_t> ofs_isort;  // [nvalid]
};

namespace bm {

constexpr int kItemMax = 4096;  // max samples per work item
constexpr int kBatchMax = 256;  // right-hand sides per batched solve

// Batched mixed-precision solve of nrhs white-noise right-hand sides sharing
// one pointing (groups of at most kBatchMax).
bm_status batched_white_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod, bm_dtype dt,
                              int32_t nrhs, double* map_out, double tol, int32_t maxiter, bm_solve_info* info);
// The same from separate buffers: rows[r] is RHS r's device TOD
// [nsamples], maps[r] its device map [npix][ncomp] (host arrays of nrhs
// pointers).
bm_status batched_white_solve_rows(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* const* rows,
                                   bm_dtype dt, int32_t nrhs, double* const* maps, double tol, int32_t maxiter,
                                   bm_solve_info* info);
// Adds kernels launched by a CUDA-graph replay to the launch counter.
void count_launches(int64_t n);

// Named grow-only scratch buffer owned by the context (released with it).
void* workspace(bm_context* ctx, const char* name, size_t bytes);
template <typename T>
T* workspace_as(bm_context* ctx, const char* name, size_t count) {
    return static_cast<T*>(workspace(ctx, name, count * sizeof(T)));
}

// Work items: pieces of <= kItemMax consecutive samples of one pixel's
// pixel-sorted segment, for every non-empty pixel (mask == NULL) or every
// kept pixel; pitem[p] .. pitem[p+1] are pixel p's items, in order.
struct Items {
    int64_t n = 0;
    DevBuf<int32_t> pix;
    DevBuf<int64_t> beg;
    DevBuf<int32_t> len;
    DevBuf<int64_t> pitem;  // [npix + 1]
};
void plan_items(bm_context* ctx, const int64_t* off, const uint8_t* mask, int64_t npix, Items& it);

// Device-wide exclusive scans.
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
// off[0..n] = exclusive prefix sums of counts[0..n) followed by the total.
void offsets_from_counts(const int32_t* counts, int64_t n, int64_t* off, cudaStream_t s);

// Deterministic FP64 reductions with a fixed grid: out = sum_i a_i b_i.
constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;

// Timing helpers
struct ScopedTimer {
    bm_context* ctx;
    const char* name;
    cudaEvent_t a = nullptr;
    ScopedTimer(bm_context* c, const char* n);
    ~ScopedTimer();
};
void resolve_timers(bm_context* ctx);

// Sum of a device FP64 array over the ranks of a sharded context (in place;
// nothing on an unsharded one): synchronises the context stream, then calls
// the caller's reduction, which returns once buf holds the sum.
void shard_reduce(bm_context* ctx, double* buf, int64_t count);

// Device address of the static scratch array of bm_matvec_white_static on
// the current device, with the code of the kernels that use it loaded.
double* static_scratch_setup();

// Launch wrappers implemented in the .cu files.
// The time-ordered trig pairs of p (cs_hi_t), built from the pixel-sorted
// pairs on the first call when the ingest deferred them (flagged samples
// get (0, 0)); an error inside a stream capture, where it cannot allocate.
const float2* time_trig(bm_pointing* p);
// The time-ordered pixel indices of p (-1 = flagged), built from the CSR
// offsets and perm on the first call when the ingest deferred them (a lazily
// filled part of the handle, hence the const argument); an error inside a
// stream capture.
const int32_t* time_pix(const bm_pointing* p);
void ingest(bm_pointing* p, const int32_t* pix, const void* psi, bm_dtype psi_dtype, const float* cos2psi,
            const float* sin2psi, const float* tod = nullptr, bool tod_on_host = false,
            const HwpModel* hwp = nullptr);
void build_precond(bm_precond* pc);
void matvec(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q,
            bm_precision prec, int64_t nrhs);
// Internal precision of the mixed solve's refinement operator: like
// BM_PREC_FP64, with the Toeplitz filter and its pixel sums in double-float.
constexpr bm_precision kPrecRefine = static_cast<bm_precision>(2);
// b = P^T N^-1 d_m; df = double-float accumulation and filter (mixed path)
// instead of FP64.
void rhs(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod, bm_dtype dt,
         int64_t nrhs, double* b, bool df = false);
void precond_apply(bm_precond* pc, const double* r, double* z, int64_t nrhs);
void pointing_apply(bm_pointing* p, const double* x, double* y);
void pointing_apply_transpose(bm_pointing* p, const double* y, double* x);
void inv_noise_apply(bm_inv_noise* n, const double* y, double* z);
// Band spectra and twiddle tables for the FFT form of a Toeplitz noise model.
void prepare_toeplitz_fft(bm_inv_noise* n);
// pc->ofs_inv of an offset-filter noise from the pointing and the pixel mask.
void build_offset_counts(bm_precond* pc);
void ang2pix_ring(bm_context* ctx, int64_t nside, int64_t n, const double* z, const double* phi,
                  int32_t* pix);
bm_status pcg_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod,
                    bm_dtype dt, int32_t nrhs, double* map_out, double tol, int32_t maxiter,
                    bm_precision prec, bm_solve_info* info);

// Grid sizing: a multiple of the SM count.
inline int grid_for(const bm_context* ctx, int64_t work_units, int per_sm = 8) {
    int64_t g = (int64_t)ctx->num_sms * per_sm;
    if (work_units < g) g = work_units > 0 ? work_units : 1;
    return (int)g;
}

// Raises (never lowers) a kernel's dynamic shared-memory limit on the current
// device; safe against concurrent launches of the same kernel.
void ensure_smem_limit(const void* kernel, size_t bytes);

// Resident blocks per SM of a kernel at a block size (queried once per kernel).
int blocks_per_sm(const void* kernel, int threads, size_t smem);

// Persistent grid: exactly the number of blocks that are resident at once
// (SM count x occupancy), capped by the work, so a grid-stride loop runs in a
// single wave.
template <typename K>
int resident_grid(const bm_context* ctx, K kernel, int threads, int64_t work_units, size_t smem = 0) {
    const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kernel), threads, smem);
    return grid_for(ctx, work_units, per_sm > 0 ? per_sm : 1);
}

}  // namespace bm

// ---------------------------------------------------------- device helpers
#ifdef __CUDACC__
namespace bm {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-detector tables of a noise model (device pointers).
struct DetTables {
    const uint32_t* off;   // [ndet + 1] sample offsets
    const float2* wdf;     // [ndet] white weight w as a double-float (hi, lo)
    const float* wsqrt;    // [ndet] sqrt(w) rounded to FP32
    uint32_t ns;           // samples per detector when all detectors have as many (else 0)
    float inv_ns;          // 1 / ns rounded to FP32
    // Per-sample weights (diagonal W with a weight per sample), in pixel-sorted
    // order, indexed like perm; null for per-detector weights.
    const float2* wsort = nullptr;    // [nvalid] w as a double-float
    const float* ssort = nullptr;     // [nvalid] sqrt(w) in FP32
    const double* w64sort = nullptr;  // [nvalid] w in FP64
};
constexpr int kMaxDetSmem = 2048;  // detector tables staged in shared memory up to this count

// The weight tables of a diagonal noise model for the pixel-sorted kernels:
// per detector, plus (weights per sample) the preconditioner's sorted copy.
inline DetTables det_tables(const bm_inv_noise* n, const bm_precond* pc) {
    DetTables t{n->det_off32.get(), n->wdf.get(), n->wsqrt.get(), n->ns_uniform, n->inv_ns};
    if (n->kind == 2 && pc) {
        t.wsort = pc->ws_df.get();
        t.ssort = pc->ws_sqrt.get();
        t.w64sort = pc->ws64.get();
    }
    return t;
}
// N^-1 diagonal (a weight per detector or per sample): A = P^T N^-1 P is block
// diagonal and the white-noise paths apply.
inline bool diagonal_noise(const bm_inv_noise* n) { return n->kind == 0 || n->kind == 2; }

__device__ __forceinline__ int find_det32(const uint32_t* off, int ndet, uint32_t t) {
    int lo = 0, hi = ndet - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Detector of sample t.  When every detector has ns samples it is t / ns:
// the quotient from the FP32 reciprocal is within one of the true value
// (relative error ~2e-7 and fewer than 2^20 detectors), and one compare each
// way corrects it.  Otherwise a binary search of the offsets.
__device__ __forceinline__ int det_of(const uint32_t* off, int ndet, uint32_t ns, float inv_ns, uint32_t t) {
    if (ns) {
        uint32_t q = (uint32_t)__fmul_rz((float)t, inv_ns);
        if ((uint64_t)q * ns > t) --q;
        else if ((uint64_t)(q + 1) * ns <= t) ++q;
        return (int)q;
    }
    return find_det32(off, ndet, t);
}

// Angle 2 theta of sample t (time index) of a half-wave-plate pointing, in
// turns as a 64-bit fraction: turn0[d] + 4 frac(nu k), k = t - off[d].
__device__ __forceinline__ unsigned long long hwp_turns(const HwpModel& m, int d, uint32_t t) {
    const uint32_t k = t - (m.ns ? (uint32_t)d * m.ns : m.off[d]);
    return m.turn0[d] + ((m.nu * (unsigned long long)k) << 2);
}
// The top 32 bits of the turn fraction of sample k of a detector whose
// turn0 has top bits turn0_hi: turn0 + 4 frac(nu k), with frac(nu k) the
// exact 64-bit product nu k mod 2^64; the carry from the dropped low bits
// (at most one unit of 2^-32 of a turn) is left out.
__device__ __forceinline__ uint32_t hwp_turns32(unsigned long long nu, uint32_t turn0_hi, uint32_t k) {
    const uint32_t nlo = (uint32_t)nu, nhi = (uint32_t)(nu >> 32);
    const uint32_t plo = nlo * k;
    const uint32_t phi = __umulhi(nlo, k) + nhi * k;
    return turn0_hi + ((phi << 2) | (plo >> 30));
}
// (cos, sin) of 2 pi a for a turn fraction whose top 32 bits are a32, in
// FP32: the table entry of the top kHwpTabBits bits rotated by the remainder
// delta (< 2 pi / kHwpTab), cos delta = 1 - delta^2/2, sin delta =
// delta (1 - delta^2/6) (truncation errors below 1e-10); bits under 2^-32 of
// a turn are dropped.  Absolute error about 1.5e-7.
constexpr int kHwpTabBits = 10;
constexpr int kHwpTab = 1 << kHwpTabBits;
__device__ __forceinline__ float2 hwp_trig32(uint32_t a32, const float2* tab) {
    const float2 cs = tab[a32 >> (32 - kHwpTabBits)];
    const float dl = (float)(a32 & ((1u << (32 - kHwpTabBits)) - 1u)) * 1.4629180792671596e-9f;  // 2 pi / 2^32
    const float d2 = dl * dl;
    const float cd = fmaf(-0.5f, d2, 1.0f);
    const float sd = dl * fmaf(-0.16666667f, d2, 1.0f);
    return make_float2(fmaf(cs.x, cd, -cs.y * sd), fmaf(cs.y, cd, cs.x * sd));
}
// (cos, sin) of 2 pi a for a 64-bit turn fraction a, in FP32 (hwp_trig32 of
// its top 32 bits).
__device__ __forceinline__ float2 hwp_trig_f32(unsigned long long a, const float2* tab) {
    return hwp_trig32((uint32_t)(a >> 32), tab);
}

// Index of the detector owning sample t: largest d with off[d] <= t.
__device__ __forceinline__ int find_det(const int64_t* off, int ndet, int64_t t) {
    int lo = 0, hi = ndet - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double2 trig64(float2 hi, float2 lo) {
    return make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
}
// Trig pair of sorted/time sample i: hi + lo, where lo may be absent (exact FP32 trig).
__device__ __forceinline__ double2 trig64_at(const float2* hi, const float2* lo, int64_t i) {
    const float2 h = hi[i];
    if (lo == nullptr) return make_double2((double)h.x, (double)h.y);
    return trig64(h, lo[i]);
}

// ---- double-float arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2), carrying ~48 significant bits on the FP32
// pipes.  Built from the error-free transformations TwoSum (Knuth) and
// TwoProduct with a fused multiply-add; every operation uses the explicitly
// rounded intrinsics so the compiler cannot reassociate or contract them.
struct df32 {
    float hi, lo;
};
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ df32 df_quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df32 df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    const df32 s = df_two_sum(a.hi, b.hi);
    return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df32 df_add(df32 a, float b) {
    const df32 s = df_two_sum(a.hi, b);
    return df_quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    const df32 p = df_two_prod(a.hi, b.hi);
    const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_quick_two_sum(p.hi, lo);
}
__device__ __forceinline__ df32 df_mul(df32 a, float b) {
    const df32 p = df_two_prod(a.hi, b);
    return df_quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df32 df_from(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df32 df_shfl_xor(df32 a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ df32 df_warp_sum(df32 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
    return a;
}

// Lazily renormalised sums of many double-float terms.  A product is kept
// as an unnormalised pair (p, e): p = fl(a.hi b.hi), e = its exact rounding
// error plus the cross terms.  acc_add adds p to the accumulator's leading
// part exactly (two_sum) and the rounding error and e to its trailing part;
// acc_norm (every kLazyNorm terms of a lane, and before the lanes are
// combined) renormalises the pair.  The trailing part then stays within
// about kLazyNorm units of the leading part's last place: about a third
// fewer instructions than a normalised double-float product and sum per
// term, at an error of a few 2^-48 per term.
constexpr int kLazyNorm = 8;
__device__ __forceinline__ void prod_u(float hi, float lo, float b, float& p, float& e) {
    p = __fmul_rn(hi, b);
    e = __fmaf_rn(lo, b, __fmaf_rn(hi, b, -p));
}
__device__ __forceinline__ void prod_u2(float ah, float al, float bh, float bl, float& p, float& e) {
    p = __fmul_rn(ah, bh);
    e = __fmaf_rn(al, bh, __fmaf_rn(ah, bl, __fmaf_rn(ah, bh, -p)));
}
__device__ __forceinline__ void acc_add(df32& a, float p, float e) {
    const df32 s = df_two_sum(a.hi, p);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void acc_norm(df32& a) { a = df_two_sum(a.hi, a.lo); }

// (cos, sin) of 2 pi a for a 64-bit turn fraction a as double-float pairs,
// on the FP32 pipes (FP64 runs at 1/74 of their rate here): the table entry
// of the top kHwpTabBits bits rotated by the remainder delta (< 2 pi /
// kHwpTab = 0.0062), cos delta = 1 - delta^2/2 + delta^4/24, sin delta =
// delta - delta^3/6 + delta^5/120 (truncation below 8e-17); the remainder
// keeps its top 48 bits (2^-58 of a turn dropped), the rest is double-float
// arithmetic (~2^-46 relative).  Returns (cos hi, sin hi, cos lo, sin lo).
__device__ __forceinline__ float4 hwp_trig_df(unsigned long long a, const float4* tab) {
    const float4 t = tab[a >> (64 - kHwpTabBits)];
    const unsigned long long r = a & ((1ull << (64 - kHwpTabBits)) - 1ull);  // < 2^54
    // r 2^-64 as a double-float: (r >> 30) 2^-34 exactly, then the low 30 bits
    const df32 rt = df_quick_two_sum(__ull2float_rz(r >> 30) * 5.820766091346741e-11f,        // 2^-34
                                     __ull2float_rn(r & 0x3FFFFFFFull) * 5.421010862427522e-20f);  // 2^-64
    const df32 two_pi = {6.28318548202514648f, -1.74845553e-7f};
    const df32 dl = df_mul(rt, two_pi);
    const df32 d2 = df_mul(dl, dl);
    const df32 third = {-0.166666672f, 4.96705388e-9f};   // -1/6
    const df32 cdt = df_add(df32{-0.5f, 0.f}, d2.hi * 0.0416666679f);  // -1/2 + d2/24
    const df32 cd = df_add(df_mul(d2, cdt), 1.0f);
    const df32 sdt = df_add(third, d2.hi * 0.00833333377f);          // -1/6 + d2/120
    const df32 sd = df_mul(dl, df_add(df_mul(d2, sdt), 1.0f));
    const df32 c0 = {t.x, t.z}, s0 = {t.y, t.w};
    const df32 ssd = df_mul(s0, sd);
    const df32 c = df_add(df_mul(c0, cd), df32{-ssd.hi, -ssd.lo});
    const df32 s = df_add(df_mul(s0, cd), df_mul(c0, sd));
    return make_float4(c.hi, s.hi, c.lo, s.lo);
}

// One sample's terms of b = P^T N^-1 d (and of the weighted transposes) in
// the lazy form: val = d w (d a float: `dh`, dl = 0; or a double-float), then
// acc[I] += val, acc[Q] += val c, acc[U] += val s with the trig pair as
// double-float (hi, lo; lo = 0 for exact FP32 trig).  Shared by the block
// assembly's fused RHS and the pixel-sorted gather-reduce, so both give the
// same bits.
template <int NC>
__device__ __forceinline__ void rhs_term_lazy(df32* acc, float dh, float dl, bool weighted, float2 w, float2 h,
                                              float2 l) {
    float vp, ve;
    if (weighted) prod_u2(dh, dl, w.x, w.y, vp, ve);
    else { vp = dh; ve = dl; }
    if (NC != 2) acc_add(acc[0], vp, ve);
    if (NC > 1) {
        float p, e;
        prod_u2(vp, ve, h.x, l.x, p, e);
        acc_add(acc[NC - 2], p, e);
        prod_u2(vp, ve, h.y, l.y, p, e);
        acc_add(acc[NC - 1], p, e);
    }
}

}  // namespace bm
#endif
