// C-ABI entry points (include/brahmap.h): argument validation, handle
// lifetime, error translation.  Every entry point catches the library's
// internal bm::Error and returns its status; no exception crosses the ABI.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <tuple>

#include "bm_internal.cuh"

namespace bm {

static thread_local char g_last_error[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}
void clear_error() { g_last_error[0] = '\0'; }

thread_local cudaStream_t tl_stream = nullptr;

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static cudaEvent_t take_event(bm_context* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

ScopedTimer::ScopedTimer(bm_context* c, const char* n) : ctx(c), name(n) {
    if (ctx && ctx->timing) {
        a = take_event(ctx);
        if (a) cudaEventRecord(a, ctx->stream);
    }
}
ScopedTimer::~ScopedTimer() {
    if (ctx && ctx->timing && a) {
        cudaEvent_t b = take_event(ctx);
        if (b) {
            cudaEventRecord(b, ctx->stream);
            ctx->pending.push_back({name, a, b});
        } else {
            ctx->event_pool.push_back(a);
        }
    }
}

// Accumulate the recorded event pairs into the per-kernel timers.
void resolve_timers(bm_context* ctx) {
    for (auto& pd : ctx->pending) {
        if (cudaEventSynchronize(pd.b) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pd.a, pd.b);
            auto& t = ctx->timers[pd.name];
            t.total_ms += ms;
            t.launches += 1;
        }
        ctx->event_pool.push_back(pd.a);
        ctx->event_pool.push_back(pd.b);
    }
    ctx->pending.clear();
    (void)cudaGetLastError();
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device and never lowers it: the limit is a per-function setting of
// the device, and threads launching the same kernel with different sizes
// (several contexts, the server's slots) must not undo each other.
void ensure_smem_limit(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;
    int dev = 0;
    BM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[{dev, kernel}];
    if (bytes <= cur) return;
    BM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
}

int blocks_per_sm(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(kernel, threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

void shard_reduce(bm_context* ctx, double* buf, int64_t count) {
    if (!ctx->allreduce || count <= 0) return;
    BM_CUDA(cudaStreamSynchronize(ctx->stream));
    const bm_status st = ctx->allreduce(buf, count, ctx->allreduce_user);
    if (st != BM_OK) {
        set_error("the sharded solve's reduction of %lld values failed (%s)", (long long)count, bm_status_string(st));
        throw Error{st};
    }
    BM_CUDA(cudaSetDevice(ctx->device));  // the callback may have switched devices
}

void* workspace(bm_context* ctx, const char* name, size_t bytes) {
    auto& b = ctx->ws[name];
    if (b.n < bytes) {
        ctx->ws_generation += 1;
        try {
            b.alloc_from(ctx->ws_pool, bytes + bytes / 8);  // stream-ordered: old users finish first
        } catch (const Error& e) {
            if (e.status != BM_ERR_OOM) throw;
            // memory freed elsewhere in the process may still be held by the
            // device's default pool (or this context's own): give it back to
            // the device and try once more
            BM_CUDA(cudaDeviceSynchronize());
            cudaMemPool_t def = nullptr;
            if (cudaDeviceGetDefaultMemPool(&def, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(def, 0);
            if (ctx->ws_pool) cudaMemPoolTrimTo(ctx->ws_pool, 0);
            clear_error();
            b.alloc_from(ctx->ws_pool, bytes + bytes / 8);
        }
    }
    return b.get();
}

}  // namespace bm

using namespace bm;

template <typename F>
static bm_status guarded(F&& f) {
    clear_error();
    try {
        return f();
    } catch (const Error& e) {
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return BM_ERR_OOM;
    } catch (...) {
        set_error("unexpected internal error");
        return BM_ERR_CUDA;
    }
}

static void use_device(const bm_context* ctx) {
    BM_CUDA(cudaSetDevice(ctx->device));
    tl_stream = ctx->stream;
}

// Host -> device copy ordered on the context stream; returns once the copy is done.
static void upload(bm_context* ctx, void* dst, const void* src, size_t bytes) {
    BM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    BM_CUDA(cudaStreamSynchronize(ctx->stream));
}

extern "C" {

const char* bm_status_string(bm_status s) {
    switch (s) {
        case BM_OK: return "ok";
        case BM_ERR_INVALID: return "invalid argument";
        case BM_ERR_OOM: return "out of device memory";
        case BM_ERR_CUDA: return "CUDA error";
        case BM_ERR_NOT_CONVERGED: return "not converged";
        case BM_ERR_BREAKDOWN: return "CG breakdown";
        case BM_ERR_TIMEOUT: return "timeout";
        case BM_ERR_BUSY: return "busy";
        case BM_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

const char* bm_last_error(void) { return g_last_error; }
const char* bm_version(void) { return "brahmap-gb300 0.1 (sm_103a)"; }

bm_status bm_context_create(int device, void* cuda_stream, bm_context** out) {
    return guarded([&] {
        BM_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        int ndev = 0;
        BM_CUDA(cudaGetDeviceCount(&ndev));
        BM_REQUIRE(device >= 0 && device < ndev, "device %d out of range [0, %d)", device, ndev);
        BM_CUDA(cudaSetDevice(device));
        auto* ctx = new bm_context();
        ctx->device = device;
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
        cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 4096);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->side_ev, cudaEventDisableTiming);
        // Keep memory freed back to the device pool for reuse by the next
        // handle instead of returning it to the driver.
        cudaMemPool_t pool = nullptr;
        if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, device);
        if (e == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        if (e == cudaSuccess) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            e = cudaMemPoolCreate(&ctx->ws_pool, &props);
            uint64_t thr = UINT64_MAX;
            if (e == cudaSuccess) e = cudaMemPoolSetAttribute(ctx->ws_pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        if (e != cudaSuccess) {
            set_error("context setup failed: %s", cudaGetErrorString(e));
            bm_context_destroy(ctx);
            return BM_ERR_CUDA;
        }
        try {
            ctx->static_scratch = static_scratch_setup();
        } catch (...) {
            bm_context_destroy(ctx);
            throw;
        }
        *out = ctx;
        return BM_OK;
    });
}

bm_status bm_context_set_allreduce(bm_context* ctx, bm_allreduce_fn fn, void* user) {
    return guarded([&] {
        BM_REQUIRE(ctx, "ctx is NULL");
        ctx->allreduce = fn;
        ctx->allreduce_user = fn ? user : nullptr;
        return BM_OK;
    });
}

void bm_context_destroy(bm_context* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    tl_stream = ctx->stream;
    cudaStreamSynchronize(ctx->stream);
    resolve_timers(ctx);
    for (cudaEvent_t ev : ctx->event_pool) cudaEventDestroy(ev);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->side_ev) cudaEventDestroy(ctx->side_ev);
    const int dev = ctx->device;
    cudaMemPool_t ws_pool = ctx->ws_pool;
    delete ctx;  // releases the workspaces (stream-ordered)
    cudaStreamSynchronize(tl_stream);
    if (ws_pool) cudaMemPoolDestroy(ws_pool);
    // Hand the pool's unused memory back to the driver.
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && pool) cudaMemPoolTrimTo(pool, 0);
    (void)cudaGetLastError();
}

int64_t bm_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

bm_status bm_context_set_timing(bm_context* ctx, int enable) {
    return guarded([&] {
        BM_REQUIRE(ctx, "ctx is NULL");
        ctx->timing = enable != 0;
        return BM_OK;
    });
}

bm_status bm_context_set_graphs(bm_context* ctx, int enable) {
    return guarded([&] {
        BM_REQUIRE(ctx, "ctx is NULL");
        ctx->graphs = enable != 0;
        return BM_OK;
    });
}

bm_status bm_context_kernel_time(bm_context* ctx, const char* name, double* total_ms,
                                 int64_t* launches) {
    return guarded([&] {
        BM_REQUIRE(ctx && name, "ctx/name is NULL");
        use_device(ctx);
        resolve_timers(ctx);
        auto it = ctx->timers.find(name);
        double ms = 0.0;
        int64_t n = 0;
        if (it != ctx->timers.end()) {
            ms = it->second.total_ms;
            n = it->second.launches;
            ctx->timers.erase(it);
        }
        if (total_ms) *total_ms = ms;
        if (launches) *launches = n;
        return BM_OK;
    });
}

bm_status bm_ang2pix_ring(bm_context* ctx, int64_t nside, int64_t n, const double* z,
                          const double* phi, int32_t* pix) {
    return guarded([&] {
        BM_REQUIRE(ctx, "ctx is NULL");
        BM_REQUIRE(nside >= 1 && nside <= 8192, "nside %lld out of [1, 8192]", (long long)nside);
        BM_REQUIRE(n >= 0, "n < 0");
        if (n == 0) return BM_OK;
        BM_REQUIRE(z && phi && pix, "NULL array");
        use_device(ctx);
        ang2pix_ring(ctx, nside, n, z, phi, pix);
        BM_CUDA(cudaStreamSynchronize(ctx->stream));
        return BM_OK;
    });
}

// Address at which the device reads a caller's input array: device or
// managed memory of the context's GPU as is; page-locked host memory through
// its device mapping (the kernel that reads it then streams it over the
// host link).  Anything else is rejected.
static const void* device_readable(const bm_context* ctx, const void* ptr, const char* what,
                                   bool* on_host = nullptr) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        a.type = cudaMemoryTypeUnregistered;
    }
    if (on_host) *on_host = a.type == cudaMemoryTypeHost;
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        BM_REQUIRE(a.type == cudaMemoryTypeManaged || a.device == ctx->device,
                   "%s lives on device %d, the context on device %d", what, a.device, ctx->device);
        return ptr;
    }
    BM_REQUIRE(a.type == cudaMemoryTypeHost && a.devicePointer != nullptr,
               "%s is neither device memory nor page-locked host memory", what);
    return a.devicePointer;
}

// The three pointing constructors: angles (psi) or FP32 trig pairs, and
// optionally one FP32 TOD sorted along with the samples.
static bm_status create_pointing(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                 const void* psi, bm_dtype psi_dtype, const float* cos2psi,
                                 const float* sin2psi, const float* tod, bm_solver_type solver,
                                 bm_pointing** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        BM_REQUIRE(npix >= 1 && npix <= (int64_t(1) << 28), "npix %lld out of [1, 2^28]", (long long)npix);
        BM_REQUIRE(nsamples >= 1 && nsamples < (int64_t(1) << 32), "nsamples out of [1, 2^32)");
        BM_REQUIRE(pix, "pix is NULL");
        BM_REQUIRE((psi != nullptr) != (cos2psi != nullptr || sin2psi != nullptr),
                   "give either psi or cos2psi and sin2psi");
        BM_REQUIRE(psi || (cos2psi && sin2psi), "cos2psi/sin2psi is NULL");
        if (psi) BM_REQUIRE(psi_dtype == BM_F32 || psi_dtype == BM_F64, "bad psi dtype");
        BM_REQUIRE(solver == BM_SOLVER_I || solver == BM_SOLVER_QU || solver == BM_SOLVER_IQU,
                   "bad solver type %d", (int)solver);
        use_device(ctx);
        pix = static_cast<const int32_t*>(device_readable(ctx, pix, "pix"));
        if (psi) {
            psi = device_readable(ctx, psi, "psi");
        } else {
            cos2psi = static_cast<const float*>(device_readable(ctx, cos2psi, "cos2psi"));
            sin2psi = static_cast<const float*>(device_readable(ctx, sin2psi, "sin2psi"));
        }
        bool tod_on_host = false;
        if (tod) tod = static_cast<const float*>(device_readable(ctx, tod, "tod", &tod_on_host));
        auto* p = new bm_pointing();
        p->ctx = ctx;
        p->npix = npix;
        p->nsamples = nsamples;
        p->ncomp = (int)solver;
        try {
            ingest(p, pix, psi, psi_dtype, cos2psi, sin2psi, tod, tod_on_host);
        } catch (...) {
            delete p;
            throw;
        }
        *out = p;
        return BM_OK;
    });
}

bm_status bm_pointing_create(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                             const void* psi, bm_dtype psi_dtype, bm_solver_type solver,
                             bm_pointing** out) {
    if (!psi) return guarded([&]() -> bm_status { BM_REQUIRE(false, "psi is NULL"); return BM_OK; });
    return create_pointing(ctx, npix, nsamples, pix, psi, psi_dtype, nullptr, nullptr, nullptr, solver, out);
}

bm_status bm_pointing_create_trig(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                  const float* cos2psi, const float* sin2psi, bm_solver_type solver,
                                  bm_pointing** out) {
    if (!cos2psi || !sin2psi)
        return guarded([&]() -> bm_status { BM_REQUIRE(false, "cos2psi/sin2psi is NULL"); return BM_OK; });
    return create_pointing(ctx, npix, nsamples, pix, nullptr, BM_F32, cos2psi, sin2psi, nullptr, solver, out);
}

bm_status bm_pointing_create_with_tod(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                      const void* psi, bm_dtype psi_dtype, const float* cos2psi,
                                      const float* sin2psi, const float* tod, bm_solver_type solver,
                                      bm_pointing** out) {
    if (!tod) return guarded([&]() -> bm_status { BM_REQUIRE(false, "tod is NULL"); return BM_OK; });
    return create_pointing(ctx, npix, nsamples, pix, psi, psi_dtype, cos2psi, sin2psi, tod, solver, out);
}

static void check_det_offsets(int32_t ndet, const int64_t* det_offsets);

namespace bm {
namespace {
// tab[j] = (cos, sin)(2 pi j / kHwpTab) in FP64, and rounded to FP32.
__global__ void hwp_table_kernel(float2* __restrict__ tab, float4* __restrict__ tabdf) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < kHwpTab; j += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)j / (double)kHwpTab, &sn, &cs);
        const float ch = (float)cs, sh = (float)sn;
        tab[j] = make_float2(ch, sh);
        tabdf[j] = make_float4(ch, sh, (float)(cs - (double)ch), (float)(sn - (double)sh));
    }
}

// A fraction of a turn in [0, 1) as a 64-bit fixed-point number (exact: x
// times a power of two, truncated only below 2^-64).
unsigned long long turn_fixed(double x) {
    x -= std::floor(x);
    const double v = std::ldexp(x, 64);
    return v >= 18446744073709551616.0 ? 0ull : (unsigned long long)v;
}
}  // namespace
}  // namespace bm

bm_status bm_pointing_create_hwp(bm_context* ctx, int64_t npix, int64_t nsamples, const int32_t* pix,
                                 int32_t ndet, const int64_t* det_offsets, const double* psi_det,
                                 double hwp_turns_per_sample, double hwp_phase0, bm_solver_type solver,
                                 bm_pointing** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        BM_REQUIRE(npix >= 1 && npix <= (int64_t(1) << 28), "npix %lld out of [1, 2^28]", (long long)npix);
        BM_REQUIRE(nsamples >= 1 && nsamples < (int64_t(1) << 32), "nsamples out of [1, 2^32)");
        BM_REQUIRE(pix && psi_det, "pix/psi_det is NULL");
        BM_REQUIRE(solver == BM_SOLVER_I || solver == BM_SOLVER_QU || solver == BM_SOLVER_IQU,
                   "bad solver type %d", (int)solver);
        check_det_offsets(ndet, det_offsets);
        BM_REQUIRE(det_offsets[ndet] == nsamples, "det_offsets[ndet] = %lld != nsamples %lld",
                   (long long)det_offsets[ndet], (long long)nsamples);
        BM_REQUIRE(std::isfinite(hwp_turns_per_sample) && std::isfinite(hwp_phase0),
                   "non-finite half-wave-plate rate or phase");
        for (int d = 0; d < ndet; ++d) BM_REQUIRE(std::isfinite(psi_det[d]), "psi_det[%d] is not finite", d);
        use_device(ctx);
        pix = static_cast<const int32_t*>(device_readable(ctx, pix, "pix"));
        auto* p = new bm_pointing();
        p->ctx = ctx;
        p->npix = npix;
        p->nsamples = nsamples;
        p->ncomp = (int)solver;
        try {
            // the model: 2 theta = 2 psi_d + 4 phi0 + 4 (2 pi nu k), in turns
            const double two_pi = 6.283185307179586476925287;
            std::vector<uint32_t> off(ndet + 1);
            std::vector<unsigned long long> turn0(ndet);
            bool uniform = true;
            for (int d = 0; d <= ndet; ++d) off[d] = (uint32_t)det_offsets[d];
            for (int d = 0; d < ndet; ++d) {
                turn0[d] = turn_fixed((2.0 * psi_det[d] + 4.0 * hwp_phase0) / two_pi);
                uniform = uniform && (det_offsets[d + 1] - det_offsets[d] == det_offsets[1]);
            }
            p->hwp = true;
            p->hwp_off.alloc(ndet + 1);
            p->hwp_turn0.alloc(ndet);
            p->hwp_tab.alloc(kHwpTab);
            p->hwp_tab_df.alloc(kHwpTab);
            BM_CUDA(cudaMemcpyAsync(p->hwp_off.get(), off.data(), sizeof(uint32_t) * (ndet + 1),
                                    cudaMemcpyHostToDevice, ctx->stream));
            BM_CUDA(cudaMemcpyAsync(p->hwp_turn0.get(), turn0.data(), sizeof(unsigned long long) * ndet,
                                    cudaMemcpyHostToDevice, ctx->stream));
            hwp_table_kernel<<<(kHwpTab + 255) / 256, 256, 0, ctx->stream>>>(p->hwp_tab.get(), p->hwp_tab_df.get());
            BM_LAUNCH_CHECK();
            HwpModel& m = p->hwp_model;
            m.off = p->hwp_off.get();
            m.turn0 = p->hwp_turn0.get();
            m.tabdf = p->hwp_tab_df.get();
            m.nu = turn_fixed(hwp_turns_per_sample);
            m.ndet = ndet;
            // t / ns for uniform detectors (as the noise handles do; fewer than 2^20 detectors)
            m.ns = uniform ? (uint32_t)det_offsets[1] : 0u;
            m.inv_ns = uniform ? (float)(1.0 / (double)det_offsets[1]) : 0.f;
            ingest(p, pix, nullptr, BM_F64, nullptr, nullptr, nullptr, false, &m);
            BM_CUDA(cudaStreamSynchronize(ctx->stream));  // the host tables above are released on return
        } catch (...) {
            delete p;
            throw;
        }
        *out = p;
        return BM_OK;
    });
}

void bm_pointing_destroy(bm_pointing* p) {
    if (!p) return;
    cudaSetDevice(p->ctx->device);
    cudaStreamSynchronize(p->ctx->stream);
    delete p;
}

bm_status bm_pointing_get_hits(const bm_pointing* p, int32_t* hits) {
    return guarded([&] {
        BM_REQUIRE(p && hits, "NULL argument");
        use_device(p->ctx);
        BM_CUDA(cudaMemcpyAsync(hits, p->hits.get(), sizeof(int32_t) * p->npix,
                                cudaMemcpyDeviceToDevice, p->ctx->stream));
        BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_pointing_get_order(const bm_pointing* p, uint32_t* order, int64_t* nvalid) {
    return guarded([&] {
        BM_REQUIRE(p, "NULL argument");
        if (nvalid) *nvalid = p->nvalid;
        if (order && p->nvalid > 0) {
            use_device(p->ctx);
            BM_CUDA(cudaMemcpyAsync(order, p->perm.get(), sizeof(uint32_t) * p->nvalid, cudaMemcpyDeviceToDevice,
                                    p->ctx->stream));
            BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        }
        return BM_OK;
    });
}

bm_status bm_pointing_apply(bm_pointing* p, const double* x, double* y) {
    return guarded([&] {
        BM_REQUIRE(p && x && y, "NULL argument");
        use_device(p->ctx);
        pointing_apply(p, x, y);
        BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_pointing_apply_transpose(bm_pointing* p, const double* y, double* x) {
    return guarded([&] {
        BM_REQUIRE(p && x && y, "NULL argument");
        use_device(p->ctx);
        pointing_apply_transpose(p, y, x);
        BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        return BM_OK;
    });
}

static void check_det_offsets(int32_t ndet, const int64_t* det_offsets) {
    BM_REQUIRE(ndet >= 1 && ndet <= (1 << 20), "ndet %d out of [1, 2^20]", ndet);
    BM_REQUIRE(det_offsets != nullptr, "det_offsets is NULL");
    BM_REQUIRE(det_offsets[0] == 0, "det_offsets[0] must be 0");
    for (int d = 0; d < ndet; ++d)
        BM_REQUIRE(det_offsets[d + 1] > det_offsets[d], "det_offsets not increasing at %d", d);
    BM_REQUIRE(det_offsets[ndet] < (int64_t(1) << 32), "more than 2^32 - 1 samples");
}

static bm_inv_noise* new_noise(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                               const double* white) {
    auto* n = new bm_inv_noise();
    n->ctx = ctx;
    n->ndet = ndet;
    n->nsamples = det_offsets[ndet];
    n->h_det_off.assign(det_offsets, det_offsets + ndet + 1);
    n->h_white.assign(white, white + ndet);
    try {
        n->det_off.alloc(ndet + 1);
        n->white.alloc(ndet);
        upload(ctx, n->det_off.get(), det_offsets, sizeof(int64_t) * (ndet + 1));
        upload(ctx, n->white.get(), white, sizeof(double) * ndet);
        std::vector<uint32_t> off32(det_offsets, det_offsets + ndet + 1);
        std::vector<float2> wdf(ndet);
        std::vector<float> wsq(ndet);
        for (int d = 0; d < ndet; ++d) {
            const float h = (float)white[d];
            wdf[d] = make_float2(h, (float)(white[d] - (double)h));
            wsq[d] = (float)std::sqrt(white[d]);
        }
        const int64_t len0 = det_offsets[1] - det_offsets[0];
        bool uniform = det_offsets[0] == 0 && len0 >= 1 && ndet < (1 << 20);
        for (int d = 1; d < ndet && uniform; ++d) uniform = det_offsets[d + 1] - det_offsets[d] == len0;
        n->ns_uniform = uniform ? (uint32_t)len0 : 0u;
        n->inv_ns = uniform ? (float)(1.0 / (double)len0) : 0.f;
        n->det_off32.alloc(ndet + 1);
        n->wdf.alloc(ndet);
        n->wsqrt.alloc(ndet);
        upload(ctx, n->det_off32.get(), off32.data(), sizeof(uint32_t) * (ndet + 1));
        upload(ctx, n->wdf.get(), wdf.data(), sizeof(float2) * ndet);
        upload(ctx, n->wsqrt.get(), wsq.data(), sizeof(float) * ndet);
    } catch (...) {
        delete n;
        throw;
    }
    return n;
}

bm_status bm_inv_noise_create_diag(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                   const double* inv_var, bm_inv_noise** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        check_det_offsets(ndet, det_offsets);
        BM_REQUIRE(inv_var != nullptr, "inv_var is NULL");
        for (int d = 0; d < ndet; ++d)
            BM_REQUIRE(inv_var[d] > 0 && inv_var[d] < 1e300, "inv_var[%d] not positive finite", d);
        use_device(ctx);
        *out = new_noise(ctx, ndet, det_offsets, inv_var);
        (*out)->kind = 0;
        return BM_OK;
    });
}

// Copies the per-sample weights and counts those that are negative or not
// finite.
__global__ void copy_check_weights_kernel(const double* __restrict__ w, int64_t n, double* __restrict__ out,
                                          unsigned long long* __restrict__ nbad) {
    unsigned bad = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[t];
        bad += !(x >= 0.0 && x < 1e300);  // false for NaN
        out[t] = x;
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(nbad, (unsigned long long)bad);
}

bm_status bm_inv_noise_create_sample_weights(bm_context* ctx, int64_t nsamples, const double* weights,
                                             bm_inv_noise** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        BM_REQUIRE(nsamples >= 1 && nsamples < (int64_t(1) << 32), "nsamples out of [1, 2^32)");
        BM_REQUIRE(weights != nullptr, "weights is NULL");
        use_device(ctx);
        weights = static_cast<const double*>(device_readable(ctx, weights, "weights"));
        // one pseudo-detector of unit weight keeps the per-detector tables valid
        const int64_t off[2] = {0, nsamples};
        const double one = 1.0;
        bm_inv_noise* n = new_noise(ctx, 1, off, &one);
        try {
            n->kind = 2;
            n->wsamp.alloc(nsamples);
            DevBuf<unsigned long long> nbad(1);
            BM_CUDA(cudaMemsetAsync(nbad.get(), 0, sizeof(unsigned long long), ctx->stream));
            copy_check_weights_kernel<<<grid_for(ctx, (nsamples + 255) / 256, 16), 256, 0, ctx->stream>>>(
                weights, nsamples, n->wsamp.get(), nbad.get());
            BM_LAUNCH_CHECK();
            unsigned long long h_bad = 0;
            BM_CUDA(cudaMemcpyAsync(&h_bad, nbad.get(), sizeof(h_bad), cudaMemcpyDeviceToHost, ctx->stream));
            BM_CUDA(cudaStreamSynchronize(ctx->stream));
            BM_REQUIRE(h_bad == 0, "%llu weights are negative or not finite", h_bad);
        } catch (...) {
            delete n;
            throw;
        }
        *out = n;
        return BM_OK;
    });
}

bm_status bm_inv_noise_create_offset_filter(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                            const double* inv_var, int64_t baseline_len, bm_inv_noise** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        check_det_offsets(ndet, det_offsets);
        BM_REQUIRE(inv_var != nullptr, "inv_var is NULL");
        BM_REQUIRE(baseline_len >= 1, "baseline_len < 1");
        for (int d = 0; d < ndet; ++d)
            BM_REQUIRE(inv_var[d] > 0 && inv_var[d] < 1e300, "inv_var[%d] not positive finite", d);
        // no detector is longer than nsamples: a longer baseline is the same filter
        const int64_t bl = std::min<int64_t>(baseline_len, det_offsets[ndet]);
        std::vector<int64_t> start(ndet + 1, 0);
        for (int d = 0; d < ndet; ++d) {
            const int64_t len = det_offsets[d + 1] - det_offsets[d];
            start[d + 1] = start[d] + len / bl + (len % bl != 0);
        }
        use_device(ctx);
        bm_inv_noise* n = new_noise(ctx, ndet, det_offsets, inv_var);
        try {
            n->kind = 3;
            n->baseline_len = bl;
            n->nint = start[ndet];
            n->int_start.alloc(ndet + 1);
            upload(ctx, n->int_start.get(), start.data(), sizeof(int64_t) * (ndet + 1));
        } catch (...) {
            delete n;
            throw;
        }
        *out = n;
        return BM_OK;
    });
}

bm_status bm_inv_noise_create_toeplitz(bm_context* ctx, int32_t ndet, const int64_t* det_offsets,
                                       int64_t chunk_len, int32_t nlags, const double* coeffs,
                                       const double* white_inv_var, bm_inv_noise** out) {
    return guarded([&] {
        BM_REQUIRE(ctx && out, "ctx/out is NULL");
        *out = nullptr;
        check_det_offsets(ndet, det_offsets);
        BM_REQUIRE(chunk_len >= 1, "chunk_len < 1");
        BM_REQUIRE(nlags >= 1 && nlags <= 1024, "nlags %d out of [1, 1024]", nlags);
        BM_REQUIRE(coeffs && white_inv_var, "coeffs/white_inv_var is NULL");
        for (int d = 0; d < ndet; ++d)
            BM_REQUIRE(white_inv_var[d] > 0 && white_inv_var[d] < 1e300,
                       "white_inv_var[%d] not positive finite", d);
        for (int64_t i = 0; i < (int64_t)ndet * nlags; ++i)
            BM_REQUIRE(coeffs[i] == coeffs[i] && coeffs[i] < 1e300 && coeffs[i] > -1e300,
                       "coeffs[%lld] not finite", (long long)i);
        use_device(ctx);
        bm_inv_noise* n = new_noise(ctx, ndet, det_offsets, white_inv_var);
        n->kind = 1;
        n->chunk_len = chunk_len;
        n->nlags = nlags;
        try {
            const size_t m = (size_t)ndet * nlags;
            std::vector<float> c32(coeffs, coeffs + m);
            n->coeffs64.alloc(m);
            n->coeffs32.alloc(m);
            upload(ctx, n->coeffs64.get(), coeffs, sizeof(double) * m);
            upload(ctx, n->coeffs32.get(), c32.data(), sizeof(float) * m);
            prepare_toeplitz_fft(n);
        } catch (...) {
            delete n;
            throw;
        }
        *out = n;
        return BM_OK;
    });
}

void bm_inv_noise_destroy(bm_inv_noise* n) {
    if (!n) return;
    cudaSetDevice(n->ctx->device);
    cudaStreamSynchronize(n->ctx->stream);
    delete n;
}

bm_status bm_inv_noise_apply(bm_inv_noise* n, const double* y, double* z) {
    return guarded([&] {
        BM_REQUIRE(n && y && z, "NULL argument");
        use_device(n->ctx);
        inv_noise_apply(n, y, z);
        BM_CUDA(cudaStreamSynchronize(n->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_blockdiag_precond_create(bm_pointing* p, bm_inv_noise* n, int32_t min_hits,
                                      double max_cond, bm_precond** out) {
    return guarded([&] {
        BM_REQUIRE(p && n && out, "NULL argument");
        *out = nullptr;
        BM_REQUIRE(p->ctx == n->ctx, "pointing and noise belong to different contexts");
        BM_REQUIRE(n->nsamples == p->nsamples, "noise covers %lld samples, pointing %lld",
                   (long long)n->nsamples, (long long)p->nsamples);
        BM_REQUIRE(min_hits >= 0, "min_hits < 0");
        BM_REQUIRE(max_cond >= 1.0, "max_cond < 1");
        use_device(p->ctx);
        auto* pc = new bm_precond();
        pc->ctx = p->ctx;
        pc->p = p;
        pc->n = n;
        pc->ncomp = p->ncomp;
        pc->nsym = p->ncomp * (p->ncomp + 1) / 2;
        pc->min_hits = min_hits;
        pc->max_cond = max_cond;
        try {
            build_precond(pc);
        } catch (...) {
            delete pc;
            throw;
        }
        *out = pc;
        return BM_OK;
    });
}

void bm_precond_destroy(bm_precond* pc) {
    if (!pc) return;
    cudaSetDevice(pc->ctx->device);
    cudaStreamSynchronize(pc->ctx->stream);
    delete pc;
}

bm_status bm_precond_get_mask(const bm_precond* pc, uint8_t* mask, int32_t* hits) {
    return guarded([&] {
        BM_REQUIRE(pc, "pc is NULL");
        use_device(pc->ctx);
        const int64_t npix = pc->p->npix;
        if (mask)
            BM_CUDA(cudaMemcpyAsync(mask, pc->mask.get(), npix, cudaMemcpyDeviceToDevice, pc->ctx->stream));
        if (hits)  // a shard's preconditioner keeps the hit counts of all ranks
            BM_CUDA(cudaMemcpyAsync(hits, pc->hits_global.get() ? pc->hits_global.get() : pc->p->hits.get(),
                                    sizeof(int32_t) * npix, cudaMemcpyDeviceToDevice, pc->ctx->stream));
        BM_CUDA(cudaStreamSynchronize(pc->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_precond_get_blocks(const bm_precond* pc, double* blocks, double* cond) {
    return guarded([&] {
        BM_REQUIRE(pc, "pc is NULL");
        use_device(pc->ctx);
        const int64_t npix = pc->p->npix;
        if (blocks)
            BM_CUDA(cudaMemcpyAsync(blocks, pc->B.get(), sizeof(double) * npix * pc->ncomp * pc->ncomp,
                                    cudaMemcpyDeviceToDevice, pc->ctx->stream));
        if (cond)
            BM_CUDA(cudaMemcpyAsync(cond, pc->cond.get(), sizeof(double) * npix,
                                    cudaMemcpyDeviceToDevice, pc->ctx->stream));
        BM_CUDA(cudaStreamSynchronize(pc->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_precond_apply(bm_precond* pc, const double* r, double* z) {
    return guarded([&] {
        BM_REQUIRE(pc && r && z, "NULL argument");
        use_device(pc->ctx);
        precond_apply(pc, r, z, 1);
        BM_CUDA(cudaStreamSynchronize(pc->ctx->stream));
        return BM_OK;
    });
}

static void check_system(bm_pointing* p, bm_inv_noise* n, bm_precond* pc) {
    BM_REQUIRE(p && n && pc, "NULL handle");
    BM_REQUIRE(pc->p == p && pc->n->nsamples == n->nsamples && p->ctx == n->ctx,
               "preconditioner was built for another pointing / sample layout");
    BM_REQUIRE(n->nsamples == p->nsamples, "noise and pointing cover different sample counts");
    if (diagonal_noise(n))
        BM_REQUIRE(pc->n == n, "a diagonal-noise system needs the preconditioner built from that noise");
    if (n->kind == 3)
        BM_REQUIRE(pc->n == n, "an offset-filter system needs the preconditioner built from that noise "
                               "(its kept samples per interval)");
}

// tod = NULL selects the TOD the pointing was created with (one RHS, white
// noise: a Toeplitz filter runs in time order).
static void check_carried_tod(const bm_pointing* p, const bm_inv_noise* n, int32_t nrhs) {
    BM_REQUIRE(p->tod_s.get() != nullptr, "tod is NULL and the pointing was not created with a TOD");
    BM_REQUIRE(nrhs == 1, "the TOD carried by the pointing is one right-hand side (nrhs = %d)", nrhs);
    BM_REQUIRE(diagonal_noise(n), "the TOD carried by the pointing is pixel-sorted; a time-ordered N^-1 "
                                  "(Toeplitz, offset filter) needs the time-ordered TOD");
}

bm_status bm_rhs(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod,
                 bm_dtype tod_dtype, int32_t nrhs, double* b) {
    return guarded([&] {
        check_system(p, n, pc);
        BM_REQUIRE(b, "NULL array");
        if (!tod) check_carried_tod(p, n, nrhs);
        BM_REQUIRE(tod_dtype == BM_F32 || tod_dtype == BM_F64, "bad tod dtype");
        BM_REQUIRE(nrhs >= 1 && nrhs <= 4096, "nrhs out of [1, 4096]");
        use_device(p->ctx);
        rhs(p, n, pc, tod, tod_dtype, nrhs, b);
        BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_matvec(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q,
                    bm_precision prec) {
    return guarded([&] {
        check_system(p, n, pc);
        BM_REQUIRE(x && q, "NULL array");
        BM_REQUIRE(prec == BM_PREC_FP64 || prec == BM_PREC_MIXED, "bad precision");
        use_device(p->ctx);
        matvec(p, n, pc, x, q, prec, 1);
        BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
        return BM_OK;
    });
}

bm_status bm_pcg_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod,
                       bm_dtype tod_dtype, int32_t nrhs, double* map_out, double tol,
                       int32_t maxiter, bm_precision prec, bm_solve_info* info) {
    return guarded([&] {
        check_system(p, n, pc);
        BM_REQUIRE(map_out, "NULL array");
        if (!tod) check_carried_tod(p, n, nrhs);
        BM_REQUIRE(tod_dtype == BM_F32 || tod_dtype == BM_F64, "bad tod dtype");
        BM_REQUIRE(nrhs >= 1 && nrhs <= 4096, "nrhs out of [1, 4096]");
        BM_REQUIRE(tol > 0 && tol < 1, "tol out of (0, 1)");
        BM_REQUIRE(maxiter >= 1, "maxiter < 1");
        BM_REQUIRE(prec == BM_PREC_FP64 || prec == BM_PREC_MIXED, "bad precision");
        use_device(p->ctx);
        // A page-locked host TOD is uploaded first: the solve reads it in
        // pixel order, a random access pattern the host link serves poorly.
        bool on_host = false;
        if (tod) tod = device_readable(p->ctx, tod, "tod", &on_host);
        if (on_host) {
            const size_t bytes = (size_t)nrhs * (size_t)p->nsamples * (tod_dtype == BM_F64 ? 8 : 4);
            void* dev = workspace(p->ctx, "tod_upload", bytes);
            BM_CUDA(cudaMemcpyAsync(dev, tod, bytes, cudaMemcpyHostToDevice, p->ctx->stream));
            tod = dev;
        }
        return pcg_solve(p, n, pc, tod, tod_dtype, nrhs, map_out, tol, maxiter, prec, info);
    });
}

}  // extern "C"
