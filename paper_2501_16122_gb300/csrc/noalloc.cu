// bm_matvec_white_static: the white-noise matvec with FP32 per-sample
// products (the operator the inner solve of the mixed path uses), for callers
// that cannot allocate device memory while they run -- for example a process
// that has handed all free device memory to another allocator (a framework's
// caching pool or a real-time pipeline that reserves its budget up front),
// or a host thread that must not call into the driver's allocator.  It reads
// the same pixel-sorted weighted stream as bm_matvec(..., BM_PREC_MIXED) and
// gives the same result, but it keeps its per-item partial sums in a
// fixed-size array that is part of the library image instead of a buffer
// allocated per call, and it converts x to FP32 inside the kernel instead of
// in a scratch copy.  It calls no cudaMalloc / cudaFree and no allocating
// routine of any library.
//
// The array (kStaticScratchDoubles FP64 values, 16 MiB) exists once per GPU
// on which the library is loaded and stays allocated until the process
// exits.  All calls on a device share it and it keeps the previous call's
// contents; every partial a call reads is written by that call first, so no
// clearing is needed.  Calls whose kernels overlap on the GPU (different
// streams or host threads at the same time) race on the array: serialise
// them.  The host code of this file finds the array's device address once
// per device with cudaGetSymbolAddress (with that device current) on the
// first call made on that device; make that first call before any stream
// capture begins.
#include <mutex>

#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr size_t kStaticScratchDoubles = size_t(1) << 21;  // 16 MiB of FP64
constexpr int kMaxDevices = 64;
constexpr int kWarps = 8;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the static array on `device` (which must be current).
double* static_scratch(int device) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    BM_REQUIRE(device >= 0 && device < kMaxDevices, "device %d out of range for the static scratch", device);
    if (g_scratch_addr[device] == nullptr) {
        void* ptr = nullptr;
        BM_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
        g_scratch_addr[device] = static_cast<double*>(ptr);
    }
    return g_scratch_addr[device];
}

// Same arithmetic as the white-noise FP32 matvec: u = sqrt(w) (cos, sin) per
// sorted sample, y = u . x_p with |u| on the I column, FP32 lane sums, FP64
// warp sums; x is read in FP64 and rounded to FP32 here.
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
white_matvec_static_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                           const int32_t* __restrict__ item_len, int64_t nitems,
                           const float2* __restrict__ wcs, const float* __restrict__ w1,
                           const double* __restrict__ x, double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        if (NC == 1) {
            const float xi = (float)x[p];
            float acc = 0.f;
            int i = lane;
            for (; i + 96 < len; i += 128) {
                const float a0 = __ldg(w1 + b + i), a1 = __ldg(w1 + b + i + 32);
                const float a2 = __ldg(w1 + b + i + 64), a3 = __ldg(w1 + b + i + 96);
                acc += (a0 + a1) + (a2 + a3);
            }
            for (; i < len; i += 32) acc += __ldg(w1 + b + i);
            const double s = warp_sum((double)acc) * (double)xi;
            if (lane == 0) partial[k] = s;
        } else {
            float xI = 0.f, xQ, xU;
            if (NC == 3) { xI = (float)x[3 * p]; xQ = (float)x[3 * p + 1]; xU = (float)x[3 * p + 2]; }
            else { xQ = (float)x[2 * p]; xU = (float)x[2 * p + 1]; }
            float aI = 0.f, aQ = 0.f, aU = 0.f;
            const float2* src = wcs + b;
            auto step = [&](float2 u) {
                const float r = NC == 3 ? sqrtf(fmaf(u.x, u.x, u.y * u.y)) : 0.f;
                const float y = fmaf(u.x, xQ, fmaf(u.y, xU, r * xI));
                if (NC == 3) aI = fmaf(y, r, aI);
                aQ = fmaf(y, u.x, aQ);
                aU = fmaf(y, u.y, aU);
            };
            int i = lane;
            for (; i + 96 < len; i += 128) {
                const float2 u0 = __ldg(src + i), u1 = __ldg(src + i + 32);
                const float2 u2 = __ldg(src + i + 64), u3 = __ldg(src + i + 96);
                step(u0); step(u1); step(u2); step(u3);
            }
            for (; i < len; i += 32) step(__ldg(src + i));
            const double sQ = warp_sum((double)aQ), sU = warp_sum((double)aU);
            const double sI = NC == 3 ? warp_sum((double)aI) : 0.0;
            if (lane == 0) {
                if (NC == 3) { partial[3 * k] = sI; partial[3 * k + 1] = sQ; partial[3 * k + 2] = sU; }
                else { partial[2 * k] = sQ; partial[2 * k + 1] = sU; }
            }
        }
    }
}

// q_p = sum of pixel p's item partials in item order (0 on masked pixels).
__global__ void finalize_static_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ partial,
                                       int64_t npix, int nc, double* __restrict__ q) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = pitem[p], k1 = pitem[p + 1];
        for (int c = 0; c < nc; ++c) {
            double s = 0.0;
            for (int64_t k = k0; k < k1; ++k) s += partial[k * nc + c];
            q[p * nc + c] = s;
        }
    }
}

void matvec_white_static(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q) {
    bm_context* ctx = p->ctx;
    BM_CUDA(cudaSetDevice(ctx->device));
    const int nc = p->ncomp;
    BM_REQUIRE(n->kind == 0, "bm_matvec_white_static needs diagonal (white) noise");
    BM_REQUIRE(pc->p == p && pc->n == n, "the preconditioner was built from another pointing or noise");
    BM_REQUIRE((size_t)pc->nitems * (size_t)nc <= kStaticScratchDoubles,
               "problem too large for the static scratch: %lld work items x %d components > %zu values "
               "(use bm_matvec)", (long long)pc->nitems, nc, kStaticScratchDoubles);
    double* partial = static_scratch(ctx->device);
    cudaStream_t s = ctx->stream;
    if (pc->nitems > 0) {
        const int grid = grid_for(ctx, (pc->nitems + kWarps - 1) / kWarps, 8);
#define BM_WS(NC)                                                                                       \
    white_matvec_static_kernel<NC><<<grid, kWarps * 32, 0, s>>>(pc->item_pix.get(), pc->item_beg.get(), \
                                                                pc->item_len.get(), pc->nitems, pc->wcs.get(), \
                                                                pc->w1.get(), x, partial)
        if (nc == 3) BM_WS(3); else if (nc == 2) BM_WS(2); else BM_WS(1);
#undef BM_WS
        BM_LAUNCH_CHECK();
    }
    const int threads = 256;
    finalize_static_kernel<<<grid_for(ctx, (p->npix + threads - 1) / threads, 16), threads, 0, s>>>(
        pc->pitem.get(), partial, p->npix, nc, q);
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

}  // namespace bm

extern "C" bm_status bm_matvec_white_static(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x,
                                            double* q) {
    bm::clear_error();
    try {
        BM_REQUIRE(p && n && pc && x && q, "NULL argument");
        bm::matvec_white_static(p, n, pc, x, q);
        return BM_OK;
    } catch (const bm::Error& e) {
        return e.status;
    } catch (...) {
        bm::set_error("unexpected internal error");
        return BM_ERR_CUDA;
    }
}
