// bm_matvec_white_static: the white-noise matvec with FP32 per-sample
// products (the operator the inner solve of the mixed path uses), for callers
// that cannot allocate device memory while they run -- for example a process
// that has handed all free device memory to another allocator (a framework's
// caching pool or a real-time pipeline that reserves its budget up front),
// or a host thread that must not call into the driver's allocator.  It runs
// the very kernels of bm_matvec(..., BM_PREC_MIXED) (white_matvec.cuh), so
// its result has the same bits, but it keeps the per-item partial sums in a
// fixed-size array that is part of the library image instead of a context
// workspace, and it reads x in FP64 and rounds it to FP32 in registers
// instead of in a scratch copy.  It calls no cudaMalloc / cudaFree and no
// allocating routine of any library.
//
// The array (kStaticScratchDoubles FP64 values, 16 MiB) exists once per GPU
// on which the library is loaded and stays allocated until the process
// exits.  bm_context_create loads it: it looks the array's device address up
// with cudaGetSymbolAddress, with the context's device current (which loads
// this file's module and its array under lazy module loading), and queries
// the kernels' attributes (which loads their code).  So a call of
// bm_matvec_white_static maps no memory, not even the first one on a device.
// All calls on a device share the array and it keeps the previous call's
// contents; every partial a call reads is written by that call first, so no
// clearing is needed.  Calls whose kernels overlap on the GPU (different
// streams or host threads at the same time) race on the array: serialise
// them.
#include "bm_internal.cuh"
#include "white_matvec.cuh"

namespace bm {

namespace {

constexpr size_t kStaticScratchDoubles = size_t(1) << 21;  // 16 MiB of FP64

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

template <int NC>
void launch_white(bm_context* ctx, bm_precond* pc, const double* x, double* partial) {
    const int64_t wunits = (pc->nitems + kWhiteWarps - 1) / kWhiteWarps;
    white_matvec_f32_kernel<NC, double>
        <<<resident_grid(ctx, white_matvec_f32_kernel<NC, double>, kWhiteWarps * 32, wunits), kWhiteWarps * 32, 0,
           ctx->stream>>>(pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems, pc->wcs.get(),
                          pc->w1.get(), x, partial);
    BM_LAUNCH_CHECK();
}

}  // namespace

// Device address of the static array on the current device, with the code
// of the kernels that use it loaded.  Called once per context.
double* static_scratch_setup() {
    void* ptr = nullptr;
    BM_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
    cudaFuncAttributes a;
    BM_CUDA(cudaFuncGetAttributes(&a, white_matvec_f32_kernel<1, double>));
    BM_CUDA(cudaFuncGetAttributes(&a, white_matvec_f32_kernel<2, double>));
    BM_CUDA(cudaFuncGetAttributes(&a, white_matvec_f32_kernel<3, double>));
    BM_CUDA(cudaFuncGetAttributes(&a, finalize_pixels_kernel));
    for (const void* k : {reinterpret_cast<const void*>(white_matvec_f32_kernel<1, double>),
                          reinterpret_cast<const void*>(white_matvec_f32_kernel<2, double>),
                          reinterpret_cast<const void*>(white_matvec_f32_kernel<3, double>)})
        (void)blocks_per_sm(k, kWhiteWarps * 32, 0);
    return static_cast<double*>(ptr);
}

void matvec_white_static(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q) {
    bm_context* ctx = p->ctx;
    BM_CUDA(cudaSetDevice(ctx->device));
    const int nc = p->ncomp;
    BM_REQUIRE(diagonal_noise(n), "bm_matvec_white_static needs a diagonal N^-1 (a weight per detector or per sample)");
    BM_REQUIRE(pc->p == p && pc->n == n, "the preconditioner was built from another pointing or noise");
    BM_REQUIRE((size_t)pc->nitems * (size_t)nc <= kStaticScratchDoubles,
               "problem too large for the static scratch: %lld work items x %d components > %zu values "
               "(use bm_matvec)", (long long)pc->nitems, nc, kStaticScratchDoubles);
    BM_REQUIRE(ctx->static_scratch != nullptr, "the context has no static scratch address");
    BM_REQUIRE(pc->nitems == 0 || (nc == 1 ? pc->w1.get() != nullptr : pc->wcs.get() != nullptr),
               "the preconditioner keeps no weighted sample stream (a half-wave-plate pointing): use bm_matvec");
    double* partial = ctx->static_scratch;
    if (pc->nitems > 0) {
        if (nc == 3) launch_white<3>(ctx, pc, x, partial);
        else if (nc == 2) launch_white<2>(ctx, pc, x, partial);
        else launch_white<1>(ctx, pc, x, partial);
    }
    const int threads = 256;
    finalize_pixels_kernel<<<grid_for(ctx, (p->npix + threads - 1) / threads, 16), threads, 0, ctx->stream>>>(
        pc->pitem.get(), partial, p->npix, nc, q);
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaStreamSynchronize(ctx->stream));
}

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
