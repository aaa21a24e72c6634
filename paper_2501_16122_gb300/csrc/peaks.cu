// Measured arithmetic peaks of the device: the FP32 and FP64 fused
// multiply-add rates, the denominators of the rooflines of the kernels that
// are bound by arithmetic (the FFT form of the Toeplitz N^-1, the
// double-float refinement operator, the FP64 matvec).  No counterpart in the
// paper; a measurement helper next to the hot path.
//
// Each thread runs kChains independent FMA chains (enough independent work
// to hide the pipe latency), so the loop issues nothing but FMAs apart from
// its counter; the grid fills every SM with resident blocks.  The result is
// stored conditionally so the compiler cannot drop the chains.
#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;

__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int iters, T a, T b, T* __restrict__ sink) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma_rn(v[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == (T)-1.2345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true for these inputs
}

template <typename T>
double measure(bm_context* ctx, int iters) {
    const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(fma_chain_kernel<T>), kPeakThreads, 0);
    const int grid = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
    T* sink = workspace_as<T>(ctx, "peak_sink", (size_t)grid * kPeakThreads);
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0, e1;
    BM_CUDA(cudaEventCreate(&e0));
    BM_CUDA(cudaEventCreate(&e1));
    double best_ms = 1e30;
    // a multiplier below 1 and an addend keep the values finite and normal
    const T a = (T)0.999999, b = (T)1e-3;
    for (int rep = 0; rep < 4; ++rep) {  // the first is a warm-up
        cudaEventRecord(e0, s);
        fma_chain_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters, a, b, sink);
        cudaEventRecord(e1, s);
        const cudaError_t le = cudaGetLastError();
        count_launch();
        if (le != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            BM_CUDA(le);
        }
        BM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best_ms) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)grid * kPeakThreads * kChains * (double)iters;
    return 2.0 * fmas / (best_ms * 1e-3);
}

}  // namespace

}  // namespace bm

extern "C" bm_status bm_measure_fma_peak(bm_context* ctx, bm_dtype dtype, double* flops_per_s) {
    bm::clear_error();
    try {
        BM_REQUIRE(ctx && flops_per_s, "NULL argument");
        BM_REQUIRE(dtype == BM_F32 || dtype == BM_F64, "bad dtype");
        BM_CUDA(cudaSetDevice(ctx->device));
        bm::tl_stream = ctx->stream;
        // ~5e6 FMAs per iteration on a full GB300 (1216 blocks x 256 threads
        // x 16 chains): FP32 32768 iterations ~4 ms at ~80 TFLOP/s nominal,
        // FP64 1024 iterations ~8 ms at ~1.25 TFLOP/s nominal.
        *flops_per_s = dtype == BM_F32 ? bm::measure<float>(ctx, 32768) : bm::measure<double>(ctx, 1024);
        return BM_OK;
    } catch (const bm::Error& e) {
        return e.status;
    } catch (...) {
        bm::set_error("unexpected internal error");
        return BM_ERR_CUDA;
    }
}
