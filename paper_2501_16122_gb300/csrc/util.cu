// Device-wide exclusive scans used by the ingest (radix-sort offsets, CSR
// offsets from hit counts) and by the work-item planner.  Three phases with a fixed decomposition, so the
// result never depends on scheduling.
#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048
constexpr int kScanTilesPerBlock = 16;
constexpr int64_t kScanChunk = (int64_t)kScanTile * kScanTilesPerBlock;  // per block

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
        T s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = s - t;  // exclusive
        if (lane == (kScanThreads / 32) - 1) *total = s;
    }
    __syncthreads();
    T r = x - v + warp_tot[w];
    __syncthreads();
    return r;
}

template <typename TI, typename T>
__global__ void scan_reduce_kernel(const TI* __restrict__ in, int64_t n, T* __restrict__ sums) {
    __shared__ T red[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    T acc = 0;
    for (int64_t i = base + threadIdx.x; i < base + kScanChunk && i < n; i += kScanThreads) acc += in[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kScanThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// Exclusive scan of the block sums in place (single block, sequential tiles);
// the grand total goes to *total_out when given.
template <typename T>
__global__ void scan_top_kernel(T* __restrict__ sums, int64_t nb, T* __restrict__ total_out) {
    __shared__ T warp_tot[kScanThreads / 32];
    __shared__ T total;
    T carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        T v = i < nb ? sums[i] : T(0);
        T e = block_exclusive_scan(v, warp_tot, &total);
        if (i < nb) sums[i] = carry + e;
        carry += total;
        __syncthreads();
    }
    if (total_out && threadIdx.x == 0) *total_out = carry;
}

template <typename TI, typename T>
__global__ void scan_apply_kernel(const TI* __restrict__ in, T* __restrict__ out, int64_t n,
                                  const T* __restrict__ sums) {
    __shared__ T warp_tot[kScanThreads / 32];
    __shared__ T total;
    T carry = sums[blockIdx.x];
    const int64_t cbase = (int64_t)blockIdx.x * kScanChunk;
    for (int t = 0; t < kScanTilesPerBlock; ++t) {
        const int64_t base = cbase + (int64_t)t * kScanTile;
        if (base >= n) break;
        T v[kScanItems];
        T local = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
            v[k] = i < n ? T(in[i]) : T(0);
            local += v[k];
        }
        T e = block_exclusive_scan(local, warp_tot, &total);
        T run = carry + e;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
            if (i < n) out[i] = run;
            run += v[k];
        }
        carry += total;
        __syncthreads();
    }
}

template <typename TI, typename T>
void exclusive_scan(const TI* in, T* out, int64_t n, cudaStream_t s, T* total_out = nullptr) {
    if (n <= 0) return;
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    DevBuf<T> sums(nb);
    scan_reduce_kernel<TI, T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.get());
    BM_LAUNCH_CHECK();
    scan_top_kernel<T><<<1, kScanThreads, 0, s>>>(sums.get(), nb, total_out);
    BM_LAUNCH_CHECK();
    scan_apply_kernel<TI, T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums.get());
    BM_LAUNCH_CHECK();  // sums is released stream-ordered after the kernels
}

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan<int64_t, int64_t>(in, out, n, s);
}
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan<uint32_t, uint32_t>(in, out, n, s);
}
void offsets_from_counts(const int32_t* counts, int64_t n, int64_t* off, cudaStream_t s) {
    exclusive_scan<int32_t, int64_t>(counts, off, n, s, off + n);
}

}  // namespace bm
