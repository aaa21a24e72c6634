// Pointing ingest: the precomputation the paper performs once before the
// solve (ProcessTimeSamples, Sec. III-A item 1).  From pix[t] and psi[t]:
//   - validate pixel indices (-1 = flagged, else [0, npix));
//   - cos 2psi, sin 2psi in FP64, stored as FP32 (hi, lo) pairs in time order;
//   - a stable sort of the valid samples by pixel (LSD radix sort, 8-bit
//     digits, deterministic tile ranks), giving the permutation perm, the CSR
//     offsets off[npix+1] and the hit counts;
//   - the trig pairs gathered into pixel-sorted order.
#include "bm_internal.cuh"

namespace bm {

namespace {

// ----------------------------------------------------------------- validate
// Checks pixel indices and angles (or the given cos/sin pairs, |.| <= 1),
// copies pix and writes the sort keys.  With cos/sin given, also interleaves
// them into the time-ordered trig array.
__global__ void validate_kernel(const int32_t* __restrict__ pix, const void* __restrict__ psi,
                                int psi_f64, const float* __restrict__ c32, const float* __restrict__ s32,
                                int64_t n, int64_t npix, int32_t* __restrict__ pix_out,
                                uint32_t* __restrict__ keys, float2* __restrict__ hi,
                                unsigned long long* __restrict__ bad) {
    unsigned long long nbad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[i];
        const bool ok_p = (p >= -1) && ((int64_t)p < npix);
        bool ok_a;
        if (c32) {
            const float c = c32[i], s = s32[i];
            ok_a = fabsf(c) <= 1.0f && fabsf(s) <= 1.0f;  // false for NaN
            hi[i] = make_float2(c, s);
        } else {
            const double a = psi_f64 ? static_cast<const double*>(psi)[i]
                                     : (double)static_cast<const float*>(psi)[i];
            ok_a = isfinite(a);
        }
        nbad += (!ok_p) + (!ok_a);
        pix_out[i] = ok_p ? p : -1;
        keys[i] = (ok_p && p >= 0) ? (uint32_t)p : (uint32_t)npix;  // flagged sort last
    }
    nbad = __reduce_add_sync(0xffffffffu, (unsigned)nbad);
    if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, nbad);
}

// cos 2psi and sin 2psi in FP64, split into FP32 hi + FP32 lo.
__global__ void trig_kernel(const void* __restrict__ psi, int psi_f64, int64_t n,
                            float2* __restrict__ hi, float2* __restrict__ lo) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = psi_f64 ? static_cast<const double*>(psi)[i]
                                 : (double)static_cast<const float*>(psi)[i];
        double s, c;
        sincos(2.0 * a, &s, &c);
        const float ch = (float)c, sh = (float)s;
        hi[i] = make_float2(ch, sh);
        lo[i] = make_float2((float)(c - (double)ch), (float)(s - (double)sh));
    }
}

// ------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                         // 32-element rounds per warp
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;       // 4096 keys per tile
constexpr int RS_BINS = 256;

__global__ void rs_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                               int64_t ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_BINS];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) h[d] = 0;
        __syncthreads();
        const int64_t base = tile * RS_TILE;
        for (int j = threadIdx.x; j < RS_TILE; j += RS_THREADS) {
            const int64_t i = base + j;
            if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) hist[(int64_t)d * ntiles + tile] = h[d];
        __syncthreads();
    }
}

// Stable scatter of one digit pass.  Each warp owns 512 consecutive keys of
// the tile and ranks them in order (match_any + popc), warps are combined by
// a per-digit prefix, and the tile is staged in shared memory in digit order
// so that the global writes of a digit run are contiguous.
__global__ void __launch_bounds__(RS_THREADS)
rs_scatter_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                  int64_t n, int shift, int64_t ntiles, const uint32_t* __restrict__ offs,
                  uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t s_keys[RS_TILE];
    __shared__ uint32_t s_vals[RS_TILE];
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
    __shared__ uint32_t dstart[RS_BINS];
    __shared__ uint32_t gbase[RS_BINS];
    __shared__ uint32_t wtot[RS_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * RS_TILE;
        const int cnt = (int)((n - base) < RS_TILE ? (n - base) : RS_TILE);
        for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
#pragma unroll
            for (int q = 0; q < RS_WARPS; ++q) wcnt[q][d] = 0;
            gbase[d] = offs[(int64_t)d * ntiles + tile];
        }
        __syncthreads();
        // 1. per-warp digit counts
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int j = w * (RS_TILE / RS_WARPS) + r * 32 + lane;
            const bool valid = j < cnt;
            const uint32_t d = valid ? ((keys_in[base + j] >> shift) & 0xFF) : 0x100u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid && lane == __ffs(peers) - 1) wcnt[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // 2. per digit: exclusive prefix over warps; tile total
        uint32_t tot = 0;
        if (threadIdx.x < RS_BINS) {
            const int d = threadIdx.x;
#pragma unroll
            for (int q = 0; q < RS_WARPS; ++q) {
                const uint32_t c = wcnt[q][d];
                wcnt[q][d] = tot;
                tot += c;
            }
        }
        // exclusive scan of tile totals over digits (RS_BINS == RS_THREADS)
        {
            uint32_t x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wtot[w] = x;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t run = 0;
                for (int q = 0; q < RS_WARPS; ++q) { const uint32_t t = wtot[q]; wtot[q] = run; run += t; }
            }
            __syncthreads();
            dstart[threadIdx.x] = x - tot + wtot[w];
        }
        __syncthreads();
        // 3. ranks; stage keys/vals in digit order
        for (int r = 0; r < RS_ROUNDS; ++r) {
            const int j = w * (RS_TILE / RS_WARPS) + r * 32 + lane;
            const bool valid = j < cnt;
            const uint32_t key = valid ? keys_in[base + j] : 0u;
            const uint32_t d = valid ? ((key >> shift) & 0xFF) : 0x100u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const uint32_t pos = dstart[d] + wcnt[w][d] + __popc(peers & lt_mask);
                s_keys[pos] = key;
                s_vals[pos] = vals_in ? vals_in[base + j] : (uint32_t)(base + j);
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wcnt[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // 4. contiguous writes per digit run
        for (int j = threadIdx.x; j < cnt; j += RS_THREADS) {
            const uint32_t key = s_keys[j];
            const uint32_t d = (key >> shift) & 0xFF;
            const uint64_t pos = (uint64_t)gbase[d] + (uint64_t)(j - (int)dstart[d]);
            keys_out[pos] = key;
            vals_out[pos] = s_vals[j];
        }
        __syncthreads();
    }
}

// off[p] = first sorted index whose key >= p, for p in [0, npix].
__global__ void lower_bound_kernel(const uint32_t* __restrict__ keys, int64_t n, int64_t npix,
                                   int64_t* __restrict__ off, int32_t* __restrict__ hits_unused) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < p) lo = mid + 1; else hi = mid;
        }
        off[p] = lo;
    }
}

__global__ void hits_kernel(const int64_t* __restrict__ off, int64_t npix, int32_t* __restrict__ hits) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x)
        hits[p] = (int32_t)(off[p + 1] - off[p]);
}

__global__ void gather_trig_kernel(const uint32_t* __restrict__ perm, int64_t n,
                                   const float2* __restrict__ hi_t, const float2* __restrict__ lo_t,
                                   float2* __restrict__ hi_s, float2* __restrict__ lo_s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = perm[i];
        hi_s[i] = hi_t[t];
        if (lo_t) lo_s[i] = lo_t[t];
    }
}

}  // namespace

void ingest(bm_pointing* p, const int32_t* pix, const void* psi, bm_dtype psi_dtype, const float* cos2psi,
            const float* sin2psi) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    ScopedTimer timer(ctx, "ingest");
    const int64_t n = p->nsamples, npix = p->npix;
    const int psi_f64 = psi_dtype == BM_F64;
    const int threads = 256;
    const int grid = grid_for(ctx, (n + threads - 1) / threads, 16);

    const bool exact_trig = cos2psi != nullptr;  // FP32 trig given: it defines the operator, no lo part
    p->pix.alloc(n);
    p->cs_hi_t.alloc(n);
    if (!exact_trig) p->cs_lo_t.alloc(n);
    DevBuf<uint32_t> keys_a(n), keys_b(n), vals_a(n), vals_b(n);
    DevBuf<unsigned long long> bad(1);
    BM_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(unsigned long long), s));
    validate_kernel<<<grid, threads, 0, s>>>(pix, psi, psi_f64, cos2psi, sin2psi, n, npix, p->pix.get(),
                                             keys_a.get(), p->cs_hi_t.get(), bad.get());
    BM_LAUNCH_CHECK();
    unsigned long long h_bad = 0;
    BM_CUDA(cudaMemcpyAsync(&h_bad, bad.get(), sizeof(h_bad), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    BM_REQUIRE(h_bad == 0, "%llu samples have a pixel index outside [-1, %lld) or a bad angle / trig value",
               h_bad, (long long)npix);

    if (!exact_trig) {
        trig_kernel<<<grid, threads, 0, s>>>(psi, psi_f64, n, p->cs_hi_t.get(), p->cs_lo_t.get());
        BM_LAUNCH_CHECK();
    }

    // LSD radix sort of (key, sample index) over the bits of npix.
    int nbits = 1;
    while (((int64_t)1 << nbits) <= npix) ++nbits;
    const int passes = (nbits + 7) / 8;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    DevBuf<uint32_t> hist((size_t)RS_BINS * ntiles);
    const int rs_grid = (int)std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * 4);
    uint32_t* kin = keys_a.get();
    uint32_t* kout = keys_b.get();
    uint32_t* vin = nullptr;  // identity on the first pass
    uint32_t* vout = vals_b.get();
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        rs_hist_kernel<<<rs_grid, RS_THREADS, 0, s>>>(kin, n, shift, ntiles, hist.get());
        BM_LAUNCH_CHECK();
        exclusive_scan_u32(hist.get(), hist.get(), (int64_t)RS_BINS * ntiles, s);
        rs_scatter_kernel<<<rs_grid, RS_THREADS, 0, s>>>(kin, vin, n, shift, ntiles, hist.get(), kout, vout);
        BM_LAUNCH_CHECK();
        std::swap(kin, kout);
        vin = vout;
        vout = (vout == vals_b.get()) ? vals_a.get() : vals_b.get();
    }
    // kin / vin now hold the sorted keys and sample indices.
    p->off.alloc(npix + 1);
    p->hits.alloc(npix);
    const int pgrid = grid_for(ctx, (npix + 1 + threads - 1) / threads, 16);
    lower_bound_kernel<<<pgrid, threads, 0, s>>>(kin, n, npix, p->off.get(), nullptr);
    BM_LAUNCH_CHECK();
    hits_kernel<<<pgrid, threads, 0, s>>>(p->off.get(), npix, p->hits.get());
    BM_LAUNCH_CHECK();
    int64_t nvalid = 0;
    BM_CUDA(cudaMemcpyAsync(&nvalid, p->off.get() + npix, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    p->nvalid = nvalid;

    p->perm.alloc(nvalid > 0 ? nvalid : 1);
    p->cs_hi_s.alloc(nvalid > 0 ? nvalid : 1);
    if (!exact_trig) p->cs_lo_s.alloc(nvalid > 0 ? nvalid : 1);
    if (nvalid > 0) {
        BM_CUDA(cudaMemcpyAsync(p->perm.get(), vin, sizeof(uint32_t) * nvalid, cudaMemcpyDeviceToDevice, s));
        gather_trig_kernel<<<grid, threads, 0, s>>>(p->perm.get(), nvalid, p->cs_hi_t.get(), p->cs_lo_t.get(),
                                                    p->cs_hi_s.get(), p->cs_lo_s.get());
        BM_LAUNCH_CHECK();
    }
    BM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bm
