// Pointing ingest: the precomputation the paper performs once before the
// solve (ProcessTimeSamples, Sec. III-A item 1).  From pix[t] and psi[t] (or
// the caller's cos 2psi, sin 2psi):
//   - validate pixel indices (-1 = flagged, else [0, npix)) and angles;
//   - cos 2psi, sin 2psi in time order (FP64 from psi, stored as FP32 hi + lo
//     pairs; or the given FP32 values, which then define the operator);
//   - a stable sort of the samples by pixel (LSD radix sort), giving the
//     permutation perm, the trig pairs in pixel-sorted order, and the CSR
//     offsets off[npix+1] and hit counts of the sorted order.
//
// Radix sort layout.  The samples are cut into G contiguous ranges, one per
// block, each a whole number of 8192-sample tiles.  A pass counts the digits
// of every range (bins x G counters), scans them digit-major, and each block
// then walks its own range tile by tile, placing a tile's samples at its
// running per-digit offsets.  The counter array stays small (G is a few
// times the SM count), so the digits can be wide: up to 10 bits, two passes
// for npix < 2^20 (nside <= 256), three up to nside 2048, one below 2^10.  Inside a tile the
// stable rank of a sample comes from per-warp counters updated round by round
// (match_any groups equal digits within a round), and the tile is staged in
// shared memory in digit order so that each digit's run is written
// contiguously.  Each thread loads its 16 samples (key, index, trig pair)
// before ranking them, so a tile costs one memory latency, not one per round.
//
// The trig pairs travel with the keys as payload (each pass reads and writes
// them once, in tile order): on this part a random 8-byte read moves about
// 100 bytes of DRAM traffic, so gathering them through perm afterwards would
// cost several times more.  Between passes a sample is one 16-byte record
// {TOD value, sample index, cos, sin} (the TOD word is used when a TOD is
// sorted along), with the keys written as their own stream for the next
// pass's histogram and ranking; the first pass takes its keys from the
// validated pixel indices.  The last pass writes only perm, the sorted trig
// pairs (and TOD), and the CSR offsets come from a binary search per pixel
// over pix[perm[i]].
#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int IG_THREADS = 256;
constexpr int IG_WARPS = IG_THREADS / 32;
constexpr int IG_PER_THREAD = 16;
constexpr int IG_TILE = IG_THREADS * IG_PER_THREAD;  // 4096 samples
// The scatter runs one 512-thread block per SM on 8192-sample tiles: the
// partly written output lines it keeps open in L2 (digits x streams x
// blocks) stay well inside the 126 MB, and each digit's run per tile is
// twice as long as with 4096-sample tiles.
constexpr int SC_THREADS = 512;
constexpr int SC_WARPS = SC_THREADS / 32;
constexpr int SC_TILE = SC_THREADS * IG_PER_THREAD;  // 8192 samples
constexpr int IG_WARP_SPAN = 512;                     // consecutive samples per warp in a tile
constexpr int SC_INFLIGHT = 4;                        // write-out: samples per thread with loads in flight
constexpr int RS_MAX_BITS = 10;
constexpr uint32_t kNoDigit = 0xFFFFFFFFu;

struct SortPlan {
    int bits = 1, passes = 1, bins = 2, grid = 1;
    int64_t range = SC_TILE;  // samples per block, a multiple of SC_TILE
};

__device__ __forceinline__ int64_t range_begin(int64_t range) { return (int64_t)blockIdx.x * range; }

// Stores that ask L2 to keep their lines (evict_last): a scatter pass writes
// each digit's output run a few samples per tile, so a 32-byte sector is
// completed by later tiles of the same block; evicting it half written would
// cost a read-modify-write in DRAM.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(uint4* p, uint4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_keep(float2* p, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}

// ----------------------------------------------------------------- validate
// Checks pixel indices and angles (or the given cos/sin pairs, |.| <= 1),
// copies pix (the first sort pass reads its keys from this copy: flagged
// samples get key npix and sort last) and writes the time-ordered trig
// pairs.  counters[0] = invalid samples,
// counters[1] = flagged samples.  With tod_dst, also copies the TOD
// (a host-memory source read once over the host link).
// MODE: kTrigIn (cos/sin given), kPsi64 or kPsi32 (angles given).
constexpr int kTrigIn = 0, kPsi64 = 1, kPsi32 = 2;
template <int MODE>
__global__ void validate_kernel(const int32_t* __restrict__ pix, const void* __restrict__ psi,
                                const float* __restrict__ c32, const float* __restrict__ s32, int64_t n,
                                int64_t npix, int32_t* __restrict__ pix_out,
                                float2* __restrict__ hi, float2* __restrict__ lo,
                                const float* __restrict__ tod_src, float* __restrict__ tod_dst,
                                unsigned long long* __restrict__ counters) {
    unsigned nbad = 0, nflag = 0;
    auto one = [&](int64_t i, int32_t p, float c, float s, double a) {
        const bool ok_p = (p >= -1) && ((int64_t)p < npix);
        bool ok_a;
        if constexpr (MODE == kTrigIn) {
            ok_a = fabsf(c) <= 1.0f && fabsf(s) <= 1.0f;  // false for NaN
            hi[i] = make_float2(c, s);
        } else {
            ok_a = isfinite(a);
            double sn, cs;
            sincos(2.0 * (ok_a ? a : 0.0), &sn, &cs);
            const float ch = (float)cs, sh = (float)sn;
            hi[i] = make_float2(ch, sh);
            lo[i] = make_float2((float)(cs - (double)ch), (float)(sn - (double)sh));
        }
        const bool kept = ok_p && p >= 0;
        nbad += (!ok_p) + (!ok_a);
        nflag += !kept;
        pix_out[i] = ok_p ? p : -1;
    };
    // four samples per thread and pass, their loads issued together
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
        int32_t p[U];
        float c[U], sv[U];
        double a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            const bool v = i < n;
            p[u] = v ? __ldcs(pix + i) : 0;
            c[u] = sv[u] = 0.f;
            a[u] = 0.0;
            if constexpr (MODE == kTrigIn) {
                if (v) {
                    c[u] = __ldcs(c32 + i);
                    sv[u] = __ldcs(s32 + i);
                }
            } else if constexpr (MODE == kPsi64) {
                if (v) a[u] = __ldcs(static_cast<const double*>(psi) + i);
            } else {
                if (v) a[u] = (double)__ldcs(static_cast<const float*>(psi) + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) one(i, p[u], c[u], sv[u], a[u]);
        }
        if (tod_dst) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * stride;
                if (i < n) tod_dst[i] = __ldcs(tod_src + i);
            }
        }
    }
    nbad = __reduce_add_sync(0xffffffffu, nbad);
    nflag = __reduce_add_sync(0xffffffffu, nflag);
    if ((threadIdx.x & 31) == 0) {
        if (nbad) atomicAdd(&counters[0], (unsigned long long)nbad);
        if (nflag) atomicAdd(&counters[1], (unsigned long long)nflag);
    }
}

// ------------------------------------------------------------ radix sort
// The first pass reads the validated pixel indices as its keys: -1 (flagged)
// becomes flag_key = npix.  Later passes (flag_key = 0) read keys as stored.
__device__ __forceinline__ uint32_t pixel_key(uint32_t raw, uint32_t flag_key) {
    return (flag_key && (int32_t)raw < 0) ? flag_key : raw;
}

// Digit counts of the block's range for one pass: hist[d * G + block].
// Each thread counts 16 consecutive keys (vector loads), adding runs of equal
// digits at once into its warp's own histogram; the warp histograms are
// summed at the end.
__global__ void __launch_bounds__(IG_THREADS)
rs_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int64_t range, int shift, int bins, int G,
               uint32_t flag_key, uint32_t* __restrict__ hist) {
    extern __shared__ __align__(16) uint32_t hh[];  // [IG_WARPS][bins]
    for (int d = threadIdx.x; d < IG_WARPS * bins; d += IG_THREADS) hh[d] = 0;
    __syncthreads();
    uint32_t* mine = hh + (threadIdx.x >> 5) * bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    const int64_t begin = range_begin(range);
    const int64_t end = begin + range < n ? begin + range : n;
    for (int64_t base = begin; base < end; base += IG_TILE) {
        const int64_t i0 = base + (int64_t)threadIdx.x * IG_PER_THREAD;
        uint32_t k[IG_PER_THREAD];
        if (i0 + IG_PER_THREAD <= end) {
            const uint4* v = reinterpret_cast<const uint4*>(keys + i0);  // i0 is a multiple of 16
#pragma unroll
            for (int q = 0; q < IG_PER_THREAD / 4; ++q) {
                const uint4 x = __ldcs(v + q);
                k[4 * q] = pixel_key(x.x, flag_key);
                k[4 * q + 1] = pixel_key(x.y, flag_key);
                k[4 * q + 2] = pixel_key(x.z, flag_key);
                k[4 * q + 3] = pixel_key(x.w, flag_key);
            }
        } else {
#pragma unroll
            for (int r = 0; r < IG_PER_THREAD; ++r) k[r] = i0 + r < end ? pixel_key(keys[i0 + r], flag_key) : kNoDigit;
        }
        uint32_t cur = kNoDigit, run = 0;
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const uint32_t d = k[r] == kNoDigit ? kNoDigit : ((k[r] >> shift) & dmask);
            if (d == cur) {
                ++run;
            } else {
                if (run) atomicAdd(&mine[cur], run);
                cur = d;
                run = d != kNoDigit;
            }
        }
        if (run) atomicAdd(&mine[cur], run);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += IG_THREADS) {
        uint32_t t = 0;
#pragma unroll
        for (int q = 0; q < IG_WARPS; ++q) t += hh[q * bins + d];
        hist[(int64_t)d * G + blockIdx.x] = t;
    }
}

// Exclusive scan of cnt[0, bins) into start[] by the whole block (THREADS threads).
template <int THREADS>
__device__ void scan_bins(const uint32_t* cnt, uint32_t* start, int bins, uint32_t* wtot) {
    constexpr int WARPS = THREADS / 32;
    const int per = bins >= THREADS ? bins / THREADS : 1;
    const int b0 = threadIdx.x * per;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < bins) local += cnt[b0 + k];
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < WARPS ? wtot[lane] : 0u;
        uint32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < WARPS) wtot[lane] = s - t;
    }
    __syncthreads();
    uint32_t run = x - local + wtot[w];
    for (int k = 0; k < per; ++k)
        if (b0 + k < bins) {
            start[b0 + k] = run;
            run += cnt[b0 + k];
        }
}

// A sample between passes: one 16-byte record {TOD value, sample index,
// cos, sin} (one store stream instead of three: the scatter's short digit
// runs then fill whole lines, which measured twice as fast).  The keys travel
// as their own stream, so the first word of the record is free for the TOD
// sample when one is sorted along (else it is unused).
struct ScatterArgs {
    const uint4* rec_in;      // records of the previous pass, or null on the first pass:
                              //   then the sample index itself, the trig pairs and the TOD in time order
    const uint32_t* keys_in;  // keys in this pass's input order
    const float2* hi_in;
    const float* tod_in;      // first pass: the TOD in time order, or null
    const float2* lo_in;      // lo halves of the trig pairs in this pass's input order, or null
    int64_t n;
    int64_t range;
    int shift, bins, G;
    const uint32_t* offs;  // [bins][G] exclusive digit-major scan of the counts
    uint4* rec_out;        // intermediate passes: records, and the keys alone for the next pass
    uint32_t* keys_out;
    uint32_t* perm_out;    // last pass: sample indices (perm) and trig pairs of the kept samples
    float2* hi_out;
    float* tod_out;        // last pass: the TOD of the kept samples in sorted order, or null
    float2* lo_out;        // every pass with lo_in: the lo halves in this pass's output order
    uint32_t key_limit;    // last pass: samples with keys >= key_limit (flagged) get no entry
    uint32_t flag_key;     // first pass: keys_in are pixel indices, -1 maps to flag_key (= npix)
};

inline size_t scatter_smem(int bins) {
    return sizeof(uint32_t) * ((size_t)SC_TILE + 3 * (size_t)bins) +
           sizeof(uint16_t) * ((size_t)SC_TILE + (size_t)SC_WARPS * bins);
}

// One stable scatter pass over the block's range (see the file comment).
// Only the key and the tile position of each sample are staged in shared
// memory (6 bytes a sample, so two 512-thread blocks fit on an SM); at write
// time the rest of the sample (index, trig pair, lo half) is read back from
// the tile's window of the input, which the key loads have just brought
// into L2.
template <bool LAST, bool FIRST>
__global__ void __launch_bounds__(SC_THREADS, 2) rs_scatter_kernel(ScatterArgs a) {
    extern __shared__ __align__(16) uint32_t ss[];
    uint32_t* s_keys = ss;
    uint32_t* run_base = s_keys + SC_TILE;  // next global position per digit
    uint32_t* tcnt = run_base + a.bins;     // tile count per digit
    uint32_t* tstart = tcnt + a.bins;       // tile-local start per digit
    uint16_t* s_src = reinterpret_cast<uint16_t*>(tstart + a.bins);  // tile position of a staged sample
    uint16_t* wcnt = s_src + SC_TILE;                                 // [warp][digit]
    __shared__ uint32_t wtot[SC_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int bins = a.bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    const int64_t begin = range_begin(a.range);
    const int64_t end = begin + a.range < a.n ? begin + a.range : a.n;
    const uint64_t pol = l2_keep_policy();

    for (int d = threadIdx.x; d < bins; d += SC_THREADS) {
        run_base[d] = a.offs[(int64_t)d * a.G + blockIdx.x];
#pragma unroll
        for (int q = 0; q < SC_WARPS; ++q) wcnt[q * bins + d] = 0;
    }
    __syncthreads();

    for (int64_t base = begin; base < end; base += SC_TILE) {
        const int cnt = (int)(end - base < SC_TILE ? end - base : SC_TILE);
        uint32_t key[IG_PER_THREAD], rank[IG_PER_THREAD];
        // 1. the warp's 512 consecutive keys, 32 per round
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const int j = w * IG_WARP_SPAN + r * 32 + lane;
            key[r] = j < cnt ? (FIRST ? pixel_key(a.keys_in[base + j], a.flag_key) : a.keys_in[base + j]) : 0u;
        }
        // 2. stable rank within the warp: counters advance round by round
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const int j = w * IG_WARP_SPAN + r * 32 + lane;
            const uint32_t d = j < cnt ? ((key[r] >> a.shift) & dmask) : kNoDigit;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (d != kNoDigit && lane == leader) {
                old = wcnt[w * bins + d];
                wcnt[w * bins + d] = (uint16_t)(old + __popc(peers));
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[r] = old + __popc(peers & lt_mask);
            __syncwarp();
        }
        __syncthreads();
        // 3. per digit: exclusive prefix over warps, tile count; then over digits
        for (int d = threadIdx.x; d < bins; d += SC_THREADS) {
            uint32_t t = 0;
#pragma unroll
            for (int q = 0; q < SC_WARPS; ++q) {
                const uint32_t c = wcnt[q * bins + d];
                wcnt[q * bins + d] = (uint16_t)t;
                t += c;
            }
            tcnt[d] = t;
        }
        __syncthreads();
        scan_bins<SC_THREADS>(tcnt, tstart, bins, wtot);
        __syncthreads();
        // 4. stage keys and tile positions in digit order
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const int j = w * IG_WARP_SPAN + r * 32 + lane;
            if (j < cnt) {
                const uint32_t d = (key[r] >> a.shift) & dmask;
                const uint32_t pos = tstart[d] + wcnt[w * bins + d] + rank[r];
                s_keys[pos] = key[r];
                s_src[pos] = (uint16_t)j;
            }
        }
        __syncthreads();
        // 5. each digit's run goes to its running global offset, the rest of
        //    each sample read back from the input window; four per thread in
        //    flight
        for (int j0 = threadIdx.x; j0 < cnt; j0 += SC_INFLIGHT * SC_THREADS) {
            uint32_t kk[SC_INFLIGHT];
            uint4 rr[SC_INFLIGHT];
#pragma unroll
            for (int u = 0; u < SC_INFLIGHT; ++u) {
                const int j = j0 + u * SC_THREADS;
                kk[u] = kNoDigit;
                if (j < cnt) {
                    kk[u] = s_keys[j];
                    const uint32_t src = s_src[j];
                    if (!FIRST) {
                        rr[u] = a.rec_in[base + src];
                    } else {
                        const float2 h = a.hi_in[base + src];
                        const float d = a.tod_in ? a.tod_in[base + src] : 0.f;
                        rr[u] = make_uint4(__float_as_uint(d), (uint32_t)(base + src), __float_as_uint(h.x),
                                           __float_as_uint(h.y));
                    }
                }
            }
            // the output positions while the loads are in flight
#pragma unroll
            for (int u = 0; u < SC_INFLIGHT; ++u) {
                if (kk[u] == kNoDigit) continue;
                const int j = j0 + u * SC_THREADS;
                const uint32_t d = (kk[u] >> a.shift) & dmask;
                const uint32_t g = run_base[d] + (uint32_t)j - tstart[d];
                if (!LAST) {
                    st_keep(a.rec_out + g, rr[u], pol);
                    st_keep(a.keys_out + g, kk[u], pol);
                    if (a.lo_in) st_keep(a.lo_out + g, a.lo_in[base + s_src[j]], pol);
                } else if (kk[u] < a.key_limit) {
                    st_keep(a.perm_out + g, rr[u].y, pol);
                    st_keep(a.hi_out + g, make_float2(__uint_as_float(rr[u].z), __uint_as_float(rr[u].w)), pol);
                    if (a.tod_out) st_keep(reinterpret_cast<uint32_t*>(a.tod_out) + g, rr[u].x, pol);
                    if (a.lo_in) st_keep(a.lo_out + g, a.lo_in[base + s_src[j]], pol);
                }
            }
        }
        __syncthreads();
        // 6. advance the running offsets, clear the warp counters
        for (int d = threadIdx.x; d < bins; d += SC_THREADS) {
            run_base[d] += tcnt[d];
#pragma unroll
            for (int q = 0; q < SC_WARPS; ++q) wcnt[q * bins + d] = 0;
        }
        __syncthreads();
    }
}

// off[p] = first sorted position whose pixel is >= p, for p in [0, npix]:
// a binary search over the kept samples, the pixel of sorted position i
// being pix[perm[i]].
__global__ void lower_bound_kernel(const uint32_t* __restrict__ perm, const int32_t* __restrict__ pix,
                                   int64_t nvalid, int64_t npix, int64_t* __restrict__ off) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nvalid;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)pix[perm[mid]] < p) lo = mid + 1; else hi = mid;
        }
        off[p] = lo;
    }
}

__global__ void hits_kernel(const int64_t* __restrict__ off, int64_t npix, int32_t* __restrict__ hits) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x)
        hits[p] = (int32_t)(off[p + 1] - off[p]);
}


SortPlan plan_sort(const bm_context* ctx, int64_t n, int64_t npix) {
    SortPlan sp;
    int nbits = 1;
    while (((int64_t)1 << nbits) <= npix) ++nbits;  // the flagged key npix must fit too
    sp.passes = (nbits + RS_MAX_BITS - 1) / RS_MAX_BITS;
    sp.bits = (nbits + sp.passes - 1) / sp.passes;
    sp.bins = 1 << sp.bits;
    const size_t smem = scatter_smem(sp.bins);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_scatter_kernel<false, true>), smem);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_scatter_kernel<false, false>), smem);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_scatter_kernel<true, true>), smem);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_scatter_kernel<true, false>), smem);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_hist_kernel), sizeof(uint32_t) * IG_WARPS * sp.bins);
    int per_sm = blocks_per_sm(reinterpret_cast<const void*>(rs_scatter_kernel<true, false>), SC_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    // four waves of equal ranges keep the tail short
    const int64_t want = (int64_t)ctx->num_sms * per_sm * 4;
    const int64_t ntiles = (n + SC_TILE - 1) / SC_TILE;
    const int64_t tiles_per_block = (ntiles + want - 1) / want;
    sp.range = tiles_per_block * SC_TILE;
    sp.grid = (int)((n + sp.range - 1) / sp.range);
    return sp;
}

}  // namespace

void ingest(bm_pointing* p, const int32_t* pix, const void* psi, bm_dtype psi_dtype, const float* cos2psi,
            const float* sin2psi, const float* tod, bool tod_on_host) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    ScopedTimer timer(ctx, "ingest");
    const int64_t n = p->nsamples, npix = p->npix;
    const bool exact_trig = cos2psi != nullptr;  // FP32 trig given: it defines the operator, no lo part
    const bool has_lo = !exact_trig;
    const SortPlan sp = plan_sort(ctx, n, npix);
    const int threads = 256;

    p->pix.alloc(n);
    p->cs_hi_t.alloc(n);
    if (has_lo) p->cs_lo_t.alloc(n);
    DevBuf<float> tod_copy;  // a host TOD, copied by the validation pass
    if (tod && tod_on_host) tod_copy.alloc(n);
    const float* tod_t = tod_on_host ? tod_copy.get() : tod;
    DevBuf<unsigned long long> counters(2);
    BM_CUDA(cudaMemsetAsync(counters.get(), 0, 2 * sizeof(unsigned long long), s));
    {
        ScopedTimer vt(ctx, "ingest_validate");
        auto kern = exact_trig ? validate_kernel<kTrigIn>
                               : (psi_dtype == BM_F64 ? validate_kernel<kPsi64> : validate_kernel<kPsi32>);
        const int grid = resident_grid(ctx, kern, threads, (n + threads - 1) / threads);
        kern<<<grid, threads, 0, s>>>(pix, psi, cos2psi, sin2psi, n, npix, p->pix.get(),
                                      p->cs_hi_t.get(), p->cs_lo_t.get(), tod_on_host ? tod : nullptr,
                                      tod_copy.get(), counters.get());
        BM_LAUNCH_CHECK();
    }
    unsigned long long h_cnt[2] = {0, 0};
    BM_CUDA(cudaMemcpyAsync(h_cnt, counters.get(), sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    BM_REQUIRE(h_cnt[0] == 0, "%llu samples have a pixel index outside [-1, %lld) or a bad angle / trig value",
               h_cnt[0], (long long)npix);
    const int64_t nvalid = n - (int64_t)h_cnt[1];
    p->nvalid = nvalid;
    p->perm.alloc(nvalid > 0 ? nvalid : 1);
    p->cs_hi_s.alloc(nvalid > 0 ? nvalid : 1);
    if (has_lo) p->cs_lo_s.alloc(nvalid > 0 ? nvalid : 1);
    if (tod) p->tod_s.alloc(nvalid > 0 ? nvalid : 1);
    else p->tod_s.release();

    // Ping-pong record buffers of the intermediate passes (and the lo halves
    // of the trig pairs when the angles were given).
    DevBuf<uint32_t> hist((size_t)sp.bins * sp.grid);
    DevBuf<uint4> rec_a, rec_b;
    DevBuf<uint32_t> keys_a, keys_b;
    DevBuf<float2> lo_a, lo_b;
    if (sp.passes > 1) {
        rec_a.alloc(n);
        keys_a.alloc(n);
        if (has_lo) lo_a.alloc(n);
    }
    if (sp.passes > 2) {
        rec_b.alloc(n);
        keys_b.alloc(n);
        if (has_lo) lo_b.alloc(n);
    }
    // the first pass reads its keys from the validated pixel indices
    const uint32_t* kin = reinterpret_cast<const uint32_t*>(p->pix.get());
    uint32_t* kout = keys_a.get();
    const size_t smem = scatter_smem(sp.bins);
    const uint4* rin = nullptr;  // the first pass reads keys, indices and trig in time order
    uint4* rout = rec_a.get();
    const float2* lin = has_lo ? p->cs_lo_t.get() : nullptr;
    float2* lout = lo_a.get();
    for (int pass = 0; pass < sp.passes; ++pass) {
        const int shift = pass * sp.bits;
        {
            ScopedTimer ht(ctx, "ingest_hist");
            const size_t hsm = sizeof(uint32_t) * IG_WARPS * sp.bins;
            rs_hist_kernel<<<sp.grid, IG_THREADS, hsm, s>>>(kin, n, sp.range, shift, sp.bins, sp.grid,
                                                            pass == 0 ? (uint32_t)npix : 0u, hist.get());
            BM_LAUNCH_CHECK();
        }
        exclusive_scan_u32(hist.get(), hist.get(), (int64_t)sp.bins * sp.grid, s);
        ScatterArgs a{};
        a.rec_in = rin;
        a.keys_in = kin;
        a.hi_in = p->cs_hi_t.get();
        a.tod_in = pass == 0 ? tod_t : nullptr;
        a.lo_in = lin;
        a.n = n;
        a.range = sp.range;
        a.shift = shift;
        a.bins = sp.bins;
        a.G = sp.grid;
        a.offs = hist.get();
        a.flag_key = (uint32_t)npix;
        ScopedTimer st(ctx, "ingest_scatter");
        if (pass + 1 < sp.passes) {
            a.rec_out = rout;
            a.keys_out = kout;
            a.lo_out = lout;
            if (pass == 0) rs_scatter_kernel<false, true><<<sp.grid, SC_THREADS, smem, s>>>(a);
            else rs_scatter_kernel<false, false><<<sp.grid, SC_THREADS, smem, s>>>(a);
            BM_LAUNCH_CHECK();
            kin = kout;
            kout = (kout == keys_a.get()) ? keys_b.get() : keys_a.get();
            rin = rout;
            rout = (rout == rec_a.get()) ? rec_b.get() : rec_a.get();
            lin = has_lo ? lout : nullptr;
            lout = (lout == lo_a.get()) ? lo_b.get() : lo_a.get();
        } else {
            a.perm_out = p->perm.get();
            a.hi_out = p->cs_hi_s.get();
            a.tod_out = tod ? p->tod_s.get() : nullptr;
            a.lo_out = has_lo ? p->cs_lo_s.get() : nullptr;
            a.key_limit = (uint32_t)npix;
            if (pass == 0) rs_scatter_kernel<true, true><<<sp.grid, SC_THREADS, smem, s>>>(a);
            else rs_scatter_kernel<true, false><<<sp.grid, SC_THREADS, smem, s>>>(a);
            BM_LAUNCH_CHECK();
        }
    }
    p->off.alloc(npix + 1);
    p->hits.alloc(npix);
    const int pgrid = grid_for(ctx, (npix + 1 + threads - 1) / threads, 16);
    lower_bound_kernel<<<pgrid, threads, 0, s>>>(p->perm.get(), p->pix.get(), nvalid, npix, p->off.get());
    BM_LAUNCH_CHECK();
    hits_kernel<<<pgrid, threads, 0, s>>>(p->off.get(), npix, p->hits.get());
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bm
