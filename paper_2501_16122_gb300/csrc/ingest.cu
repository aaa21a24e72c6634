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
// for npix < 2^20 (nside <= 256), three up to nside 2048, one below 2^10.  A
// tile's keys and payload arrive in shared memory by bulk (TMA) copies; the
// stable rank of a sample comes from per-warp counters updated round by round
// (the lanes of a round holding the same digit found through lane-mask tables
// in shared memory), and the tile is staged in digit order so that each
// digit's run is written contiguously (see rs_scatter_kernel).
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
#include <algorithm>
#include <type_traits>

#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int IG_THREADS = 256;
constexpr int IG_WARPS = IG_THREADS / 32;
constexpr int IG_PER_THREAD = 16;
constexpr int IG_TILE = IG_THREADS * IG_PER_THREAD;  // 4096 samples
// The scatter: SC_THREADS threads a block, 16 samples a thread, so a tile of
// SC_TILE samples; the tile's keys and payload window sit in shared memory
// (see scatter_smem).
constexpr int SC_THREADS = 512;
constexpr int SC_WARPS = SC_THREADS / 32;
constexpr int SC_TILE = SC_THREADS * IG_PER_THREAD;
static_assert(SC_TILE <= 8192, "the last pass packs a tile position into 13 bits");
constexpr int SC_MIN_BLOCKS = SC_THREADS == 256 ? 2 : 1;  // blocks per SM the shared memory allows
constexpr int IG_WARP_SPAN = 512;                          // consecutive samples per warp in a tile
constexpr int RS_MAX_BITS = 10;
constexpr uint32_t kNoDigit = 0xFFFFFFFFu;

struct SortPlan {
    int bits = 1, passes = 1, bins = 2, grid = 1;
    int64_t range = SC_TILE;  // samples per block, a multiple of SC_TILE
    bool key16 = true;        // the keys between passes (the digits not yet consumed) fit in 16 bits
};

__device__ __forceinline__ int64_t range_begin(int64_t range) { return (int64_t)blockIdx.x * range; }

// Stores that ask L2 to keep their lines (evict_last): a scatter pass writes
// each digit's output run a few samples per tile, so a 32-byte sector is
// completed by later tiles of the same block; evicting it half written would
// cost a read-modify-write in DRAM (plain stores measured slower).
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(uint16_t* p, uint16_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(uint4* p, uint4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float2* p, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}

// ----------------------------------------------------------------- validate
// Checks pixel indices and angles (or the given cos/sin pairs, |.| <= 1),
// copies pix (the first sort pass reads its keys from this copy: flagged
// samples get key npix and sort last) and writes the time-ordered trig
// pairs.  counters[0] = invalid samples,
// counters[1] = flagged samples.  With tod_dst, also copies the TOD
// (a host-memory source read once over the host link).
// MODE: kTrigIn (cos/sin given), kPsi64 or kPsi32 (angles given), kHwp
// (the half-wave-plate model), or kPixOnly (cos/sin given and left to the
// first sort pass, which reads them once, checks them and writes the
// time-ordered pairs or leaves them to time_trig: this pass then reads and
// copies the pixels alone).
// HIST: also the first sort pass's digit counts (the sort key of each
// validated sample, flagged ones as npix, masked to the low digit) of each
// range of `range` samples, hist[d * G + range], as rs_hist_kernel counts
// them; `sub` blocks share a range (its equal parts), each adding its counts
// to the zeroed hist.  Without HIST the loop is grid-strided.
constexpr int kTrigIn = 0, kPsi64 = 1, kPsi32 = 2, kHwp = 3, kPixOnly = 4;
constexpr int kVHist = 4;  // shared-memory digit histograms per validation block
template <int MODE, bool HIST>
__global__ void __launch_bounds__(256)
validate_kernel(const int32_t* __restrict__ pix, const void* __restrict__ psi,
                const float* __restrict__ c32, const float* __restrict__ s32, int64_t n,
                int64_t npix, int32_t* __restrict__ pix_out,
                float2* __restrict__ hi, float2* __restrict__ lo,
                const float* __restrict__ tod_src, float* __restrict__ tod_dst,
                unsigned long long* __restrict__ counters, int64_t range, int sub, int bins, int G,
                uint32_t* __restrict__ hist, HwpModel hwp) {
    extern __shared__ __align__(16) uint32_t vh[];  // HIST: [kVHist][bins], one per pair of warps
    uint32_t* mine = nullptr;
    if (HIST) {
        for (int d = threadIdx.x; d < kVHist * bins; d += blockDim.x) vh[d] = 0;
        __syncthreads();
        mine = vh + ((threadIdx.x >> 5) % kVHist) * bins;
    }
    const uint32_t dmask = (uint32_t)bins - 1u;
    unsigned nbad = 0, nflag = 0;
    auto one = [&](int64_t i, int32_t p, float c, float s, double a) {
        const bool ok_p = (p >= -1) && ((int64_t)p < npix);
        bool ok_a;
        if constexpr (MODE == kTrigIn) {
            ok_a = fabsf(c) <= 1.0f && fabsf(s) <= 1.0f;  // false for NaN
            hi[i] = make_float2(c, s);
        } else if constexpr (MODE == kPixOnly) {
            ok_a = true;
        } else if constexpr (MODE == kHwp) {
            // 2 theta of the half-wave-plate model in turns, reduced exactly,
            // and its cos and sin as double-float pairs (table and short
            // polynomials on the FP32 pipes)
            ok_a = true;
            const int d = det_of(hwp.off, hwp.ndet, hwp.ns, hwp.inv_ns, (uint32_t)i);
            const unsigned long long a2 = hwp_turns(hwp, d, (uint32_t)i);
            const float4 t = hwp_trig_df(a2, hwp.tabdf);
            hi[i] = make_float2(t.x, t.y);
            lo[i] = make_float2(t.z, t.w);
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
        if (pix_out) pix_out[i] = ok_p ? p : -1;  // (null: the copy is deferred)
        if (HIST) atomicAdd(&mine[(kept ? (uint32_t)p : (uint32_t)npix) & dmask], 1u);
    };
    // four samples per thread and pass, their loads issued together
    constexpr int U = 4;
    const int64_t stride = HIST ? (int64_t)blockDim.x : (int64_t)gridDim.x * blockDim.x;
    const int64_t part = range / sub;
    const int64_t begin = HIST ? (int64_t)(blockIdx.x / sub) * range + (int64_t)(blockIdx.x % sub) * part : 0;
    const int64_t end = HIST ? (begin + part < n ? begin + part : n) : n;
    for (int64_t i0 = begin + (HIST ? 0 : (int64_t)blockIdx.x * blockDim.x) + threadIdx.x; i0 < end;
         i0 += U * stride) {
        int32_t p[U];
        float c[U], sv[U];
        double a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            const bool v = i < end;
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
            } else if constexpr (MODE == kPsi32) {
                if (v) a[u] = (double)__ldcs(static_cast<const float*>(psi) + i);
            }  // kHwp and kPixOnly read no angle
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < end) one(i, p[u], c[u], sv[u], a[u]);
        }
        if (tod_dst) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + u * stride;
                if (i < end) tod_dst[i] = __ldcs(tod_src + i);
            }
        }
    }
    if (HIST) {
        __syncthreads();
        for (int d = threadIdx.x; d < bins; d += blockDim.x) {
            uint32_t t = 0;
            for (int q = 0; q < kVHist; ++q) t += vh[q * bins + d];
            if (t) atomicAdd(&hist[(int64_t)d * G + blockIdx.x / sub], t);
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

// Digit counts of the block's range for a pass after the first:
// hist[d * G + block], the digit being the low bits of the stored key (each
// pass stores the key shifted past the digit it sorted on).  Each thread
// counts 16 consecutive keys (vector loads), adding runs of equal digits at
// once into its warp's own histogram; the warp histograms are summed at the
// end.
template <typename KT>
__global__ void __launch_bounds__(IG_THREADS)
rs_hist_kernel(const KT* __restrict__ keys, int64_t n, int64_t range, int bins, int G, uint32_t* __restrict__ hist) {
    extern __shared__ __align__(16) uint32_t hh[];  // [IG_WARPS][bins]
    for (int d = threadIdx.x; d < IG_WARPS * bins; d += IG_THREADS) hh[d] = 0;
    __syncthreads();
    uint32_t* mine = hh + (threadIdx.x >> 5) * bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    const int64_t begin = range_begin(range);
    const int64_t end = begin + range < n ? begin + range : n;
    constexpr int kPerVec = 16 / sizeof(KT);
    for (int64_t base = begin; base < end; base += IG_TILE) {
        const int64_t i0 = base + (int64_t)threadIdx.x * IG_PER_THREAD;
        uint32_t k[IG_PER_THREAD];
        if (i0 + IG_PER_THREAD <= end) {
            const uint4* v = reinterpret_cast<const uint4*>(keys + i0);  // i0 is a multiple of 16
#pragma unroll
            for (int q = 0; q < IG_PER_THREAD / kPerVec; ++q) {
                const uint4 x = __ldcs(v + q);
                const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < kPerVec; ++e)
                    k[kPerVec * q + e] = sizeof(KT) == 4 ? w4[e] : (w4[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
            }
        } else {
#pragma unroll
            for (int r = 0; r < IG_PER_THREAD; ++r) k[r] = i0 + r < end ? (uint32_t)keys[i0 + r] : kNoDigit;
        }
        uint32_t cur = kNoDigit, run = 0;
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const uint32_t d = k[r] == kNoDigit ? kNoDigit : (k[r] & dmask);
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
template <int THREADS, typename T>
__device__ void scan_bins(const T* cnt, T* start, int bins, uint32_t* wtot) {
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
            start[b0 + k] = (T)run;
            run += cnt[b0 + k];
        }
}

// A sample between passes: one 16-byte record {TOD value, sample index,
// cos, sin} (one store stream instead of three: the scatter's short digit
// runs then fill whole lines, which measured twice as fast).  The keys travel
// as their own stream, so the first word of the record is free for the TOD
// sample when one is sorted along (else it is unused).  A pass sorts on the
// low `bits` bits of its key and stores the key shifted past them, so every
// pass reads its digit from the low bits, and the stored keys are 16-bit
// when what is left of the pixel index fits (2 bytes a sample instead of 4,
// written once and read once).
struct ScatterArgs {
    const uint4* rec_in;      // records of the previous pass, or null on the first pass:
                              //   then the sample index itself, the trig pairs and the TOD in time order
    const void* keys_in;      // keys in this pass's input order: the validated pixel indices (int32) on
                              //   the first pass, else the stored keys (KT)
    const float2* hi_in;      // first pass: the trig pairs in time order; or, with c_in and s_in,
    const float* c_in;        //   the caller's cos 2psi and sin 2psi (16-byte aligned), which the
    const float* s_in;        //   pass checks (|.| <= 1) and writes as pairs to hi_t_out in time order
    float2* hi_t_out;         //   (null: the time-ordered pairs are deferred)
    unsigned long long* bad;  //   (samples with a bad pair are counted here)
    const float* tod_in;      // first pass: the TOD in time order, or null
    const float2* lo_in;      // lo halves of the trig pairs in this pass's input order, or null
    int64_t n;
    int64_t range;
    int bits, bins, G;
    const uint32_t* offs;  // [bins][G] exclusive digit-major scan of the counts
    uint4* rec_out;        // intermediate passes: records, and the keys alone for the next pass
    void* keys_out;        //   (KT, shifted right by bits)
    uint32_t* perm_out;    // last pass: sample indices (perm) and trig pairs of the kept samples
    float2* hi_out;
    float* tod_out;        // last pass: the TOD of the kept samples in sorted order, or null
    float2* lo_out;        // every pass with lo_in: the lo halves in this pass's output order
    uint32_t nvalid;       // last pass: the kept samples; flagged ones (key npix, the largest) sort to
                           //   positions >= nvalid and get no entry
    uint32_t flag_key;     // first pass: keys_in are pixel indices, -1 maps to flag_key (= npix)
    unsigned long long* err;  // set to 1 if a wait for a bulk copy gave up
};

// Shared memory of one scatter block: the tile's payload window (records,
// or trig pairs + TOD values on the first pass), its keys (input order, then
// the lane-mask tables of the ranking), the tile position of each staged
// sample, the per-warp digit counters (whose region then holds the keys
// staged in digit order), and per digit the running global offset and the
// tile's count and start.
inline size_t scatter_smem(int bins) {
    const size_t tile = SC_TILE;
    return 16 * tile + 4 * tile + 2 * tile + std::max(2 * (size_t)SC_WARPS * bins, 4 * tile) + 4 * (size_t)bins +
           2 * 2 * (size_t)bins;
}

// Bulk copies global -> shared memory by the TMA engine, completed on an
// mbarrier (transaction bytes), and bounded waits on it.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Polls for the completion of the barrier phase with this parity; false if
// it did not complete within the poll limit (each poll may suspend the
// thread for a short, hardware-defined time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One stable scatter pass over the block's range (see the file comment).
// Per tile, one thread starts two bulk copies into shared memory: the keys
// and the payload window (the intermediate records, or on the first pass
// the time-ordered trig pairs and TOD values).  The keys are ranked as soon
// as they arrive, while the window is still on its way; each sample's key
// and tile position are then staged in digit order, and the write-out reads
// the payload of a staged sample from the window in shared memory and
// stores the digit runs at their running global offsets.
template <bool LAST, bool FIRST, typename KT, bool TRIG2>
__global__ void __launch_bounds__(SC_THREADS, SC_MIN_BLOCKS) rs_scatter_kernel(ScatterArgs a) {
    using KI = typename std::conditional<FIRST, uint32_t, KT>::type;  // the input keys' type
    constexpr int kKeysPer16 = 16 / (int)sizeof(KI);
    extern __shared__ __align__(128) unsigned char smem[];
    uint4* s_rec = reinterpret_cast<uint4*>(smem);                          // window: records
    float2* s_hi = reinterpret_cast<float2*>(smem);                         // window, first pass: trig pairs
    float* s_c = reinterpret_cast<float*>(smem);                            //   or (TRIG2) cos and sin
    float* s_s = reinterpret_cast<float*>(smem + 4 * SC_TILE);
    float* s_tod = reinterpret_cast<float*>(smem + 8 * SC_TILE);            //   and TOD values
    KI* s_keys = reinterpret_cast<KI*>(smem + 16 * SC_TILE);                // keys
    uint16_t* s_src = reinterpret_cast<uint16_t*>(smem + 20 * SC_TILE);     // tile position of a staged sample
    uint16_t* wcnt = reinterpret_cast<uint16_t*>(smem + 22 * SC_TILE);      // [warp][digit]
    uint32_t* s_stk = reinterpret_cast<uint32_t*>(wcnt);                   // staged keys (after the counters' use)
    uint32_t* run_base = reinterpret_cast<uint32_t*>(
        smem + 22 * SC_TILE + (2 * SC_WARPS * a.bins > 4 * SC_TILE ? 2 * SC_WARPS * a.bins : 4 * SC_TILE));  // next global position per digit
    uint16_t* tcnt = reinterpret_cast<uint16_t*>(run_base + a.bins);       // tile count per digit
    uint16_t* tstart = tcnt + a.bins;                                       // tile-local start per digit
    __shared__ uint32_t wtot[SC_WARPS];
    __shared__ __align__(8) uint64_t bar[3];  // [0] keys, [1] window: first part, [2] window: second part
    // lane-mask tables of the ranking, outside the payload window, so that
    // the whole window of the next tile is copied in while the current one
    // is written out: on the first pass, whose window (trig pairs and TOD
    // values) leaves its last quarter free, 4 KB a warp in that quarter and
    // the keys' buffer (the keys are in registers by then); on later passes,
    // whose records fill the window, 2 KB a warp in the keys' buffer alone
    constexpr int kTblEntries = FIRST ? 512 : 256;  // entries of each of a warp's two tables
    uint32_t* s_tbl = reinterpret_cast<uint32_t*>(smem + (FIRST ? 12 : 16) * SC_TILE);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int bins = a.bins;
    const uint32_t dmask = (uint32_t)bins - 1u;
    const int64_t begin = range_begin(a.range);
    const int64_t end = begin + a.range < a.n ? begin + a.range : a.n;
    const uint64_t pol = l2_keep_policy();
    // a caller's TOD array may start off a 16-byte boundary: then it is read
    // with plain loads
    const bool tod_bulk = FIRST && a.tod_in && (reinterpret_cast<uintptr_t>(a.tod_in) & 15u) == 0;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        mbar_init(&bar[2]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int d = threadIdx.x; d < bins; d += SC_THREADS) {
        run_base[d] = a.offs[(int64_t)d * a.G + blockIdx.x];
#pragma unroll
        for (int q = 0; q < SC_WARPS; ++q) wcnt[q * bins + d] = 0;
    }
    __syncthreads();

    // One thread starts the copies of the tile at `base`, keys and window
    // separately: whole 16-byte units (the rest of a ragged last tile is
    // loaded by the threads).  The fence orders the block's earlier accesses
    // of the buffer (made visible by a barrier) before the copy's writes.
    const KI* keys_in = static_cast<const KI*>(a.keys_in);
    auto issue_keys = [&](int64_t base, int cnt) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t kbytes = (uint32_t)(cnt & ~(kKeysPer16 - 1)) * (uint32_t)sizeof(KI);
        mbar_arrive_expect(&bar[0], kbytes);
        if (kbytes) bulk_g2s(s_keys, keys_in + base, kbytes, &bar[0]);
    };
    // the window's first part: records of the tile's first half, or the
    // trig pairs (or cos and sin)
    auto issue_win1 = [&](int64_t base, int cnt) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!FIRST) {
            const uint32_t n1 = cnt < SC_TILE / 2 ? (uint32_t)cnt : SC_TILE / 2;
            mbar_arrive_expect(&bar[1], n1 * 16u);
            bulk_g2s(s_rec, a.rec_in + base, n1 * 16u, &bar[1]);
        } else if (TRIG2) {
            const uint32_t cbytes = (uint32_t)(cnt & ~3) * 4u;
            mbar_arrive_expect(&bar[1], 2u * cbytes);
            if (cbytes) {
                bulk_g2s(s_c, a.c_in + base, cbytes, &bar[1]);
                bulk_g2s(s_s, a.s_in + base, cbytes, &bar[1]);
            }
        } else {
            const uint32_t hbytes = (uint32_t)(cnt & ~1) * 8u;
            mbar_arrive_expect(&bar[1], hbytes);
            if (hbytes) bulk_g2s(s_hi, a.hi_in + base, hbytes, &bar[1]);
        }
    };
    // the second part: records of the second half, or the TOD values
    auto issue_win2 = [&](int64_t base, int cnt) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!FIRST) {
            const uint32_t n2 = cnt > SC_TILE / 2 ? (uint32_t)(cnt - SC_TILE / 2) : 0u;
            mbar_arrive_expect(&bar[2], n2 * 16u);
            if (n2) bulk_g2s(s_rec + SC_TILE / 2, a.rec_in + base + SC_TILE / 2, n2 * 16u, &bar[2]);
        } else {
            const uint32_t tbytes = tod_bulk ? (uint32_t)(cnt & ~3) * 4u : 0u;
            mbar_arrive_expect(&bar[2], tbytes);
            if (tbytes) bulk_g2s(s_tod, a.tod_in + base, tbytes, &bar[2]);
        }
    };
    // Gives up the block after a failed wait: flags the error, waits (again
    // bounded) for the copies still in flight so that none lands after the
    // block has exited, and returns true.
    auto give_up = [&](bool failed, uint32_t key_parity, uint32_t win_parity, bool win2_issued) {
        if (!__syncthreads_or(failed)) return false;
        if (threadIdx.x == 0) {
            atomicExch(a.err, 1ull);
            mbar_wait(&bar[0], key_parity);
            mbar_wait(&bar[1], win_parity);
            if (win2_issued) mbar_wait(&bar[2], win_parity);
        }
        return true;
    };

    if (threadIdx.x == 0 && begin < end) {
        issue_keys(begin, (int)(end - begin < SC_TILE ? end - begin : SC_TILE));
        issue_win1(begin, (int)(end - begin < SC_TILE ? end - begin : SC_TILE));
        issue_win2(begin, (int)(end - begin < SC_TILE ? end - begin : SC_TILE));
    }
    uint32_t parity = 0;
    uint32_t nbad = 0;
    for (int64_t base = begin; base < end; base += SC_TILE, parity ^= 1u) {
        const int cnt = (int)(end - base < SC_TILE ? end - base : SC_TILE);
        // the ragged end of the last tile, with plain loads
        for (int j = (cnt & ~(kKeysPer16 - 1)) + threadIdx.x; j < cnt; j += SC_THREADS) s_keys[j] = keys_in[base + j];
        if (FIRST && !TRIG2 && (cnt & 1) && threadIdx.x == 0) s_hi[cnt - 1] = a.hi_in[base + cnt - 1];
        if (TRIG2)
            for (int j = (cnt & ~3) + threadIdx.x; j < cnt; j += SC_THREADS) {
                s_c[j] = a.c_in[base + j];
                s_s[j] = a.s_in[base + j];
            }
        if (give_up(!mbar_wait(&bar[0], parity), parity, parity, true)) return;
        __syncthreads();  // the plain-loaded keys too
        uint32_t key[IG_PER_THREAD], rank[IG_PER_THREAD];
        // 1. the warp's 512 consecutive keys, 32 per round
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const int j = w * IG_WARP_SPAN + r * 32 + lane;
            key[r] = j < cnt ? (FIRST ? pixel_key(s_keys[j], a.flag_key) : (uint32_t)s_keys[j]) : 0u;
        }
        // 2. stable rank within the warp, two rounds at a time.  The lanes
        //    of a round that hold the same digit are found through a table of
        //    lane masks in shared memory (each lane ORs its bit into its
        //    digit's entry and reads the entry back; the lanes clear it
        //    afterwards): a warp-wide match instruction costs ~60 cycles of
        //    the SM here, these shared-memory operations ~2.  Rounds A and B
        //    (B's samples after A's) have a table each (512 entries on the
        //    first pass, 256 later: 4 or 2 KB a warp); digits wider than a
        //    table index it with their low bits and a vote on each higher
        //    bit splits the entries.  Every lane
        //    reads its digit's warp counter c before the pair: a sample of A
        //    ranks at c + (A lanes below it with its digit), one of B at c +
        //    (A lanes with its digit, read from A's table at B's digit) + (B
        //    lanes below it); the lowest lane of each digit adds the pair's
        //    count.  Ranks follow the input order (a stable sort), and the
        //    pair takes three shared-memory round trips where two single
        //    rounds took six.  The 16-bit counters are stored as halves (a
        //    warp counts at most 512 samples a digit); two leaders never
        //    store the same counter in one pair.
        __syncthreads();  // every warp has its keys before the tables overwrite them
        {
            uint4* z = reinterpret_cast<uint4*>(s_tbl);
            for (int i = threadIdx.x; i < SC_WARPS * 2 * kTblEntries / 4; i += SC_THREADS)
                z[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        {
            uint16_t* wc = wcnt + w * bins;
            uint32_t* tA = s_tbl + w * 2 * kTblEntries;
            uint32_t* tB = tA + kTblEntries;
            // digits wider than a table: a vote on each bit above it splits
            // the entries (one bit on the first pass, up to two later)
            constexpr int kB0 = FIRST ? 9 : 8;
            const int nvote = bins <= kTblEntries ? 0 : (bins <= 2 * kTblEntries ? 1 : 2);
            const uint32_t tmask = (uint32_t)(bins < kTblEntries ? bins : kTblEntries) - 1u;
            const unsigned me = 1u << lane;
#pragma unroll
            for (int r = 0; r < IG_PER_THREAD; r += 2) {
                const int jA = w * IG_WARP_SPAN + r * 32 + lane;
                const bool vA = jA < cnt, vB = jA + 32 < cnt;
                const uint32_t dA = key[r] & dmask, dB = key[r + 1] & dmask;
                const uint32_t iA = dA & tmask, iB = dB & tmask;
                if (vA) atomicOr(tA + iA, me);
                if (vB) atomicOr(tB + iB, me);
                const unsigned hA0 = nvote > 0 ? __ballot_sync(0xffffffffu, vA && ((dA >> kB0) & 1u)) : 0u;
                const unsigned hB0 = nvote > 0 ? __ballot_sync(0xffffffffu, vB && ((dB >> kB0) & 1u)) : 0u;
                const unsigned hA1 = nvote > 1 ? __ballot_sync(0xffffffffu, vA && ((dA >> (kB0 + 1)) & 1u)) : 0u;
                const unsigned hB1 = nvote > 1 ? __ballot_sync(0xffffffffu, vB && ((dB >> (kB0 + 1)) & 1u)) : 0u;
                __syncwarp();
                unsigned pA = tA[iA], pB = tB[iB];
                unsigned xAB = tA[iB], xBA = tB[iA];  // A lanes on B's entry, B lanes on A's entry
                const uint32_t cA = wc[dA], cB = wc[dB];
                __syncwarp();
                if (nvote > 0) {  // keep the lanes whose bits above the table match the digit's
                    auto filt = [&](uint32_t d, unsigned h0, unsigned h1) {
                        unsigned f = ((d >> kB0) & 1u) ? h0 : ~h0;
                        if (nvote > 1) f &= ((d >> (kB0 + 1)) & 1u) ? h1 : ~h1;
                        return f;
                    };
                    pA &= filt(dA, hA0, hA1);
                    xAB &= filt(dB, hA0, hA1);
                    pB &= filt(dB, hB0, hB1);
                    xBA &= filt(dA, hB0, hB1);
                }
                if (vA) tA[iA] = 0u;
                if (vB) tB[iB] = 0u;
                const uint32_t nAB = (uint32_t)__popc(xAB), nBA = (uint32_t)__popc(xBA);
                rank[r] = cA + (uint32_t)__popc(pA & lt_mask);
                rank[r + 1] = cB + nAB + (uint32_t)__popc(pB & lt_mask);
                if (vA && lane == __ffs(pA) - 1) wc[dA] = (uint16_t)(cA + (uint32_t)__popc(pA) + nBA);
                if (vB && nAB == 0u && lane == __ffs(pB) - 1) wc[dB] = (uint16_t)(cB + (uint32_t)__popc(pB));
                __syncwarp();  // entries clear and counters stored before the next pair
            }
        }
        __syncthreads();
        // given cos/sin (TRIG2) and not deferred: the tile's time-ordered
        // pairs, written while the digits are counted and staged (in the
        // write-out these stores measured 3k cycles a tile)
        if (TRIG2 && a.hi_t_out) {
            if (give_up(!mbar_wait(&bar[1], parity), parity, parity, true)) return;
            for (int j = threadIdx.x; j < cnt; j += SC_THREADS) __stcs(a.hi_t_out + base + j, make_float2(s_c[j], s_s[j]));
        }
        // 3. per digit: the tile count (the warps' counts summed), the scan
        //    over digits, then each warp's start of each digit in the tile
        //    (the digit's start + the counts of the warps before it) written
        //    over its counter.  Two 16-bit digits a 32-bit word: every value
        //    is below 2^13, so the halves add without carries.  run_base
        //    becomes the offset of the tile's digit-ordered position j to its
        //    global position: g = run_base[d] + j.
        {
            uint32_t* wc32 = reinterpret_cast<uint32_t*>(wcnt);
            uint32_t* tcnt32 = reinterpret_cast<uint32_t*>(tcnt);
            const uint32_t* tstart32 = reinterpret_cast<const uint32_t*>(tstart);
            const int hb = bins >> 1;
            for (int t = threadIdx.x; t < hb; t += SC_THREADS) {
                uint32_t sum = 0;
#pragma unroll
                for (int q = 0; q < SC_WARPS; ++q) sum += wc32[q * hb + t];
                tcnt32[t] = sum;
            }
            __syncthreads();
            scan_bins<SC_THREADS>(tcnt, tstart, bins, wtot);
            __syncthreads();
            for (int t = threadIdx.x; t < hb; t += SC_THREADS) {
                uint32_t run = tstart32[t];
#pragma unroll
                for (int q = 0; q < SC_WARPS; ++q) {
                    const uint32_t c = wc32[q * hb + t];
                    wc32[q * hb + t] = run;
                    run += c;
                }
                run_base[2 * t] -= tstart[2 * t];
                run_base[2 * t + 1] -= tstart[2 * t + 1];
            }
            __syncthreads();
        }
        // 4. stage keys and tile positions in digit order: the positions
        //    first (they read the counters), then the keys into the
        //    counters' region; the keys' buffer is free from here on, so the
        //    next tile's keys start arriving during the write-out
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) rank[r] += wcnt[w * bins + (key[r] & dmask)];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < IG_PER_THREAD; ++r) {
            const int j = w * IG_WARP_SPAN + r * 32 + lane;
            if (j < cnt) {
                if (LAST) {  // the last pass needs only the digit: digit and position in one word
                    s_stk[rank[r]] = ((key[r] & dmask) << 13) | (uint32_t)j;
                } else {
                    s_stk[rank[r]] = key[r];
                    s_src[rank[r]] = (uint16_t)j;
                }
            }
        }
        // a TOD that is not bulk-copied (off a 16-byte boundary, or the
        // ragged end), with plain loads
        if (FIRST && a.tod_in)
            for (int j = (tod_bulk ? (cnt & ~3) : 0) + threadIdx.x; j < cnt; j += SC_THREADS) s_tod[j] = a.tod_in[base + j];
        __syncthreads();
        if (threadIdx.x == 0 && base + SC_TILE < end)
            issue_keys(base + SC_TILE, (int)(end - base - SC_TILE < SC_TILE ? end - base - SC_TILE : SC_TILE));
        // (the next tile's keys may be on their way: the other key phase)
        {
            const uint32_t kp = base + SC_TILE < end ? parity ^ 1u : parity;
            if (give_up(!mbar_wait(&bar[1], parity), kp, parity, true)) return;
            if (give_up(!mbar_wait(&bar[2], parity), kp, parity, true)) return;
        }
        // 5. each digit's run goes to its running global offset, the rest of
        //    each sample from the window in shared memory
        for (int j = threadIdx.x; j < cnt; j += SC_THREADS) {
            const uint32_t k = s_stk[j];
            const uint32_t src = LAST ? (k & 8191u) : s_src[j];
            const uint32_t d = LAST ? (k >> 13) : (k & dmask);
            const uint32_t g = run_base[d] + (uint32_t)j;
            uint4 rr;
            if (!FIRST) {
                rr = s_rec[src];
            } else {
                const float2 h = TRIG2 ? make_float2(s_c[src], s_s[src]) : s_hi[src];
                if (TRIG2) nbad += !(fabsf(h.x) <= 1.0f && fabsf(h.y) <= 1.0f);  // each sample once; NaN counts
                const float dv = a.tod_in ? s_tod[src] : 0.f;
                rr = make_uint4(__float_as_uint(dv), (uint32_t)(base + src), __float_as_uint(h.x), __float_as_uint(h.y));
            }
            if (!LAST) {
                st_keep(a.rec_out + g, rr, pol);
                st_keep(static_cast<KT*>(a.keys_out) + g, (KT)(k >> a.bits), pol);
                if (a.lo_in) st_keep(a.lo_out + g, a.lo_in[base + src], pol);
            } else if (g < a.nvalid) {
                st_keep(a.perm_out + g, rr.y, pol);
                st_keep(a.hi_out + g, make_float2(__uint_as_float(rr.z), __uint_as_float(rr.w)), pol);
                if (a.tod_out) st_keep(reinterpret_cast<uint32_t*>(a.tod_out) + g, rr.x, pol);
                if (a.lo_in) st_keep(a.lo_out + g, a.lo_in[base + src], pol);
            }
        }
        __syncthreads();
        // 6. advance the running offsets, clear the warp counters, start the
        //    next tile's window
        for (int d = threadIdx.x; d < bins; d += SC_THREADS) run_base[d] += tstart[d] + tcnt[d];
        {
            uint4* z = reinterpret_cast<uint4*>(wcnt);
            for (int i = threadIdx.x; i < SC_WARPS * bins / 8; i += SC_THREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (threadIdx.x == 0 && base + SC_TILE < end) {
            issue_win1(base + SC_TILE, (int)(end - base - SC_TILE < SC_TILE ? end - base - SC_TILE : SC_TILE));
            issue_win2(base + SC_TILE, (int)(end - base - SC_TILE < SC_TILE ? end - base - SC_TILE : SC_TILE));
        }
        __syncthreads();
    }
    if (TRIG2) {
        nbad = __reduce_add_sync(0xffffffffu, nbad);
        if (lane == 0 && nbad) atomicAdd(a.bad, (unsigned long long)nbad);
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


using ScatterFn = void (*)(ScatterArgs);
ScatterFn scatter_fn(bool last, bool first, bool key16, bool trig2) {
    if (first && trig2)
        return last ? rs_scatter_kernel<true, true, uint32_t, true>
                    : (key16 ? rs_scatter_kernel<false, true, uint16_t, true>
                             : rs_scatter_kernel<false, true, uint32_t, true>);
    if (first)
        return last ? rs_scatter_kernel<true, true, uint32_t, false>
                    : (key16 ? rs_scatter_kernel<false, true, uint16_t, false>
                             : rs_scatter_kernel<false, true, uint32_t, false>);
    if (last)
        return key16 ? rs_scatter_kernel<true, false, uint16_t, false> : rs_scatter_kernel<true, false, uint32_t, false>;
    return key16 ? rs_scatter_kernel<false, false, uint16_t, false> : rs_scatter_kernel<false, false, uint32_t, false>;
}

SortPlan plan_sort(const bm_context* ctx, int64_t n, int64_t npix) {
    SortPlan sp;
    int nbits = 1;
    while (((int64_t)1 << nbits) <= npix) ++nbits;  // the flagged key npix must fit too
    sp.passes = (nbits + RS_MAX_BITS - 1) / RS_MAX_BITS;
    sp.bits = (nbits + sp.passes - 1) / sp.passes;
    sp.bins = 1 << sp.bits;
    sp.key16 = nbits - sp.bits <= 16;
    const size_t smem = scatter_smem(sp.bins);
    for (int pass = 0; pass < sp.passes; ++pass)
        for (bool trig2 : {false, true})
            ensure_smem_limit(reinterpret_cast<const void*>(scatter_fn(pass + 1 == sp.passes, pass == 0, sp.key16, trig2)),
                              smem);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_hist_kernel<uint16_t>), sizeof(uint32_t) * IG_WARPS * sp.bins);
    ensure_smem_limit(reinterpret_cast<const void*>(rs_hist_kernel<uint32_t>), sizeof(uint32_t) * IG_WARPS * sp.bins);
    for (const void* k : {reinterpret_cast<const void*>(validate_kernel<kTrigIn, true>),
                          reinterpret_cast<const void*>(validate_kernel<kPixOnly, true>),
                          reinterpret_cast<const void*>(validate_kernel<kPsi64, true>),
                          reinterpret_cast<const void*>(validate_kernel<kPsi32, true>),
                          reinterpret_cast<const void*>(validate_kernel<kHwp, true>)})
        ensure_smem_limit(k, sizeof(uint32_t) * kVHist * sp.bins);
    int per_sm = blocks_per_sm(reinterpret_cast<const void*>(scatter_fn(true, sp.passes == 1, sp.key16, false)),
                               SC_THREADS, smem);
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
            const float* sin2psi, const float* tod, bool tod_on_host, const HwpModel* hwp) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    ScopedTimer timer(ctx, "ingest");
    const int64_t n = p->nsamples, npix = p->npix;
    const bool exact_trig = cos2psi != nullptr;  // FP32 trig given: it defines the operator, no lo part
    const bool has_lo = !exact_trig;
    // cos/sin in device memory at 16-byte boundaries: the first sort pass
    // bulk-copies them itself, checks them and writes the time-ordered
    // pairs; the validation then reads the pixels alone
    auto in_device_memory = [](const void* ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice;
    };
    const bool trig2 = exact_trig && !hwp &&
                       ((reinterpret_cast<uintptr_t>(cos2psi) | reinterpret_cast<uintptr_t>(sin2psi)) & 15u) == 0 &&
                       in_device_memory(cos2psi) && in_device_memory(sin2psi);
    const SortPlan sp = plan_sort(ctx, n, npix);
    const int threads = 256;

    // A pointing that carries a TOD is made for white-noise solves, which
    // read only the pixel-sorted pairs: given cos/sin, its time-ordered pairs
    // (8 bytes a sample) are built from the sorted ones by the first
    // time-ordered operator that needs them (time_trig).
    const bool defer_t = trig2 && tod != nullptr;
    // likewise its time-ordered pixel copy, when the caller's pixels are in
    // device memory at a 16-byte boundary: the first sort pass and the CSR
    // offsets read them there, and time_pix builds the copy on first use
    const bool defer_pix = defer_t && (reinterpret_cast<uintptr_t>(pix) & 15u) == 0 && in_device_memory(pix);
    if (!defer_pix) p->pix.alloc(n);
    if (!defer_t) p->cs_hi_t.alloc(n);
    p->trig_t_deferred = defer_t;
    p->pix_deferred = defer_pix;
    if (has_lo) p->cs_lo_t.alloc(n);
    DevBuf<float> tod_copy;  // a host TOD, copied by the validation pass
    if (tod && tod_on_host) tod_copy.alloc(n);
    const float* tod_t = tod_on_host ? tod_copy.get() : tod;
    // invalid samples, flagged samples, a scatter wait that gave up, samples
    // with a bad cos/sin pair found by the first sort pass
    DevBuf<unsigned long long> counters(4);
    BM_CUDA(cudaMemsetAsync(counters.get(), 0, 4 * sizeof(unsigned long long), s));
    // digit counts of every sort pass; the first pass's come from the validation
    DevBuf<uint32_t> hist((size_t)sp.bins * sp.grid);
    {
        ScopedTimer vt(ctx, "ingest_validate");
        BM_CUDA(cudaMemsetAsync(hist.get(), 0, sizeof(uint32_t) * (size_t)sp.bins * sp.grid, s));
        auto kern = trig2        ? validate_kernel<kPixOnly, true>
                    : exact_trig ? validate_kernel<kTrigIn, true>
                    : hwp      ? validate_kernel<kHwp, true>
                               : (psi_dtype == BM_F64 ? validate_kernel<kPsi64, true> : validate_kernel<kPsi32, true>);
        constexpr int kSub = 2;  // two blocks a range: eight resident blocks per SM
        kern<<<sp.grid * kSub, IG_THREADS, sizeof(uint32_t) * kVHist * sp.bins, s>>>(
            pix, psi, cos2psi, sin2psi, n, npix, defer_pix ? nullptr : p->pix.get(), p->cs_hi_t.get(), p->cs_lo_t.get(),
            tod_on_host ? tod : nullptr, tod_copy.get(), counters.get(), sp.range, kSub, sp.bins, sp.grid,
            hist.get(), hwp ? *hwp : HwpModel{});
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
    // of the trig pairs when the angles were given): context workspaces, kept
    // for the next ingest, so that these large transient buffers do not
    // fragment the device memory pool the handles allocate from.
    uint4 *rec_a = nullptr, *rec_b = nullptr;
    void *keys_a = nullptr, *keys_b = nullptr;
    float2 *lo_a = nullptr, *lo_b = nullptr;
    const size_t key_bytes = sp.key16 ? 2 : 4;
    if (sp.passes > 1) {
        rec_a = workspace_as<uint4>(ctx, "ingest_rec_a", n);
        keys_a = workspace(ctx, "ingest_keys_a", key_bytes * n);
        if (has_lo) lo_a = workspace_as<float2>(ctx, "ingest_lo_a", n);
    }
    if (sp.passes > 2) {
        rec_b = workspace_as<uint4>(ctx, "ingest_rec_b", n);
        keys_b = workspace(ctx, "ingest_keys_b", key_bytes * n);
        if (has_lo) lo_b = workspace_as<float2>(ctx, "ingest_lo_b", n);
    }
    // the first pass reads its keys from the validated pixel indices
    const int32_t* pix_keys = defer_pix ? pix : p->pix.get();  // validated: every index in [-1, npix)
    const void* kin = pix_keys;
    void* kout = keys_a;
    const size_t smem = scatter_smem(sp.bins);
    const uint4* rin = nullptr;  // the first pass reads keys, indices and trig in time order
    uint4* rout = rec_a;
    const float2* lin = has_lo ? p->cs_lo_t.get() : nullptr;
    float2* lout = lo_a;
    for (int pass = 0; pass < sp.passes; ++pass) {
        if (pass > 0) {
            ScopedTimer ht(ctx, "ingest_hist");
            const size_t hsm = sizeof(uint32_t) * IG_WARPS * sp.bins;
            if (sp.key16)
                rs_hist_kernel<uint16_t><<<sp.grid, IG_THREADS, hsm, s>>>(static_cast<const uint16_t*>(kin), n,
                                                                          sp.range, sp.bins, sp.grid, hist.get());
            else
                rs_hist_kernel<uint32_t><<<sp.grid, IG_THREADS, hsm, s>>>(static_cast<const uint32_t*>(kin), n,
                                                                          sp.range, sp.bins, sp.grid, hist.get());
            BM_LAUNCH_CHECK();
        }
        exclusive_scan_u32(hist.get(), hist.get(), (int64_t)sp.bins * sp.grid, s);
        ScatterArgs a{};
        a.rec_in = rin;
        a.keys_in = kin;
        a.hi_in = p->cs_hi_t.get();
        const bool pass_trig2 = trig2 && pass == 0;
        if (pass_trig2) {
            a.c_in = cos2psi;
            a.s_in = sin2psi;
            a.hi_t_out = defer_t ? nullptr : p->cs_hi_t.get();
            a.bad = counters.get() + 3;
        }
        a.tod_in = pass == 0 ? tod_t : nullptr;
        a.lo_in = lin;
        a.n = n;
        a.range = sp.range;
        a.bits = sp.bits;
        a.bins = sp.bins;
        a.G = sp.grid;
        a.offs = hist.get();
        a.flag_key = (uint32_t)npix;
        a.err = counters.get() + 2;
        ScopedTimer st(ctx, "ingest_scatter");
        if (pass + 1 < sp.passes) {
            a.rec_out = rout;
            a.keys_out = kout;
            a.lo_out = lout;
            scatter_fn(false, pass == 0, sp.key16, pass_trig2)<<<sp.grid, SC_THREADS, smem, s>>>(a);
            BM_LAUNCH_CHECK();
            kin = kout;
            kout = (kout == keys_a) ? keys_b : keys_a;
            rin = rout;
            rout = (rout == rec_a) ? rec_b : rec_a;
            lin = has_lo ? lout : nullptr;
            lout = (lout == lo_a) ? lo_b : lo_a;
        } else {
            a.perm_out = p->perm.get();
            a.hi_out = p->cs_hi_s.get();
            a.tod_out = tod ? p->tod_s.get() : nullptr;
            a.lo_out = has_lo ? p->cs_lo_s.get() : nullptr;
            a.nvalid = (uint32_t)nvalid;
            scatter_fn(true, pass == 0, sp.key16, pass_trig2)<<<sp.grid, SC_THREADS, smem, s>>>(a);
            BM_LAUNCH_CHECK();
        }
    }
    p->off.alloc(npix + 1);
    p->hits.alloc(npix);
    const int pgrid = grid_for(ctx, (npix + 1 + threads - 1) / threads, 16);
    lower_bound_kernel<<<pgrid, threads, 0, s>>>(p->perm.get(), pix_keys, nvalid, npix, p->off.get());
    BM_LAUNCH_CHECK();
    hits_kernel<<<pgrid, threads, 0, s>>>(p->off.get(), npix, p->hits.get());
    BM_LAUNCH_CHECK();
    unsigned long long h_err[2] = {0, 0};
    BM_CUDA(cudaMemcpyAsync(h_err, counters.get() + 2, sizeof(h_err), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    if (h_err[0]) {
        set_error("the pixel sort gave up waiting for a bulk copy into shared memory");
        throw Error{BM_ERR_TIMEOUT};
    }
    BM_REQUIRE(h_err[1] == 0, "%llu samples have a pixel index outside [-1, %lld) or a bad angle / trig value",
               h_err[1], (long long)npix);
}

namespace {
__global__ void time_trig_kernel(const uint32_t* __restrict__ perm, const float2* __restrict__ hi_s, int64_t nvalid,
                                 float2* __restrict__ hi_t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvalid; i += (int64_t)gridDim.x * blockDim.x)
        hi_t[perm[i]] = hi_s[i];
}
}  // namespace

namespace {
// pix_t[perm[i]] = q for every sorted position i of pixel q (one thread a pixel)
__global__ void time_pix_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ perm, int64_t npix,
                                int32_t* __restrict__ pix_t) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x)
        for (int64_t i = off[q]; i < off[q + 1]; ++i) pix_t[perm[i]] = (int32_t)q;
}
}  // namespace

const int32_t* time_pix(const bm_pointing* pc) {
    bm_pointing* p = const_cast<bm_pointing*>(pc);  // a lazily filled part of the handle
    if (p->pix_deferred) {
        bm_context* ctx = p->ctx;
        cudaStream_t s = ctx->stream;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        BM_CUDA(cudaStreamIsCapturing(s, &cs));
        BM_REQUIRE(cs == cudaStreamCaptureStatusNone,
                   "the time-ordered pixels of a pointing that carries a TOD are built on first use, "
                   "which a stream capture cannot hold: make one time-ordered call before capturing");
        ScopedTimer timer(ctx, "time_pix");
        p->pix.alloc(p->nsamples);
        BM_CUDA(cudaMemsetAsync(p->pix.get(), 0xFF, sizeof(int32_t) * (size_t)p->nsamples, s));  // -1: flagged
        time_pix_kernel<<<grid_for(ctx, (p->npix + 255) / 256, 16), 256, 0, s>>>(p->off.get(), p->perm.get(), p->npix,
                                                                                 p->pix.get());
        BM_LAUNCH_CHECK();
        p->pix_deferred = false;
    }
    return p->pix.get();
}

const float2* time_trig(bm_pointing* p) {
    if (p->trig_t_deferred) {
        bm_context* ctx = p->ctx;
        cudaStream_t s = ctx->stream;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        BM_CUDA(cudaStreamIsCapturing(s, &cs));
        BM_REQUIRE(cs == cudaStreamCaptureStatusNone,
                   "the time-ordered trig pairs of a pointing that carries a TOD are built on first use, "
                   "which a stream capture cannot hold: make one time-ordered call before capturing");
        ScopedTimer timer(ctx, "time_trig");
        p->cs_hi_t.alloc(p->nsamples);
        BM_CUDA(cudaMemsetAsync(p->cs_hi_t.get(), 0, sizeof(float2) * (size_t)p->nsamples, s));
        if (p->nvalid > 0) {
            time_trig_kernel<<<grid_for(ctx, (p->nvalid + 255) / 256, 16), 256, 0, s>>>(p->perm.get(), p->cs_hi_s.get(),
                                                                                        p->nvalid, p->cs_hi_t.get());
            BM_LAUNCH_CHECK();
        }
        p->trig_t_deferred = false;
    }
    return p->cs_hi_t.get();
}

}  // namespace bm
