// The operator A = P^T N^-1 P (paper Eq. 6) and the right-hand side
// b = P^T N^-1 d, plus the individual operators P, P^T and N^-1.
//
// White noise (N^-1 diagonal, the paper's InvNoiseCovUnCorr): the matvec
// streams the samples in pixel-sorted order.  One warp takes one work item
// (<= kItemMax consecutive samples of one kept pixel p): it gathers
// y_t = v_t . x_p, weights it, and accumulates w_t y_t v_t; the item partial
// is written in FP64 and a per-pixel pass sums a pixel's items in item order.
// No atomics, so every result is bitwise reproducible.
//   FP32 form: reads the weighted stream u_t = sqrt(w) (cos 2psi, sin 2psi)
//              (8 B/sample; sqrt(w) = |u_t|), FP32 products, FP32 lane sums,
//              FP64 warp sums.
//   FP64 form: reads perm, the FP32 (hi, lo) trig pairs and w_d (20 B/sample),
//              FP64 products and sums.
//
// Toeplitz noise: time-ordered tiles of each chunk gather y = P x (masked and
// flagged samples give 0), apply the banded filter from a shared-memory halo,
// and write z; the scatter P^T z is the pixel-sorted gather-reduce
// q_p = sum_{t in p} z_t v_t.
#include <type_traits>

#include "bm_internal.cuh"
#include "fft_filter.cuh"
#include "white_matvec.cuh"

namespace bm {

namespace {

constexpr int kWarps = 8;  // warps per block in the warp-per-item kernels
static_assert(kWarps == kWhiteWarps, "the white-noise kernels share the warp-per-item grid");

// x (FP64, [npix][NC]) -> FP32 copy with masked pixels zeroed.
template <typename TO>
__global__ void masked_copy_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask,
                                   int64_t npix, int nc, TO* __restrict__ out) {
    const int64_t n = npix * nc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mask[i / nc] ? TO(0) : TO(x[i]);
}

// x (FP64, [npix][NC]) -> one FP32 (a, b, c, 0) per pixel with y = a + b cos
// + c sin, masked pixels zeroed: IQU (I, Q, U), QU (0, Q, U), I (I, 0, 0).
// Sixteen aligned bytes per pixel, so P x reads its map entry in one load.
__global__ void masked_copy4_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask,
                                    int64_t npix, int nc, float4* __restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!mask[p]) {
            const double* xp = x + p * nc;
            if (nc == 3) v = make_float4((float)xp[0], (float)xp[1], (float)xp[2], 0.f);
            else if (nc == 2) v = make_float4(0.f, (float)xp[0], (float)xp[1], 0.f);
            else v.x = (float)xp[0];
        }
        out[p] = v;
    }
}

// ---------------------------------- white, FP32 form, half-wave-plate angle
// The same operator for a pointing whose angle follows the half-wave-plate
// model (bm_pointing_create_hwp): per sorted sample the kernel reads only its
// time index t (4 bytes), finds its detector d (t / ns for equal detectors,
// else a search of the offsets), rebuilds (cos 2 theta, sin 2 theta) in FP32
// from the exactly reduced phase (hwp_turns32, hwp_trig32: a table of
// kHwpTab entries and a short polynomial) and accumulates w_d y v with
// y = v . x_p: FP32 products, FP32 group sums of 8 samples folded into
// double-float, warp sums in double-float, an FP64 partial per item.  The
// eight samples of a lane in flight are independent (each looks its
// detector up); the per-detector angle offsets and weights sit in shared
// memory up to kMaxDetSmem detectors.
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
white_matvec_hwp_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                        const int32_t* __restrict__ item_len, int64_t nitems, const uint32_t* __restrict__ perm,
                        HwpModel m, const float2* __restrict__ tab_g, const float2* __restrict__ wdf,
                        const float* __restrict__ x32, double* __restrict__ partial) {
    static_assert(NC > 1, "I-only maps do not depend on the angle");
    __shared__ float2 tab[kHwpTab];
    __shared__ uint32_t s_a0[kMaxDetSmem];
    __shared__ float s_w[kMaxDetSmem];
    for (int j = threadIdx.x; j < kHwpTab; j += blockDim.x) tab[j] = tab_g[j];
    const bool in_smem = m.ndet <= kMaxDetSmem;
    if (in_smem)
        for (int d = threadIdx.x; d < m.ndet; d += blockDim.x) {
            s_a0[d] = (uint32_t)(m.turn0[d] >> 32);
            s_w[d] = wdf[d].x;
        }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        float xI = 0.f, xQ, xU;
        if (NC == 3) { xI = x32[3 * p]; xQ = x32[3 * p + 1]; xU = x32[3 * p + 2]; }
        else { xQ = x32[2 * p]; xU = x32[2 * p + 1]; }
        float aI = 0.f, aQ = 0.f, aU = 0.f;
        df32 AI = {0.f, 0.f}, AQ = {0.f, 0.f}, AU = {0.f, 0.f};
        auto step = [&](uint32_t t) {
            const int d = det_of(m.off, m.ndet, m.ns, m.inv_ns, t);
            const uint32_t dbeg = m.ns ? (uint32_t)d * m.ns : m.off[d];
            const uint32_t a0 = in_smem ? s_a0[d] : (uint32_t)(m.turn0[d] >> 32);
            const float w = in_smem ? s_w[d] : wdf[d].x;
            const float2 cs = hwp_trig32(hwp_turns32(m.nu, a0, t - dbeg), tab);
            float y = fmaf(cs.x, xQ, cs.y * xU);
            if (NC == 3) y += xI;
            const float wy = w * y;
            if (NC == 3) aI += wy;
            aQ = fmaf(wy, cs.x, aQ);
            aU = fmaf(wy, cs.y, aU);
        };
        auto fold = [&]() {
            if (NC == 3) AI = df_add(AI, aI);
            AQ = df_add(AQ, aQ);
            AU = df_add(AU, aU);
            aI = aQ = aU = 0.f;
        };
        int i = lane;
        for (; i + 224 < len; i += 256) {  // eight samples a lane, their loads issued together
            uint32_t t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = __ldcs(perm + b + i + 32 * u);
#pragma unroll
            for (int u = 0; u < 8; ++u) step(t[u]);
            fold();
        }
        for (; i < len; i += 32) step(__ldcs(perm + b + i));
        fold();
        AQ = df_warp_sum(AQ);
        AU = df_warp_sum(AU);
        if (NC == 3) AI = df_warp_sum(AI);
        if (lane == 0) {
            if (NC == 3) {
                partial[3 * k] = df_to_double(AI);
                partial[3 * k + 1] = df_to_double(AQ);
                partial[3 * k + 2] = df_to_double(AU);
            } else {
                partial[2 * k] = df_to_double(AQ);
                partial[2 * k + 1] = df_to_double(AU);
            }
        }
    }
}

// ------------------------------------------------------- white, FP64 form

template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
white_matvec_f64_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                        const int32_t* __restrict__ item_len, int64_t nitems,
                        const uint32_t* __restrict__ perm, const float2* __restrict__ hi,
                        const float2* __restrict__ lo, const uint32_t* __restrict__ det_off, int ndet,
                        uint32_t ns, float inv_ns, const double* __restrict__ white,
                        const double* __restrict__ w64sort, const double* __restrict__ x,
                        double* __restrict__ partial) {
    __shared__ uint32_t s_off[kMaxDetSmem + 1];
    const bool in_smem = ndet <= kMaxDetSmem;
    if (in_smem)
        for (int d = threadIdx.x; d <= ndet; d += blockDim.x) s_off[d] = det_off[d];
    __syncthreads();
    const uint32_t* offp = in_smem ? s_off : det_off;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        double xv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] = x[NC * p + c];
        double acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0;
        // the lane's samples are in increasing time order: the detector is
        // looked up only when t passes the current one's end
        uint32_t dend = 0;
        double w = 0.0;
        auto add = [&](int64_t si, uint32_t t) {
            if (w64sort) {  // a weight per sample
                w = w64sort[si];
            } else if (t >= dend) {
                const int d = det_of(offp, ndet, ns, inv_ns, t);
                dend = ns ? (uint32_t)(d + 1) * ns : offp[d + 1];
                w = white[d];
            }
            if (NC == 1) {
                acc[0] += w * xv[0];
            } else {
                const double2 cs = trig64_at(hi, lo, si);
                double y = cs.x * xv[NC - 2] + cs.y * xv[NC - 1];
                if (NC == 3) y += xv[0];
                const double wy = w * y;
                if (NC == 3) acc[0] += wy;
                acc[NC - 2] += wy * cs.x;
                acc[NC - 1] += wy * cs.y;
            }
        };
        int i = lane;
        for (; i + 96 < len; i += 128) {  // four samples' permutation loads together
            uint32_t t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) t[u] = perm[b + i + 32 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u) add(b + i + 32 * u, t[u]);
        }
        for (; i < len; i += 32) add(b + i, perm[b + i]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = warp_sum(acc[c]);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < NC; ++c) partial[NC * k + c] = acc[c];
    }
}

// ---------------------------------------------- pixel-sorted gather-reduce
// q_p partial = sum over item samples of g[perm_i] * f * v_i, where
// f = w_d(perm_i) when `weighted`, else 1, and v_i the pointing row.  G is
// float or double.  With gs (an FP32 TOD already in pixel-sorted order) the
// value is gs[i], read as a stream, instead of the gather g[perm_i].  Two
// arithmetic forms:
//   DF = false: FP64 products and sums (trig hi + lo), as the FP64 path needs;
//   DF = true : double-float products and sums on the FP32 pipes (~48 bits);
//               the trig pair is (hi, lo) when present, else the exact hi.
// The gathered value as a double-float pair or an FP64 number: an FP32
// value, an FP64 value, or a double-float pair stored as float2 (hi, lo).
__device__ __forceinline__ df32 as_df(float v) { return {v, 0.f}; }
__device__ __forceinline__ df32 as_df(double v) { return df_from(v); }
__device__ __forceinline__ df32 as_df(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ double as_f64(float v) { return v; }
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float2 v) { return (double)v.x + (double)v.y; }
template <typename G> __device__ __forceinline__ G from_f32(float v) { return (G)v; }
template <> __device__ __forceinline__ float2 from_f32<float2>(float v) { return make_float2(v, 0.f); }

template <int NC, typename G, bool DF>
__global__ void __launch_bounds__(kWarps * 32)
gather_reduce_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                     const int32_t* __restrict__ item_len, int64_t nitems,
                     const uint32_t* __restrict__ perm, const float2* __restrict__ hi,
                     const float2* __restrict__ lo, const G* __restrict__ g, const float* __restrict__ gs,
                     bool weighted, DetTables dt, const double* __restrict__ white, int ndet,
                     double* __restrict__ partial) {
    __shared__ uint32_t s_off[kMaxDetSmem + 1];
    __shared__ float2 s_w[kMaxDetSmem];
    const bool in_smem = weighted && ndet <= kMaxDetSmem;
    if (in_smem) {
        for (int d = threadIdx.x; d <= ndet; d += blockDim.x) s_off[d] = dt.off[d];
        for (int d = threadIdx.x; d < ndet; d += blockDim.x) s_w[d] = dt.wdf[d];
    }
    __syncthreads();
    const uint32_t* offp = in_smem ? s_off : dt.off;
    const float2* wp = in_smem ? s_w : dt.wdf;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        if (DF) {
            df32 acc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = {0.f, 0.f};
            // a lane's samples of one item are in increasing time order: the
            // detector is looked up only when t passes the current one's end
            uint32_t dend = 0;
            float2 w = make_float2(0.f, 0.f);
            // lazily renormalised sums (rhs_term_lazy, the block assembly's
            // fused RHS uses the same steps): renormalised after every
            // kLazyNorm samples of the lane and at the end
            int nadd = 0;
            auto add = [&](int64_t si, uint32_t t, G gv, float2 h, float2 l) {
                df32 val;
                val = as_df(gv);
                if (weighted) {
                    if (dt.wsort) {  // a weight per sample
                        w = dt.wsort[si];
                    } else if (t >= dend) {
                        const int d = det_of(offp, ndet, dt.ns, dt.inv_ns, t);
                        dend = dt.ns ? (uint32_t)(d + 1) * dt.ns : offp[d + 1];
                        w = wp[d];
                    }
                }
                rhs_term_lazy<NC>(acc, val.hi, val.lo, weighted, w, h, l);
                if (++nadd == kLazyNorm) {
                    nadd = 0;
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc_norm(acc[c]);
                }
            };
            // Eight samples per lane in flight (the gathers g[perm] are
            // independent); the lane's samples are still added in order.
            constexpr int U = 8;
            int i = lane;
            for (; i + 32 * (U - 1) < len; i += 32 * U) {
                uint32_t t[U];
                G gv[U];
                float2 h[U], l[U];
#pragma unroll
                for (int u = 0; u < U; ++u) t[u] = perm[b + i + 32 * u];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    gv[u] = gs ? from_f32<G>(gs[b + i + 32 * u]) : g[t[u]];
                    h[u] = NC > 1 ? hi[b + i + 32 * u] : make_float2(0.f, 0.f);
                    l[u] = (NC > 1 && lo) ? lo[b + i + 32 * u] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) add(b + i + 32 * u, t[u], gv[u], h[u], l[u]);
            }
            for (; i < len; i += 32) {
                const int64_t si = b + i;
                const uint32_t t = perm[si];
                const float2 h = NC > 1 ? hi[si] : make_float2(0.f, 0.f);
                const float2 l = (NC > 1 && lo) ? lo[si] : make_float2(0.f, 0.f);
                add(si, t, gs ? from_f32<G>(gs[si]) : g[t], h, l);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                acc_norm(acc[c]);
                acc[c] = df_warp_sum(acc[c]);
            }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < NC; ++c) partial[NC * k + c] = df_to_double(acc[c]);
        } else {
            double acc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = 0.0;
            uint32_t dend = 0;
            double wd = 0.0;
            auto add = [&](uint32_t t, G gv, int64_t si) {
                double val = as_f64(gv);
                if (weighted) {
                    if (dt.w64sort) {  // a weight per sample
                        wd = dt.w64sort[si];
                    } else if (t >= dend) {
                        const int d = det_of(offp, ndet, dt.ns, dt.inv_ns, t);
                        dend = dt.ns ? (uint32_t)(d + 1) * dt.ns : offp[d + 1];
                        wd = white[d];
                    }
                    val *= wd;
                }
                if (NC == 1) {
                    acc[0] += val;
                } else {
                    const double2 cs = trig64_at(hi, lo, si);
                    if (NC == 3) acc[0] += val;
                    acc[NC - 2] += val * cs.x;
                    acc[NC - 1] += val * cs.y;
                }
            };
            int i = lane;
            for (; i + 96 < len; i += 128) {
                uint32_t t[4];
                G gv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) t[u] = perm[b + i + 32 * u];
#pragma unroll
                for (int u = 0; u < 4; ++u) gv[u] = gs ? from_f32<G>(gs[b + i + 32 * u]) : g[t[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) add(t[u], gv[u], b + i + 32 * u);
            }
            for (; i < len; i += 32) {
                const uint32_t t = perm[b + i];
                add(t, gs ? from_f32<G>(gs[b + i]) : g[t], b + i);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = warp_sum(acc[c]);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < NC; ++c) partial[NC * k + c] = acc[c];
        }
    }
}

// The transpose of the FP32 inner operator: q_p partial = sum over the item
// of z[perm_i] v_i with the FP32 trig (no weight, no lo part).  Products in
// FP32, eight samples per lane summed in FP32 and folded into a double-float
// accumulator (as the FP32 white matvec), lanes combined in double-float:
// the accuracy of the FP32 operator at a third of the instructions of
// per-sample double-float products.
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
gather_reduce_f32_kernel(const int64_t* __restrict__ item_beg, const int32_t* __restrict__ item_len, int64_t nitems,
                         const uint32_t* __restrict__ perm, const float2* __restrict__ hi,
                         const float* __restrict__ z, double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        float a[NC];
        df32 A[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            a[c] = 0.f;
            A[c] = {0.f, 0.f};
        }
        auto step = [&](float v, float2 h) {
            if (NC == 1) {
                a[0] += v;
            } else {
                if (NC == 3) a[0] += v;
                a[NC - 2] = fmaf(v, h.x, a[NC - 2]);
                a[NC - 1] = fmaf(v, h.y, a[NC - 1]);
            }
        };
        auto fold = [&]() {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                A[c] = df_add(A[c], a[c]);
                a[c] = 0.f;
            }
        };
        constexpr int U = 8;
        int i = lane;
        for (; i + 32 * (U - 1) < len; i += 32 * U) {
            uint32_t t[U];
            float v[U];
            float2 h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) t[u] = perm[b + i + 32 * u];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = z[t[u]];
                h[u] = NC > 1 ? hi[b + i + 32 * u] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) step(v[u], h[u]);
            fold();
        }
        for (; i < len; i += 32) step(z[perm[b + i]], NC > 1 ? hi[b + i] : make_float2(0.f, 0.f));
        fold();
#pragma unroll
        for (int c = 0; c < NC; ++c) A[c] = df_warp_sum(A[c]);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < NC; ++c) partial[NC * k + c] = df_to_double(A[c]);
    }
}

// ------------------------------------------------ time-chunked transpose
// The mixed Toeplitz operator's transpose q_p = sum_i z[perm_i] v_i gathers
// 4-byte z values at random time positions: each costs a DRAM sector.  It
// runs instead one time chunk of kPtChunk samples at a time (64 MB of z, which
// stays in L2), over each kept pixel's samples in that chunk: a pixel's
// samples are in time order in the sorted layout, so those of one chunk are
// contiguous.  Each pixel's double-float accumulator is updated chunk after
// chunk by one group of lanes (a fixed order: deterministic).
constexpr int kPtChunkBits = 24;
constexpr int kPtLanes = 8;  // lanes per segment (4 measured slower)

// sub[c * npix + p] = the first position of pixel p's run (counted from
// off[p]) whose sample lies in chunk c or later, for c in [0, nch]; c = nch
// gives the run's length.  Chunk-major, so that a chunk's pass reads two
// contiguous rows.  One warp per pixel; every entry is written exactly once.
__global__ void pt_bounds_kernel(const int64_t* __restrict__ off, const uint32_t* __restrict__ perm, int64_t npix,
                                 int nch, int32_t* __restrict__ sub) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npix; p += nwarps) {
        const int64_t b = off[p];
        const int32_t len = (int32_t)(off[p + 1] - b);
        int32_t* s = sub + p;
        const int f = len ? (int)(perm[b] >> kPtChunkBits) : nch;
        const int l = len ? (int)(perm[b + len - 1] >> kPtChunkBits) : nch;
        for (int c = lane; c <= nch; c += 32) {
            if (c <= f) s[(int64_t)c * npix] = 0;
            else if (c > l) s[(int64_t)c * npix] = len;
        }
        // each sample's chunk read once; the previous sample's from the
        // neighbouring lane (lane 0: the last lane of the previous round)
        int carry = f;
        for (int32_t i0 = 0; i0 < len; i0 += 32) {
            const int32_t i = i0 + lane;
            const int c1 = i < len ? (int)(perm[b + i] >> kPtChunkBits) : l;
            int c0 = __shfl_up_sync(0xffffffffu, c1, 1);
            if (lane == 0) c0 = carry;
            carry = __shfl_sync(0xffffffffu, c1, 31);
            if (i >= 1 && i < len)
                for (int c = c0 + 1; c <= c1; ++c) s[(int64_t)c * npix] = i;
        }
    }
}

// The chunk-major copy of the kept samples.  seglen[c][p] = samples of kept
// pixel p in chunk c (0 for masked pixels), nz[c][p] = 1 if any.
__global__ void cm_seglen_kernel(const int32_t* __restrict__ sub, const uint8_t* __restrict__ mask, int64_t npix,
                                 int nch, uint32_t* __restrict__ seglen, uint32_t* __restrict__ nz) {
    const int64_t n = (int64_t)nch * npix;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % npix;
        const uint32_t len = mask[p] ? 0u : (uint32_t)(sub[e + npix] - sub[e]);
        seglen[e] = len;
        nz[e] = len ? 1u : 0u;
    }
}

// Sample i of kept pixel p's sorted run goes to segpos[c][p] + (i - sub[c][p])
// with c its time chunk: within a segment the samples keep their (time)
// order.  One warp per pixel.
__global__ void cm_scatter_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ sub,
                                  const uint32_t* __restrict__ segpos, const uint8_t* __restrict__ mask,
                                  int64_t npix, const uint32_t* __restrict__ perm, const float2* __restrict__ hi,
                                  uint32_t* __restrict__ cm_t, float2* __restrict__ cm_cs) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npix; p += nwarps) {
        if (mask[p]) continue;
        const int64_t b = off[p];
        const int32_t len = (int32_t)(off[p + 1] - b);
        for (int32_t i = lane; i < len; i += 32) {
            const uint32_t t = perm[b + i];
            const int64_t e = (int64_t)(t >> kPtChunkBits) * npix + p;
            const uint32_t dst = segpos[e] + (uint32_t)(i - sub[e]);
            cm_t[dst] = t;
            cm_cs[dst] = hi[b + i];
        }
    }
}

// The non-empty segments in (chunk, pixel) order.
__global__ void cm_segments_kernel(const uint32_t* __restrict__ seglen, const uint32_t* __restrict__ segpos,
                                   const uint32_t* __restrict__ segidx, int64_t npix, int nch,
                                   int32_t* __restrict__ seg_pix, uint32_t* __restrict__ seg_beg,
                                   int32_t* __restrict__ seg_len) {
    const int64_t n = (int64_t)nch * npix;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t len = seglen[e];
        if (!len) continue;
        const uint32_t k = segidx[e];
        seg_pix[k] = (int32_t)(e % npix);
        seg_beg[k] = segpos[e];
        seg_len[k] = (int32_t)len;
    }
}

// One chunk of the transpose: per segment (a kept pixel's samples in chunk
// c, contiguous in the chunk-major order), the sum of z v (FP32 products,
// summed in FP32 groups of up to 8 per lane and folded into double-float),
// added to the pixel's accumulator.  z stays in time order: a chunk of it is
// 64 MB, which L2 keeps while the launch gathers from it; the chunk-major
// streams are read once with an evict-first hint so that they do not push it
// out.  kPtLanes lanes per segment, the warp's groups on consecutive
// segments; within a chunk a pixel has one segment, so each accumulator has
// one writer per launch, and the launches run in chunk order
// (deterministic).
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
pt_chunk_kernel(const int32_t* __restrict__ seg_pix, const uint32_t* __restrict__ seg_beg,
                const int32_t* __restrict__ seg_len, int64_t seg0, int64_t nseg,
                const uint32_t* __restrict__ cm_t, const float2* __restrict__ cm_cs,
                const float* __restrict__ z, float2* __restrict__ acc) {
    constexpr int G = 32 / kPtLanes;
    constexpr int U = 8;  // samples in flight per lane (4 measured slower)
    const int lane = threadIdx.x & 31, gl = lane % kPtLanes, grp = lane / kPtLanes;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t kw = ((int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)) * G; kw < nseg; kw += nwarps * G) {
        const int64_t k = kw + grp;
        int64_t p = 0, b = 0;
        int32_t len = 0;
        if (k < nseg) {
            p = seg_pix[seg0 + k];
            b = seg_beg[seg0 + k];
            len = seg_len[seg0 + k];
        }
        float a[NC];
        df32 A[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            a[c] = 0.f;
            A[c] = {0.f, 0.f};
        }
        for (int32_t i0 = 0; i0 < len; i0 += U * kPtLanes) {
            uint32_t t[U];
            float v[U];
            float2 h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t i = i0 + gl + u * kPtLanes;
                t[u] = i < len ? __ldcs(cm_t + b + i) : 0xFFFFFFFFu;
                h[u] = (NC > 1 && i < len) ? __ldcs(cm_cs + b + i) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = t[u] != 0xFFFFFFFFu ? z[t[u]] : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (NC == 1) {
                    a[0] += v[u];
                } else {
                    if (NC == 3) a[0] += v[u];
                    a[NC - 2] = fmaf(v[u], h[u].x, a[NC - 2]);
                    a[NC - 1] = fmaf(v[u], h[u].y, a[NC - 1]);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                A[c] = df_add(A[c], a[c]);
                a[c] = 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int o = kPtLanes / 2; o > 0; o >>= 1) A[c] = df_add(A[c], df_shfl_xor(A[c], o));
        }
        if (gl == 0 && len > 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float2 old = acc[p * NC + c];
                const df32 s = df_add(df32{old.x, old.y}, A[c]);
                acc[p * NC + c] = make_float2(s.hi, s.lo);
            }
        }
    }
}

// The double-float form of the chunk transpose (the refinement operator's and
// the RHS's pixel sums of z given as (hi, lo) pairs, for exact FP32 trig):
// one half of chunk c's time range per launch -- so that the 64 MB of z
// pairs it gathers stay in L2 -- i.e. of each segment the first seg_mid
// samples (half 0) or the rest (half 1), its samples being in time order;
// summed in the lazily renormalised double-float form of the gather-reduce
// (rhs_term_lazy) by kPtLanes lanes per segment, then added to the pixel's
// double-float accumulator (one writer per launch; launches in time order).
// Metadata one iteration ahead and the accumulator read early (the FP32
// pt_chunk_kernel measured slower with the same change: its extra registers
// cut it from five resident blocks per SM to four).
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
pt_chunk_df_kernel(const int32_t* __restrict__ seg_pix, const uint32_t* __restrict__ seg_beg,
                   const int32_t* __restrict__ seg_len, const int32_t* __restrict__ seg_mid, int64_t seg0,
                   int64_t nseg, int half, const uint32_t* __restrict__ cm_t, const float2* __restrict__ cm_cs,
                   const float2* __restrict__ z, float2* __restrict__ acc) {
    constexpr int G = 32 / kPtLanes;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31, gl = lane % kPtLanes, grp = lane / kPtLanes;
    const int64_t stride = (int64_t)gridDim.x * kWarps * G;
    auto meta = [&](int64_t k, int64_t& p, int64_t& b, int32_t& i_lo, int32_t& i_hi) {
        p = 0;
        b = 0;
        i_lo = 0;
        i_hi = 0;
        if (k < nseg) {
            p = seg_pix[seg0 + k];
            b = seg_beg[seg0 + k];
            const int32_t mid = seg_mid[seg0 + k];
            i_lo = half ? mid : 0;
            i_hi = half ? seg_len[seg0 + k] : mid;
        }
    };
    int64_t kw = ((int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)) * G;
    int64_t p, b;
    int32_t i_lo, i_hi;
    meta(kw + grp, p, b, i_lo, i_hi);
    for (; kw < nseg; kw += stride) {
        int64_t pn, bn;
        int32_t lon, hin;
        meta(kw + stride + grp, pn, bn, lon, hin);
        const bool writer = gl == 0 && i_hi > i_lo;
        float2 old[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) old[c] = writer ? acc[p * NC + c] : make_float2(0.f, 0.f);
        df32 A[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) A[c] = {0.f, 0.f};
        int nadd = 0;
        for (int32_t i0 = i_lo; i0 < i_hi; i0 += U * kPtLanes) {
            uint32_t t[U];
            float2 h[U], v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t i = i0 + gl + u * kPtLanes;
                t[u] = i < i_hi ? __ldcs(cm_t + b + i) : 0xFFFFFFFFu;
                h[u] = (NC > 1 && i < i_hi) ? __ldcs(cm_cs + b + i) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = t[u] != 0xFFFFFFFFu ? z[t[u]] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t[u] != 0xFFFFFFFFu) {
                    rhs_term_lazy<NC>(A, v[u].x, v[u].y, false, make_float2(0.f, 0.f), h[u], make_float2(0.f, 0.f));
                    if (++nadd == kLazyNorm) {
                        nadd = 0;
#pragma unroll
                        for (int c = 0; c < NC; ++c) acc_norm(A[c]);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            acc_norm(A[c]);
#pragma unroll
            for (int o = kPtLanes / 2; o > 0; o >>= 1) A[c] = df_add(A[c], df_shfl_xor(A[c], o));
        }
        if (writer) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const df32 s = df_add(df32{old[c].x, old[c].y}, A[c]);
                acc[p * NC + c] = make_float2(s.hi, s.lo);
            }
        }
        p = pn;
        b = bn;
        i_lo = lon;
        i_hi = hin;
    }
}

// seg_mid[k] = the number of segment k's samples (in time order) before
// t_mid, the middle of its chunk's time range: one binary search per segment
// when the chunk-major order is built.
__global__ void cm_seg_mid_kernel(const uint32_t* __restrict__ seg_beg, const int32_t* __restrict__ seg_len,
                                  int64_t seg0, int64_t nseg, uint32_t t_mid, const uint32_t* __restrict__ cm_t,
                                  int32_t* __restrict__ seg_mid) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nseg; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = seg_beg[seg0 + k];
        int32_t lo = 0, hi = seg_len[seg0 + k];
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (cm_t[b + mid] < t_mid) lo = mid + 1; else hi = mid;
        }
        seg_mid[seg0 + k] = lo;
    }
}

__global__ void pt_finalize_kernel(const float2* __restrict__ acc, const uint8_t* __restrict__ mask, int64_t npix,
                                   int nc, double* __restrict__ q) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < nc; ++k) {
            const float2 s = acc[p * nc + k];
            q[p * nc + k] = mask[p] ? 0.0 : (double)s.x + (double)s.y;
        }
}

// ------------------------------------------------------- time-ordered work
// y = P x over every non-flagged sample (FP64 trig).
__global__ void pointing_apply_kernel(const int32_t* __restrict__ pix, const float2* __restrict__ hi,
                                      const float2* __restrict__ lo, int64_t n, int nc,
                                      const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[t];
        double v = 0.0;
        if (p >= 0) {
            if (nc == 1) {
                v = x[p];
            } else {
                const double2 cs = trig64_at(hi, lo, t);
                const double* xp = x + (int64_t)p * nc;
                v = cs.x * xp[nc - 2] + cs.y * xp[nc - 1];
                if (nc == 3) v += xp[0];
            }
        }
        y[t] = v;
    }
}

// --------------------------------------------------------- Toeplitz filter
// Sample sources for the filter input y_t.
template <typename D>
struct SrcMaskedTod {  // y_t = d_t on kept samples, else 0 (in the TOD's own type)
    const int32_t* pix; const uint8_t* mask; const D* d;
    __device__ D operator()(int64_t t) const {
        const int32_t p = pix[t];
        if (p < 0 || mask[p]) return D(0);
        return d[t];
    }
};
struct SrcPlain {
    const double* y;
    __device__ double operator()(int64_t t) const { return y[t]; }
};
struct SrcPlainF32 {
    const float* y;
    __device__ float operator()(int64_t t) const { return y[t]; }
};
struct SrcPlainDF {  // a double-float (hi, lo) pair per sample
    const float2* y;
    __device__ float2 operator()(int64_t t) const { return y[t]; }
};

// The masked TOD as double-float pairs (SrcMaskedTod's values, written once
// before the double-float filter so that its loads are plain streams rather
// than a pixel-then-mask gather per sample).
template <typename D>
__global__ void masked_tod_df_kernel(const int32_t* __restrict__ pix, const uint8_t* __restrict__ mask,
                                     const D* __restrict__ d, int64_t n, float2* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = __ldcs(pix + t);
        const D v = __ldcs(d + t);
        float2 o = make_float2(0.f, 0.f);
        if (p >= 0 && !mask[p]) {
            if (sizeof(D) == 4) {
                o.x = (float)v;
            } else {
                const df32 f = df_from((double)v);
                o = make_float2(f.hi, f.lo);
            }
        }
        out[t] = o;
    }
}

// y = P x over every sample in double-float on the FP32 pipes (the
// refinement operator's input): the trig pair as (hi, lo) (lo absent: the
// exact FP32 values), the map as masked_copy_df_kernel writes it (two float4
// of (hi, lo) pairs per pixel: I, Q; U, 0); y written as
// (hi, lo) pairs.  Flagged samples and masked pixels give 0.
__global__ void pointing_apply_df_kernel(const int32_t* __restrict__ pix, const float2* __restrict__ hi,
                                         const float2* __restrict__ lo, int64_t n, const float4* __restrict__ x2,
                                         float2* __restrict__ y) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = pix[t];
        df32 v = {0.f, 0.f};
        if (p >= 0) {
            const float2 h = hi[t];
            const float2 l = lo ? lo[t] : make_float2(0.f, 0.f);
            const float4 u = x2[2 * (int64_t)p], w = x2[2 * (int64_t)p + 1];
            const df32 c = {h.x, l.x}, s = {h.y, l.y};
            v = df_add(df_add(df32{u.x, u.y}, df_mul(c, df32{u.z, u.w})), df_mul(s, df32{w.x, w.y}));
        }
        y[t] = make_float2(v.hi, v.lo);
    }
}

// z (FP64) -> (hi, lo) pairs.
__global__ void to_df_kernel(const double* __restrict__ z, int64_t n, float2* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const df32 v = df_from(z[t]);
        out[t] = make_float2(v.hi, v.lo);
    }
}

// y = P x over every sample in FP32, from the padded map x4 (zero on masked
// pixels, so their samples give 0; flagged samples give 0): the filter's
// input, computed by a full-occupancy elementwise pass so that the filter
// kernel reads it with plain coalesced loads instead of a dependent
// pixel-then-map gather.
__global__ void pointing_apply_f32_kernel(const int32_t* __restrict__ pix, const float2* __restrict__ hi, int64_t n,
                                          const float4* __restrict__ x4, float* __restrict__ y) {
    // four consecutive samples per thread and iteration, with 16-byte loads
    // and stores (pix and y by four, the trig pairs by two) and the four map
    // gathers issued together; the arrays are 16-byte aligned device buffers
    const int64_t nq = n >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int4* pix4 = reinterpret_cast<const int4*>(pix);
    const float4* hi4 = reinterpret_cast<const float4*>(hi);
    float4* y4 = reinterpret_cast<float4*>(y);
    // two groups of four per iteration, all their loads issued first (more
    // memory requests in flight per thread)
    auto group = [&](const int4 p, const float4 ha, const float4 hb, int64_t q) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 x0 = p.x >= 0 ? x4[p.x] : z, x1 = p.y >= 0 ? x4[p.y] : z;
        const float4 x2 = p.z >= 0 ? x4[p.z] : z, x3 = p.w >= 0 ? x4[p.w] : z;
        float4 out;
        out.x = fmaf(ha.x, x0.y, fmaf(ha.y, x0.z, x0.x));
        out.y = fmaf(ha.z, x1.y, fmaf(ha.w, x1.z, x1.x));
        out.z = fmaf(hb.x, x2.y, fmaf(hb.y, x2.z, x2.x));
        out.w = fmaf(hb.z, x3.y, fmaf(hb.w, x3.z, x3.x));
        y4[q] = out;
    };
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < nq; q += 2 * stride) {
        const int64_t q2 = q + stride;
        const int4 pa = __ldcs(pix4 + q), pb = __ldcs(pix4 + q2);
        const float4 ha = __ldcs(hi4 + 2 * q), hb = __ldcs(hi4 + 2 * q + 1);
        const float4 hc = __ldcs(hi4 + 2 * q2), hd = __ldcs(hi4 + 2 * q2 + 1);
        group(pa, ha, hb, q);
        group(pb, hc, hd, q2);
    }
    if (q < nq) group(__ldcs(pix4 + q), __ldcs(hi4 + 2 * q), __ldcs(hi4 + 2 * q + 1), q);
    // the last n mod 4 samples
    for (int64_t t = 4 * nq + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const int32_t pp = pix[t];
        const float2 h = hi[t];
        const float4 xv = pp >= 0 ? x4[pp] : make_float4(0.f, 0.f, 0.f, 0.f);
        y[t] = fmaf(h.x, xv.y, fmaf(h.y, xv.z, xv.x));
    }
}

constexpr int kTzThreads = 256;

struct TzGeom {
    const int64_t* det_off;      // [ndet + 1]
    const int64_t* tile_start;   // [ndet + 1] prefix of tiles per detector
    int ndet;
    int64_t chunk_len;
    int64_t tiles_per_chunk;
    int64_t ntiles;
};

__device__ __forceinline__ int find_tile_det(const int64_t* ts, int ndet, int64_t tile) {
    int lo = 0, hi = ndet - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ts[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One block per tile of TT outputs; each thread computes R consecutive
// outputs from a register window of 2R samples that advances R taps at a
// time (R*R FMAs per R buffer loads).  The FP32 buffer is padded by one word
// every 32 (index a -> a + a/32) so that the window loads of the 32 lanes
// (R = 8 apart) fall in distinct banks.  The tap array is zero-padded to a
// multiple of R and the buffer carries 2R trailing zeros.
template <typename T, int R>
__host__ __device__ __forceinline__ int tz_taps_padded(int L) { return ((2 * L - 1 + R - 1) / R) * R; }

template <typename T, int R, class Src>
__global__ void __launch_bounds__(kTzThreads)
toeplitz_kernel(Src src, const T* __restrict__ coeffs, int L, TzGeom geo, T* __restrict__ z) {
    constexpr int TT = kTzThreads * R;
    extern __shared__ __align__(16) unsigned char tz_smem[];
    const int ntap = tz_taps_padded<T, R>(L);
    T* kern = reinterpret_cast<T*>(tz_smem);  // [ntap]
    T* buf = kern + ntap;                      // padded halo buffer
    auto pad = [](int a) { return sizeof(T) == 4 ? a + (a >> 5) : a; };

    for (int64_t tile = blockIdx.x; tile < geo.ntiles; tile += gridDim.x) {
        const int d = find_tile_det(geo.tile_start, geo.ndet, tile);
        const int64_t local = tile - geo.tile_start[d];
        const int64_t c = local / geo.tiles_per_chunk, kk = local % geo.tiles_per_chunk;
        const int64_t cs = geo.det_off[d] + c * geo.chunk_len;
        const int64_t ce = min(cs + geo.chunk_len, geo.det_off[d + 1]);
        const int64_t t0 = cs + kk * TT;
        if (t0 >= ce) continue;  // uniform across the block
        const int64_t t1 = min(t0 + (int64_t)TT, ce);
        const int64_t b0 = t0 - (L - 1);  // buffer index 0 <-> sample b0
        const int nbuf = (int)(t1 - t0) + 2 * (L - 1);
        const int nfill = (int)(t1 - t0) + ntap + 2 * R;
        __syncthreads();  // previous tile done with smem
        for (int j = threadIdx.x; j < ntap; j += kTzThreads)
            kern[j] = j < 2 * L - 1 ? coeffs[(int64_t)d * L + abs(j - (L - 1))] : T(0);
        for (int j = threadIdx.x; j < nfill; j += kTzThreads) {
            const int64_t t = b0 + j;
            buf[pad(j)] = (j < nbuf && t >= cs && t < ce) ? T(src(t)) : T(0);
        }
        __syncthreads();
        const int o0 = threadIdx.x * R;  // first output (relative to t0)
        if (t0 + o0 < t1) {
            T acc[R];
            T win[2 * R];
#pragma unroll
            for (int r = 0; r < R; ++r) { acc[r] = T(0); win[R + r] = buf[pad(o0 + r)]; }
            for (int j = 0; j < ntap; j += R) {
#pragma unroll
                for (int r = 0; r < R; ++r) { win[r] = win[R + r]; win[R + r] = buf[pad(o0 + j + R + r)]; }
#pragma unroll
                for (int jj = 0; jj < R; ++jj) {
                    const T kj = kern[j + jj];
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] = fma(kj, win[r + jj], acc[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (t0 + o0 + r < t1) z[t0 + o0 + r] = acc[r];
        }
    }
}

template <typename T, int R>
size_t toeplitz_smem(int L) {
    const int TT = kTzThreads * R;
    const int ntap = tz_taps_padded<T, R>(L);
    const int nfill = TT + ntap + 2 * R;
    const int padded = sizeof(T) == 4 ? nfill + nfill / 32 + 1 : nfill;
    return sizeof(T) * ((size_t)ntap + padded);
}

}  // namespace

// --------------------------------------------------------------- wrappers
struct ToeplitzPlan {
    TzGeom geo;
};

// Tiles of TT outputs per chunk of each detector; the per-detector tile
// prefix is uploaded once per noise model and tile length.
static void plan_toeplitz(bm_inv_noise* n, int TT, ToeplitzPlan& tp) {
    auto it = n->tile_plans.find(TT);
    if (it == n->tile_plans.end()) {
        int64_t maxlen = 0;
        for (int d = 0; d < n->ndet; ++d) maxlen = std::max(maxlen, n->h_det_off[d + 1] - n->h_det_off[d]);
        const int64_t eff_chunk = std::min(n->chunk_len, maxlen);
        const int64_t tpc = (eff_chunk + TT - 1) / TT;
        std::vector<int64_t> ts(n->ndet + 1, 0);
        for (int d = 0; d < n->ndet; ++d) {
            const int64_t len = n->h_det_off[d + 1] - n->h_det_off[d];
            const int64_t nch = (len + n->chunk_len - 1) / n->chunk_len;
            ts[d + 1] = ts[d] + nch * tpc;
        }
        bm_inv_noise::TilePlan& pl = n->tile_plans[TT];
        pl.tile_start.alloc(n->ndet + 1);
        BM_CUDA(cudaMemcpyAsync(pl.tile_start.get(), ts.data(), sizeof(int64_t) * (n->ndet + 1),
                                cudaMemcpyHostToDevice, n->ctx->stream));
        BM_CUDA(cudaStreamSynchronize(n->ctx->stream));  // ts is a host temporary
        pl.tiles_per_chunk = tpc;
        pl.ntiles = ts[n->ndet];
        it = n->tile_plans.find(TT);
    }
    tp.geo = TzGeom{n->det_off.get(), it->second.tile_start.get(), n->ndet, n->chunk_len,
                    it->second.tiles_per_chunk, it->second.ntiles};
}

template <typename T, int R, class Src>
static void run_toeplitz(bm_inv_noise* n, const Src& src, const T* coeffs, T* z) {
    bm_context* ctx = n->ctx;
    ToeplitzPlan tp;
    plan_toeplitz(n, kTzThreads * R, tp);
    if (tp.geo.ntiles == 0) return;
    const size_t smem = toeplitz_smem<T, R>(n->nlags);
    ensure_smem_limit(reinterpret_cast<const void*>(toeplitz_kernel<T, R, Src>), smem);
    const int grid = (int)std::min<int64_t>(tp.geo.ntiles, (int64_t)ctx->num_sms * 8);
    toeplitz_kernel<T, R, Src><<<grid, kTzThreads, smem, ctx->stream>>>(src, coeffs, n->nlags, tp.geo, z);
    BM_LAUNCH_CHECK();  // tile_start is released stream-ordered after the kernel
}

// The band spectra of every detector for an N-point transform (see
// band_spectrum_kernel), in the requested forms.
static void band_spectrum(bm_inv_noise* n, int N, double* spec64, float* spec32, float2* spec_df) {
    bm_context* ctx = n->ctx;
    const int threads = 256;
    DevBuf<double> cost(N);
    cos_table_kernel<<<(N + threads - 1) / threads, threads, 0, ctx->stream>>>(N, cost.get());
    BM_LAUNCH_CHECK();
    const int kb = (N / 2 + 1 + kBandK - 1) / kBandK;
    const size_t smem = sizeof(double) * ((size_t)N + (size_t)n->nlags);
    ensure_smem_limit(reinterpret_cast<const void*>(band_spectrum_kernel), smem);
    band_spectrum_kernel<<<(unsigned)((int64_t)n->ndet * kb), threads, smem, ctx->stream>>>(
        n->coeffs64.get(), cost.get(), n->ndet, n->nlags, N, kb, spec64, spec32, spec_df);
    BM_LAUNCH_CHECK();  // the table is released stream-ordered after the kernel
}

// FFT size for a band of L lags: the smallest power of two with at least half
// of each transform producing outputs (H >= N/2), grown toward a whole chunk,
// at most `cap`; 0 if the band is too long for `cap` (direct filter).
static int fft_size(int L, int64_t chunk_len, int cap) {
    const int64_t need = 4 * (int64_t)(L - 1);
    int64_t N = 64;
    while (N < need) N <<= 1;
    const int64_t want = chunk_len + 2 * (int64_t)(L - 1);
    while (N < cap && N < want) N <<= 1;
    return N <= cap ? (int)N : 0;
}

constexpr int kFftMinLags = 32;  // shorter bands: the direct filter is cheaper

void prepare_toeplitz_fft(bm_inv_noise* n) {
    if (n->nlags < kFftMinLags) return;
    bm_context* ctx = n->ctx;
    int64_t maxlen = 0;
    for (int d = 0; d < n->ndet; ++d) maxlen = std::max(maxlen, n->h_det_off[d + 1] - n->h_det_off[d]);
    const int64_t eff_chunk = std::min(n->chunk_len, maxlen);
    n->fft_n32 = fft_size(n->nlags, eff_chunk, 8192);
    n->fft_n64 = fft_size(n->nlags, eff_chunk, 4096);
    const int threads = 256;
    if (n->fft_n32) {
        const int N = n->fft_n32;
        n->spec32.alloc((size_t)n->ndet * (N / 2 + 1));
        n->tw32.alloc(N);
        band_spectrum(n, N, nullptr, n->spec32.get(), nullptr);
        twiddle_kernel<<<(N + threads - 1) / threads, threads, 0, ctx->stream>>>(N, nullptr, n->tw32.get());
        BM_LAUNCH_CHECK();
    }
    if (n->fft_n64) {
        const int N = n->fft_n64;
        n->spec64.alloc((size_t)n->ndet * (N / 2 + 1));
        n->spec_df.alloc((size_t)n->ndet * (N / 2 + 1));
        n->tw64.alloc(N);
        band_spectrum(n, N, n->spec64.get(), nullptr, n->spec_df.get());
        twiddle_kernel<<<(N + threads - 1) / threads, threads, 0, ctx->stream>>>(N, n->tw64.get(), nullptr);
        BM_LAUNCH_CHECK();
    }
    BM_CUDA(cudaStreamSynchronize(ctx->stream));
}

template <typename T, class Src>
static void run_toeplitz_fft(bm_inv_noise* n, const Src& src, int N, const typename FftIO<T>::spec_t* spec,
                             const cpx<typename FftIO<T>::tw_t>* tw, typename FftIO<T>::out_t* z) {
    bm_context* ctx = n->ctx;
    const int H = N - 2 * (n->nlags - 1);
    ToeplitzPlan tp;
    plan_toeplitz(n, H, tp);
    if (tp.geo.ntiles == 0) return;
    const FftGeom geo{tp.geo.det_off, tp.geo.tile_start, tp.geo.ndet, tp.geo.chunk_len, tp.geo.tiles_per_chunk,
                      tp.geo.ntiles};
    const size_t smem = fft_smem<T>(N);
    auto kern = toeplitz_fft_kernel<T, Src>;
    ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
    const int grid = resident_grid(ctx, kern, kFftThreads, tp.geo.ntiles, smem);
    kern<<<grid, kFftThreads, smem, ctx->stream>>>(src, spec, tw, N, n->nlags, geo, z);
    BM_LAUNCH_CHECK();
}

// z = band * y per chunk: FFT overlap-save when prepared, else the direct filter.
template <class Src>
static void apply_toeplitz_f32(bm_inv_noise* n, const Src& src, float* z) {
    if (n->fft_n32)
        run_toeplitz_fft<float>(n, src, n->fft_n32, n->spec32.get(), reinterpret_cast<const cpx<float>*>(n->tw32.get()), z);
    else
        run_toeplitz<float, 8>(n, src, n->coeffs32.get(), z);
}
// df: the FFT in double-float on the FP32 pipes (~48-bit arithmetic, for the
// refinement operator of the mixed solve) instead of FP64.
template <class Src>
static void apply_toeplitz_f64(bm_inv_noise* n, const Src& src, double* z) {
    const auto* tw = reinterpret_cast<const cpx<double>*>(n->tw64.get());
    if (n->fft_n64)
        run_toeplitz_fft<double>(n, src, n->fft_n64, n->spec64.get(), tw, z);
    else
        run_toeplitz<double, 4>(n, src, n->coeffs64.get(), z);
}
// A sample source read as FP64 (for the direct filter of short bands).
template <class Src>
struct SrcAsF64 {
    Src src;
    __device__ double operator()(int64_t t) const { return as_f64(src(t)); }
};
// The same in double-float, z as (hi, lo) pairs (the mixed path's RHS and
// refinement operator): the FFT form in double-float on the FP32 pipes; the
// direct filter (short bands) in FP64, converted.
template <class Src>
static void apply_toeplitz_df(bm_inv_noise* n, const Src& src, float2* z) {
    if (n->fft_n64) {
        const auto* tw = reinterpret_cast<const cpx<double>*>(n->tw64.get());
        run_toeplitz_fft<df32>(n, src, n->fft_n64, n->spec_df.get(), tw, z);
    } else {
        double* z64 = workspace_as<double>(n->ctx, "z64_direct", n->nsamples);
        run_toeplitz<double, 4>(n, SrcAsF64<Src>{src}, n->coeffs64.get(), z64);
        to_df_kernel<<<grid_for(n->ctx, (n->nsamples + 255) / 256, 16), 256, 0, n->ctx->stream>>>(z64, n->nsamples, z);
        BM_LAUNCH_CHECK();
    }
}

// ----------------------------------------------------------- offset filter
// W y for white noise with one baseline offset per interval marginalised out
// (Eq. 4 with the offsets as a template, W = Nk - Nk F (F^T Nk F)^-1 F^T Nk,
// F the interval indicators): on the kept samples of interval I,
// z_t = w_d (y_t - m_I), m_I the mean of y over those samples.  y is zero on
// every sample that is not kept (flagged, or in a masked pixel), so m_I is the
// interval's plain sum times 1 / (its kept samples).  The transpose reads z
// on kept samples only; elsewhere z is written by the same formula.
struct OffsetGeom {
    const int64_t* det_off;    // [ndet + 1]
    const int64_t* int_start;  // [ndet + 1] index of each detector's first interval
    int ndet;
    int64_t baseline_len;
    int64_t nint;
};

__device__ __forceinline__ void offset_interval(const OffsetGeom& g, int64_t j, int& d, int64_t& a, int64_t& e) {
    d = find_tile_det(g.int_start, g.ndet, j);
    a = g.det_off[d] + (j - g.int_start[d]) * g.baseline_len;
    e = min(a + g.baseline_len, g.det_off[d + 1]);
}

// One warp per interval.  The sum: FP32 (or FP64) groups of up to 8 per lane
// folded into FP64, then a butterfly over the warp, which leaves the same
// value in every lane (IEEE addition commutes); a fixed order, so the result
// is deterministic.  The second pass reads the interval again (from L2 for
// intervals of a few thousand samples) and writes z.
// Out = float2: z as double-float pairs (hi, lo), computed on the FP32 pipes
// (the gather-reduce reads them without FP64 conversions).
template <typename T, class Src, typename Out = T>
__global__ void __launch_bounds__(256)
offset_filter_kernel(Src src, OffsetGeom g, const double* __restrict__ white, const double* __restrict__ inv_cnt,
                     Out* __restrict__ z) {
    constexpr int U = 8;
    constexpr bool kF32Src = std::is_same<decltype(src(int64_t(0))), float>::value && std::is_same<T, double>::value;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nint; j += nwarps) {
        int d;
        int64_t a, e;
        offset_interval(g, j, d, a, e);
        double s = 0.0;
        if constexpr (kF32Src) {
            // an FP32 source summed in double-float on the FP32 pipes (the
            // FP64 pipe runs at 1/64 of their rate); df_add commutes, so the
            // butterfly leaves the same pair in every lane
            df32 acc = {0.f, 0.f};
            for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
                float v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = t0 + 32 * u < e ? src(t0 + 32 * u) : 0.f;
#pragma unroll
                for (int u = 0; u < U; ++u) acc = df_add(acc, v[u]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
            s = df_to_double(acc);
        } else {
            for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
                T v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = t0 + 32 * u < e ? src(t0 + 32 * u) : T(0);
                T ps = v[0];
#pragma unroll
                for (int u = 1; u < U; ++u) ps += v[u];
                s += (double)ps;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        const double m = s * (inv_cnt ? inv_cnt[j] : 1.0 / (double)(e - a));
        if constexpr (std::is_same<Out, float2>::value) {
            using V = decltype(src(int64_t(0)));
            const df32 md = df_from(m), wd = df_from(white[d]);
            const df32 nm = {-md.hi, -md.lo};
            for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
                V v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = t0 + 32 * u < e ? src(t0 + 32 * u) : V(0);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (t0 + 32 * u < e) {
                        const df32 zz = df_mul(wd, df_add(as_df(v[u]), nm));
                        z[t0 + 32 * u] = make_float2(zz.hi, zz.lo);
                    }
            }
        } else {
            const T mt = (T)m, w = (T)white[d];
            for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
                T v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = t0 + 32 * u < e ? src(t0 + 32 * u) : T(0);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (t0 + 32 * u < e) z[t0 + 32 * u] = w * (v[u] - mt);
            }
        }
    }
}

// 1 / (the kept samples of each interval), 0 where there are none; a sample
// is kept when it is not flagged and its pixel is not masked.
__global__ void offset_counts_kernel(const int32_t* __restrict__ pix, const uint8_t* __restrict__ mask, OffsetGeom g,
                                     double* __restrict__ inv) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nint; j += nwarps) {
        int d;
        int64_t a, e;
        offset_interval(g, j, d, a, e);
        unsigned c = 0;
        for (int64_t t = a + lane; t < e; t += 32) {
            const int32_t p = pix[t];
            c += p >= 0 && !mask[p];
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) inv[j] = c ? 1.0 / (double)c : 0.0;
    }
}

static void finalize(bm_context* ctx, const int64_t* pitem, const double* partial, int64_t npix, int nc,
                     double* q);

// isort[i] = the interval of sample perm[i] (pixel-sorted order).
__global__ void offset_isort_kernel(const uint32_t* __restrict__ perm, int64_t nvalid, OffsetGeom g,
                                    uint32_t* __restrict__ isort) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvalid;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = perm[i];
        const int d = find_tile_det(g.det_off, g.ndet, t);
        // t - det_off[d] < 2^32 and baseline_len <= nsamples < 2^32: a 32-bit division
        isort[i] = (uint32_t)g.int_start[d] + (uint32_t)(t - g.det_off[d]) / (uint32_t)g.baseline_len;
    }
}

// The mixed operator of the offset template in its destriping form,
//   A x = P^T Nk P x - P^T Nk F m,   m = (F^T Nk F)^-1 F^T Nk P x,
// two streaming passes instead of P x, the filter and a transpose.  The
// first, in time order, gives each interval's mean of P x over its kept
// samples (x4 is zero on masked pixels and flagged samples give 0, so the
// interval's plain sum over the kept count); it stores sqrt(w_d) m_I for
// IQU and QU (the sorted pass forms sqrt(w) v . x from the weighted stream)
// and m_I for I.  One warp per interval, sums as in offset_filter_kernel.
__global__ void __launch_bounds__(256)
offset_means_f32_kernel(const int32_t* __restrict__ pix, const float2* __restrict__ hi,
                        const float4* __restrict__ x4, OffsetGeom g, const double* __restrict__ inv_cnt,
                        const double* __restrict__ white, bool sqrt_weighted, float* __restrict__ mw) {
    constexpr int U = 8;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nint; j += nwarps) {
        int d;
        int64_t a, e;
        offset_interval(g, j, d, a, e);
        double s = 0.0;
        for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
            int32_t p[U];
            float2 h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = t0 + 32 * u;
                p[u] = t < e ? pix[t] : -1;
                h[u] = t < e ? hi[t] : make_float2(0.f, 0.f);
            }
            float ps = 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (p[u] >= 0) {
                    const float4 xv = x4[p[u]];
                    ps += fmaf(h[u].x, xv.y, fmaf(h[u].y, xv.z, xv.x));
                }
            s += (double)ps;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double m = s * inv_cnt[j];
            mw[j] = (float)(sqrt_weighted ? m * sqrt(white[d]) : m);
        }
    }
}

// The pixel-sorted pass: per kept sample, with u = sqrt(w)(cos, sin) from
// the weighted stream and r = |u| = sqrt(w),
//   y = r x_I + u . (x_Q, x_U) - sqrt(w) m_I,  q += y (r, u)   (IQU, QU),
//   q_I += w (x_I - m_I)                                      (I),
// summed per work item as the white kernel does (FP32 groups of 8 per lane
// folded into double-float, warp sums in double-float).
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
offset_matvec_f32_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                         const int32_t* __restrict__ item_len, int64_t nitems, const float2* __restrict__ wcs,
                         const float* __restrict__ w1, const uint32_t* __restrict__ isort,
                         const float* __restrict__ mw, const float4* __restrict__ x4,
                         double* __restrict__ partial) {
    constexpr int U = 8;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k], e = b + item_len[k];
        const float4 xv = x4[p];
        float a[NC];
        df32 A[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            a[c] = 0.f;
            A[c] = {0.f, 0.f};
        }
        for (int64_t i0 = b + lane; i0 < e; i0 += 32 * U) {
            // every stream load of the group is issued before the dependent
            // gathers of the means
            float m[U];
            uint32_t it[U];
            float2 wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = i0 + 32 * u < e;
                it[u] = in ? __ldg(isort + i0 + 32 * u) : 0u;
                if (NC == 1) wv[u].x = in ? __ldg(w1 + i0 + 32 * u) : 0.f;
                else wv[u] = in ? __ldg(wcs + i0 + 32 * u) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) m[u] = i0 + 32 * u < e ? __ldg(mw + it[u]) : 0.f;
            if (NC == 1) {
#pragma unroll
                for (int u = 0; u < U; ++u) a[0] = fmaf(wv[u].x, xv.x - m[u], a[0]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float2 w = wv[u];
                    float r = 0.f;
                    if (NC == 3) {
                        const float u2 = fmaf(w.x, w.x, w.y * w.y);
                        r = u2 > 0.f ? u2 * rsqrtf(u2) : 0.f;
                    }
                    const float y = fmaf(w.x, xv.y, fmaf(w.y, xv.z, r * xv.x)) - m[u];
                    if (NC == 3) a[0] = fmaf(y, r, a[0]);
                    a[NC - 2] = fmaf(y, w.x, a[NC - 2]);
                    a[NC - 1] = fmaf(y, w.y, a[NC - 1]);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                A[c] = df_add(A[c], a[c]);
                a[c] = 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) A[c] = df_warp_sum(A[c]);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < NC; ++c) partial[NC * k + c] = df_to_double(A[c]);
    }
}

// x (FP64, [npix][NC]) -> per pixel two float4 of double-float pairs
// (I.hi, I.lo, Q.hi, Q.lo), (U.hi, U.lo, 0, 0); zero on masked pixels and
// for the components the system does not have.
__global__ void masked_copy_df_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask, int64_t npix,
                                      int nc, float4* __restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        double v[3] = {0.0, 0.0, 0.0};
        if (!mask[p]) {
            const double* xp = x + p * nc;
            if (nc == 3) { v[0] = xp[0]; v[1] = xp[1]; v[2] = xp[2]; }
            else if (nc == 2) { v[1] = xp[0]; v[2] = xp[1]; }
            else v[0] = xp[0];
        }
        df32 d[3];
        for (int c = 0; c < 3; ++c) d[c] = df_from(v[c]);
        out[2 * p] = make_float4(d[0].hi, d[0].lo, d[1].hi, d[1].lo);
        out[2 * p + 1] = make_float4(d[2].hi, d[2].lo, 0.f, 0.f);
    }
}

// The refinement operator of the offset template (the destriping form of
// offset_means_f32_kernel in double-float, ~48-bit): each interval's mean of
// P x over its kept samples, times w_d, stored as a double-float pair.
// Products and sums per sample in double-float on the FP32 pipes; lo = NULL
// when the trig is exact in FP32.
__global__ void __launch_bounds__(256)
offset_means_df_kernel(const int32_t* __restrict__ pix, const float2* __restrict__ hi, const float2* __restrict__ lo,
                       const float4* __restrict__ xd, OffsetGeom g, const double* __restrict__ inv_cnt,
                       const double* __restrict__ white, int nc, float2* __restrict__ mwd) {
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < g.nint; j += nwarps) {
        int d;
        int64_t a, e;
        offset_interval(g, j, d, a, e);
        df32 acc = {0.f, 0.f};
        for (int64_t t0 = a + lane; t0 < e; t0 += 32 * U) {
            int32_t p[U];
            float2 h[U], l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = t0 + 32 * u;
                p[u] = t < e ? pix[t] : -1;
                h[u] = (t < e && nc > 1) ? hi[t] : make_float2(0.f, 0.f);
                l[u] = (t < e && nc > 1 && lo) ? lo[t] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (p[u] < 0) continue;
                const float4 a0 = xd[2 * (int64_t)p[u]];
                df32 y = {a0.x, a0.y};
                if (nc > 1) {
                    const float4 a1 = xd[2 * (int64_t)p[u] + 1];
                    y = df_add(y, df_mul(df32{a0.z, a0.w}, df32{h[u].x, l[u].x}));
                    y = df_add(y, df_mul(df32{a1.x, a1.y}, df32{h[u].y, l[u].y}));
                }
                acc = df_add(acc, y);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
        if (lane == 0) {
            const df32 m = df_from(df_to_double(acc) * inv_cnt[j] * white[d]);
            mwd[j] = make_float2(m.hi, m.lo);
        }
    }
}

// q_p partial = sum over the item's samples of (w_d m_I) (1, cos, sin) in
// double-float, the interval read from the sorted table.
template <int NC>
__global__ void __launch_bounds__(kWarps * 32)
offset_pt_df_kernel(const int64_t* __restrict__ item_beg, const int32_t* __restrict__ item_len, int64_t nitems,
                    const uint32_t* __restrict__ isort, const float2* __restrict__ hi, const float2* __restrict__ lo,
                    const float2* __restrict__ mwd, double* __restrict__ partial) {
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t b = item_beg[k], e = b + item_len[k];
        df32 A[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) A[c] = {0.f, 0.f};
        for (int64_t i0 = b + lane; i0 < e; i0 += 32 * U) {
            uint32_t it[U];
            float2 h[U], l[U], m[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = i0 + 32 * u < e;
                it[u] = in ? isort[i0 + 32 * u] : 0u;
                h[u] = (in && NC > 1) ? hi[i0 + 32 * u] : make_float2(0.f, 0.f);
                l[u] = (in && NC > 1 && lo) ? lo[i0 + 32 * u] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) m[u] = i0 + 32 * u < e ? mwd[it[u]] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const df32 v = {m[u].x, m[u].y};
                if (NC != 2) A[0] = df_add(A[0], v);
                if (NC > 1) {
                    A[NC - 2] = df_add(A[NC - 2], df_mul(v, df32{h[u].x, l[u].x}));
                    A[NC - 1] = df_add(A[NC - 1], df_mul(v, df32{h[u].y, l[u].y}));
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) A[c] = df_warp_sum(A[c]);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < NC; ++c) partial[NC * k + c] = df_to_double(A[c]);
    }
}

// q_p = B_p x_p - t_p on kept pixels (B the FP64 blocks P^T Nk P of the
// preconditioner build), 0 on masked ones.
template <int NC>
__global__ void block_minus_kernel(const double* __restrict__ B, const uint8_t* __restrict__ mask,
                                   const double* __restrict__ x, int64_t npix, double* __restrict__ q) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double* Bp = B + p * NC * NC;
        const double* xp = x + p * NC;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < NC; ++j) s = fma(Bp[i * NC + j], xp[j], s);
            q[p * NC + i] = mask[p] ? 0.0 : s - q[p * NC + i];
        }
    }
}

static OffsetGeom offset_geom(const bm_inv_noise* n) {
    return {n->det_off.get(), n->int_start.get(), n->ndet, n->baseline_len, n->nint};
}

void build_offset_counts(bm_precond* pc) {
    bm_context* ctx = pc->ctx;
    const bm_inv_noise* n = pc->n;
    const bm_pointing* p = pc->p;
    pc->ofs_inv.alloc(std::max<int64_t>(n->nint, 1));
    pc->ofs_isort.alloc(std::max<int64_t>(p->nvalid, 1));
    if (n->nint == 0) return;
    const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
    offset_counts_kernel<<<resident_grid(ctx, offset_counts_kernel, 256, (n->nint + 7) / 8), 256, 0, ctx->stream>>>(
        pix_t, pc->mask.get(), offset_geom(n), pc->ofs_inv.get());
    BM_LAUNCH_CHECK();
    if (p->nvalid > 0) {
        offset_isort_kernel<<<grid_for(ctx, (p->nvalid + 255) / 256, 16), 256, 0, ctx->stream>>>(
            p->perm.get(), p->nvalid, offset_geom(n), pc->ofs_isort.get());
        BM_LAUNCH_CHECK();
    }
}

// q = A x with the refinement operator of the offset template (see
// offset_means_df_kernel).
static void offset_matvec_refine(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int nc = p->ncomp;
    const int threads = 256;
    const int pgrid = grid_for(ctx, (p->npix + threads - 1) / threads, 16);
    float4* xd = workspace_as<float4>(ctx, "ofs_xd", 2 * p->npix);
    masked_copy_df_kernel<<<pgrid, threads, 0, s>>>(x, pc->mask.get(), p->npix, nc, xd);
    BM_LAUNCH_CHECK();
    float2* mwd = workspace_as<float2>(ctx, "ofs_mwd", std::max<int64_t>(n->nint, 1));
    if (n->nint > 0) {
        ScopedTimer timer(ctx, "offset_means_df");
        const float2* trig_t = time_trig(p);  // built here on first use when deferred
        const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
        offset_means_df_kernel<<<resident_grid(ctx, offset_means_df_kernel, 256, (n->nint + 7) / 8), 256, 0, s>>>(
            pix_t, trig_t, p->cs_lo_t.get(), xd, offset_geom(n), pc->ofs_inv.get(), n->white.get(),
            nc, mwd);
        BM_LAUNCH_CHECK();
    }
    double* partial = workspace_as<double>(ctx, "partial", (size_t)std::max<int64_t>(pc->nitems, 1) * nc);
    if (pc->nitems > 0) {
        ScopedTimer timer(ctx, "offset_pt_df");
        const int64_t wunits = (pc->nitems + kWarps - 1) / kWarps;
#define BM_OP(NC)                                                                                                  \
    offset_pt_df_kernel<NC><<<resident_grid(ctx, offset_pt_df_kernel<NC>, kWarps * 32, wunits), kWarps * 32, 0, s>>>( \
        pc->item_beg.get(), pc->item_len.get(), pc->nitems, pc->ofs_isort.get(), p->cs_hi_s.get(), p->cs_lo_s.get(), \
        mwd, partial)
        if (nc == 3) BM_OP(3); else if (nc == 2) BM_OP(2); else BM_OP(1);
#undef BM_OP
        BM_LAUNCH_CHECK();
    }
    finalize(ctx, pc->pitem.get(), partial, p->npix, nc, q);
#define BM_BM(NC) block_minus_kernel<NC><<<pgrid, threads, 0, s>>>(pc->B.get(), pc->mask.get(), x, p->npix, q)
    if (nc == 3) BM_BM(3); else if (nc == 2) BM_BM(2); else BM_BM(1);
#undef BM_BM
    BM_LAUNCH_CHECK();
}

// q = A x with the mixed operator of the offset template (see
// offset_means_f32_kernel).
static void offset_matvec_mixed(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int nc = p->ncomp;
    const int threads = 256;
    float4* x4 = workspace_as<float4>(ctx, "x4", p->npix);
    masked_copy4_kernel<<<grid_for(ctx, (p->npix + threads - 1) / threads, 16), threads, 0, s>>>(
        x, pc->mask.get(), p->npix, nc, x4);
    BM_LAUNCH_CHECK();
    float* mw = workspace_as<float>(ctx, "ofs_mw", std::max<int64_t>(n->nint, 1));
    if (n->nint > 0) {
        ScopedTimer timer(ctx, "offset_means_f32");
        const float2* trig_t = time_trig(p);  // built here on first use when deferred
        const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
        offset_means_f32_kernel<<<resident_grid(ctx, offset_means_f32_kernel, 256, (n->nint + 7) / 8), 256, 0, s>>>(
            pix_t, trig_t, x4, offset_geom(n), pc->ofs_inv.get(), n->white.get(), nc > 1, mw);
        BM_LAUNCH_CHECK();
    }
    double* partial = workspace_as<double>(ctx, "partial", (size_t)std::max<int64_t>(pc->nitems, 1) * nc);
    if (pc->nitems > 0) {
        ScopedTimer timer(ctx, "offset_matvec_f32");
        const int64_t wunits = (pc->nitems + kWarps - 1) / kWarps;
#define BM_OM(NC)                                                                                                      offset_matvec_f32_kernel<NC><<<resident_grid(ctx, offset_matvec_f32_kernel<NC>, kWarps * 32, wunits),                                             kWarps * 32, 0, s>>>(pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(),                                                         pc->nitems, pc->wcs.get(), pc->w1.get(),                                                                           pc->ofs_isort.get(), mw, x4, partial)
        if (nc == 3) BM_OM(3); else if (nc == 2) BM_OM(2); else BM_OM(1);
#undef BM_OM
        BM_LAUNCH_CHECK();
    }
    finalize(ctx, pc->pitem.get(), partial, p->npix, nc, q);
}

// inv_cnt = NULL: every sample is kept.
template <typename T, class Src, typename Out = T>
static void run_offset_filter(bm_inv_noise* n, const Src& src, const double* inv_cnt, Out* z) {
    bm_context* ctx = n->ctx;
    if (n->nint == 0) return;
    ScopedTimer timer(ctx, "offset_filter_f64");
    auto kern = offset_filter_kernel<T, Src, Out>;
    kern<<<resident_grid(ctx, kern, 256, (n->nint + 7) / 8), 256, 0, ctx->stream>>>(src, offset_geom(n),
                                                                                    n->white.get(), inv_cnt, z);
    BM_LAUNCH_CHECK();
}

// The time-ordered N^-1 of a non-diagonal model (a Toeplitz band or, in
// FP64, the offset filter) on the kept samples of the system `pc` belongs to.
template <class Src>
static void apply_filter_f32(bm_inv_noise* n, const bm_precond*, const Src& src, float* z) {
    apply_toeplitz_f32(n, src, z);  // the offset template's mixed operator is offset_matvec_mixed
}
template <class Src>
static void apply_filter_f64(bm_inv_noise* n, const bm_precond* pc, const Src& src, double* z) {
    if (n->kind == 3) run_offset_filter<double>(n, src, pc->ofs_inv.get(), z);
    else apply_toeplitz_f64(n, src, z);
}

static void finalize(bm_context* ctx, const int64_t* pitem, const double* partial, int64_t npix, int nc,
                     double* q) {
    const int threads = 256;
    finalize_pixels_kernel<<<grid_for(ctx, (npix + threads - 1) / threads, 16), threads, 0, ctx->stream>>>(
        pitem, partial, npix, nc, q);
    BM_LAUNCH_CHECK();
}

// q = P^T-style pixel sums of g[perm] (times w_d when `wn` is given) over the
// given items; lo = the sorted trig's lo part (or NULL to use hi exactly);
// df selects double-float instead of FP64 arithmetic.
struct ItemsView {
    const int32_t* pix;
    const int64_t* beg;
    const int32_t* len;
    int64_t n;
    const int64_t* pitem;
};
static ItemsView kept_items(const bm_precond* pc) {
    return {pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems, pc->pitem.get()};
}

static void gather_reduce_f32(bm_pointing* p, const ItemsView& it, const float* z, double* q) {
    bm_context* ctx = p->ctx;
    const int nc = p->ncomp;
    double* partial = workspace_as<double>(ctx, "partial", (size_t)std::max<int64_t>(it.n, 1) * nc);
    if (it.n > 0) {
        const int64_t wunits = (it.n + kWarps - 1) / kWarps;
#define BM_GR32(NC)                                                                                              \
    gather_reduce_f32_kernel<NC><<<resident_grid(ctx, gather_reduce_f32_kernel<NC>, kWarps * 32, wunits),      \
                                   kWarps * 32, 0, ctx->stream>>>(it.beg, it.len, it.n, p->perm.get(),         \
                                                                  p->cs_hi_s.get(), z, partial)
        if (nc == 3) BM_GR32(3); else if (nc == 2) BM_GR32(2); else BM_GR32(1);
#undef BM_GR32
        BM_LAUNCH_CHECK();
    }
    finalize(ctx, it.pitem, partial, p->npix, nc, q);
}

// The inner Toeplitz operator's transpose, time chunk by time chunk (see
// pt_chunk_kernel), over the chunk-major order of the kept samples; built on
// first use for an FFT-form filter unless its temporary tables would exceed
// kPtTableMaxBytes (then the plain pixel-sorted gather runs instead).
constexpr size_t kPtTableMaxBytes = size_t(1) << 32;
static void build_chunk_major(bm_pointing* p, bm_precond* pc, int nch) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t npix = p->npix;
    const int64_t ne = (int64_t)nch * npix;
    ScopedTimer timer(ctx, "toeplitz_pt_bounds");
    // sub[c][p]: position of pixel p's first sample in chunk c or later
    DevBuf<int32_t> sub((size_t)npix * (nch + 1));
    pt_bounds_kernel<<<grid_for(ctx, (npix + 7) / 8, 16), 256, 0, s>>>(p->off.get(), p->perm.get(), npix, nch,
                                                                     sub.get());
    BM_LAUNCH_CHECK();
    DevBuf<uint32_t> seglen(ne), segpos(ne), segidx(ne + 1);
    cm_seglen_kernel<<<grid_for(ctx, (ne + 255) / 256, 16), 256, 0, s>>>(sub.get(), pc->mask.get(), npix, nch,
                                                                         seglen.get(), segidx.get());
    BM_LAUNCH_CHECK();
    BM_CUDA(cudaMemsetAsync(segidx.get() + ne, 0, sizeof(uint32_t), s));
    exclusive_scan_u32(seglen.get(), segpos.get(), ne, s);
    exclusive_scan_u32(segidx.get(), segidx.get(), ne + 1, s);  // [ne] = the number of segments
    // chunk c's first segment is segidx[c * npix]; the kept samples are
    // segpos[ne - 1] + seglen[ne - 1]
    std::vector<uint32_t> h_first(nch + 1);
    for (int c = 0; c <= nch; ++c)
        BM_CUDA(cudaMemcpyAsync(&h_first[c], segidx.get() + (int64_t)c * npix, sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s));
    uint32_t last_pos = 0, last_len = 0;
    BM_CUDA(cudaMemcpyAsync(&last_pos, segpos.get() + ne - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaMemcpyAsync(&last_len, seglen.get() + ne - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    const int64_t nkept = (int64_t)last_pos + last_len;
    const int64_t nseg = h_first[nch];
    pc->cseg.assign(h_first.begin(), h_first.end());
    pc->cm_t.alloc(std::max<int64_t>(nkept, 1));
    pc->cm_cs.alloc(std::max<int64_t>(nkept, 1));
    pc->seg_pix.alloc(std::max<int64_t>(nseg, 1));
    pc->seg_beg.alloc(std::max<int64_t>(nseg, 1));
    pc->seg_len.alloc(std::max<int64_t>(nseg, 1));
    cm_scatter_kernel<<<grid_for(ctx, (npix + 7) / 8, 16), 256, 0, s>>>(p->off.get(), sub.get(), segpos.get(),
                                                                      pc->mask.get(), npix, p->perm.get(),
                                                                      p->cs_hi_s.get(), pc->cm_t.get(),
                                                                      pc->cm_cs.get());
    BM_LAUNCH_CHECK();
    cm_segments_kernel<<<grid_for(ctx, (ne + 255) / 256, 16), 256, 0, s>>>(seglen.get(), segpos.get(), segidx.get(),
                                                                            npix, nch, pc->seg_pix.get(),
                                                                            pc->seg_beg.get(), pc->seg_len.get());
    BM_LAUNCH_CHECK();
    // each segment's split at the middle of its chunk (the double-float
    // transpose runs half a chunk per launch)
    pc->seg_mid.alloc(std::max<int64_t>(nseg, 1));
    for (int c = 0; c < nch; ++c) {
        const int64_t seg0 = pc->cseg[c], n = pc->cseg[c + 1] - seg0;
        if (n == 0) continue;
        const uint64_t t_mid = ((uint64_t)c << kPtChunkBits) + (uint64_t(1) << (kPtChunkBits - 1));
        cm_seg_mid_kernel<<<grid_for(ctx, (n + 255) / 256, 16), 256, 0, s>>>(
            pc->seg_beg.get(), pc->seg_len.get(), seg0, n, (uint32_t)std::min<uint64_t>(t_mid, 0xFFFFFFFFull),
            pc->cm_t.get(), pc->seg_mid.get());
        BM_LAUNCH_CHECK();
    }
}

// True when the chunk-major order is (or has now been) built.
static bool ensure_chunk_major(bm_pointing* p, bm_inv_noise* n, bm_precond* pc) {
    if (pc->pt_nch == 0) {
        const int nch = (int)((p->nsamples + (int64_t(1) << kPtChunkBits) - 1) >> kPtChunkBits);
        // temporaries: the bounds table and three [nch][npix] tables
        if (n->fft_n32 == 0 || (size_t)p->npix * (size_t)(4 * nch + 2) * sizeof(int32_t) > kPtTableMaxBytes) {
            pc->pt_nch = -1;
        } else {
            build_chunk_major(p, pc, nch);
            pc->pt_nch = nch;
        }
    }
    return pc->pt_nch > 0;
}

// q = P^T z for double-float z pairs in time order (exact FP32 trig), by
// half chunks of the chunk-major order.
static void pt_chunked_df(bm_pointing* p, bm_precond* pc, const float2* z, double* q) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int nc = p->ncomp;
    const int64_t npix = p->npix;
    const int nch = pc->pt_nch;
    float2* acc = workspace_as<float2>(ctx, "pt_acc", (size_t)npix * nc);
    BM_CUDA(cudaMemsetAsync(acc, 0, sizeof(float2) * (size_t)npix * nc, s));
    for (int c = 0; c < nch; ++c) {
        const int64_t seg0 = pc->cseg[c], nseg = pc->cseg[c + 1] - seg0;
        if (nseg == 0) continue;
        const int64_t wunits = ((nseg + 32 / kPtLanes - 1) / (32 / kPtLanes) + kWarps - 1) / kWarps;
        for (int half = 0; half < 2; ++half) {
#define BM_PTD(NC)                                                                                              \
    pt_chunk_df_kernel<NC><<<resident_grid(ctx, pt_chunk_df_kernel<NC>, kWarps * 32, wunits), kWarps * 32, 0, s>>>( \
        pc->seg_pix.get(), pc->seg_beg.get(), pc->seg_len.get(), pc->seg_mid.get(), seg0, nseg, half,              \
        pc->cm_t.get(), pc->cm_cs.get(), z, acc)
            if (nc == 3) BM_PTD(3); else if (nc == 2) BM_PTD(2); else BM_PTD(1);
#undef BM_PTD
            BM_LAUNCH_CHECK();
        }
    }
    pt_finalize_kernel<<<grid_for(ctx, (npix + 255) / 256, 16), 256, 0, s>>>(acc, pc->mask.get(), npix, nc, q);
    BM_LAUNCH_CHECK();
}

// q = P^T z for z in time order, by chunks of the chunk-major order.
static void pt_chunked(bm_pointing* p, bm_precond* pc, const float* z, double* q) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int nc = p->ncomp;
    const int64_t npix = p->npix;
    const int nch = pc->pt_nch;
    float2* acc = workspace_as<float2>(ctx, "pt_acc", (size_t)npix * nc);
    BM_CUDA(cudaMemsetAsync(acc, 0, sizeof(float2) * (size_t)npix * nc, s));
    for (int c = 0; c < nch; ++c) {
        const int64_t seg0 = pc->cseg[c], nseg = pc->cseg[c + 1] - seg0;
        if (nseg == 0) continue;
        const int64_t wunits = ((nseg + 32 / kPtLanes - 1) / (32 / kPtLanes) + kWarps - 1) / kWarps;
#define BM_PT(NC)                                                                                                  \
    pt_chunk_kernel<NC><<<resident_grid(ctx, pt_chunk_kernel<NC>, kWarps * 32, wunits), kWarps * 32, 0, s>>>(       \
        pc->seg_pix.get(), pc->seg_beg.get(), pc->seg_len.get(), seg0, nseg, pc->cm_t.get(), pc->cm_cs.get(), z, acc)
        if (nc == 3) BM_PT(3); else if (nc == 2) BM_PT(2); else BM_PT(1);
#undef BM_PT
        BM_LAUNCH_CHECK();
    }
    pt_finalize_kernel<<<grid_for(ctx, (npix + 255) / 256, 16), 256, 0, s>>>(acc, pc->mask.get(), npix, nc, q);
    BM_LAUNCH_CHECK();
}

template <typename G>
static void gather_reduce(bm_pointing* p, const ItemsView& it, const G* g, const bm_inv_noise* wn,
                          const float2* lo, bool df, double* q, const float* gs = nullptr,
                          const bm_precond* wpc = nullptr) {
    bm_context* ctx = p->ctx;
    const int nc = p->ncomp;
    double* partial = workspace_as<double>(ctx, "partial", (size_t)std::max<int64_t>(it.n, 1) * nc);
    if (it.n > 0) {
        const int64_t wunits = (it.n + kWarps - 1) / kWarps;
        const bool weighted = wn != nullptr;
        // (wpc: the preconditioner holding the sorted weights of a noise
        // model with a weight per sample)
        const DetTables dt = weighted ? det_tables(wn, wpc) : DetTables{nullptr, nullptr, nullptr, 0u, 0.f};
        const double* white = weighted ? wn->white.get() : nullptr;
        const int ndet = weighted ? wn->ndet : 0;
#define BM_GR(NC, D)                                                                                           \
    gather_reduce_kernel<NC, G, D><<<resident_grid(ctx, gather_reduce_kernel<NC, G, D>, kWarps * 32, wunits), kWarps * 32, 0, ctx->stream>>>(it.pix, it.beg, it.len, it.n,          \
                                                                         p->perm.get(), p->cs_hi_s.get(), lo, g, gs, \
                                                                         weighted, dt, white, ndet, partial)
        if (df) {
            if (nc == 3) BM_GR(3, true); else if (nc == 2) BM_GR(2, true); else BM_GR(1, true);
        } else {
            if (nc == 3) BM_GR(3, false); else if (nc == 2) BM_GR(2, false); else BM_GR(1, false);
        }
#undef BM_GR
        BM_LAUNCH_CHECK();
    }
    finalize(ctx, it.pitem, partial, p->npix, nc, q);
}

void matvec(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const double* x, double* q,
            bm_precision prec, int64_t nrhs) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int nc = p->ncomp;
    const int64_t nvec = p->npix * nc;
    const int threads = 256;
    const int vgrid = grid_for(ctx, (nvec + threads - 1) / threads, 16);
    for (int64_t r = 0; r < nrhs; ++r) {
        const double* xr = x + r * nvec;
        double* qr = q + r * nvec;
        if (diagonal_noise(n)) {
            double* partial = workspace_as<double>(ctx, "partial", (size_t)std::max<int64_t>(pc->nitems, 1) * nc);
            const int64_t wunits = (pc->nitems + kWarps - 1) / kWarps;
            if (prec == BM_PREC_MIXED) {
                float* x32 = workspace_as<float>(ctx, "x32", nvec);
                masked_copy_kernel<float><<<vgrid, threads, 0, s>>>(xr, pc->mask.get(), p->npix, nc, x32);
                BM_LAUNCH_CHECK();
                if (pc->nitems > 0 && p->hwp && n->kind == 0 && nc > 1) {
                    // the angle rebuilt from the half-wave-plate model
                    ScopedTimer timer(ctx, "matvec_white_hwp");
#define BM_WHWP(NC)                                                                                                 \
    white_matvec_hwp_kernel<NC><<<resident_grid(ctx, white_matvec_hwp_kernel<NC>, kWarps * 32, wunits), kWarps * 32, \
                                  0, s>>>(pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems,   \
                                          p->perm.get(), p->hwp_model, p->hwp_tab.get(), n->wdf.get(), x32, partial)
                    if (nc == 3) BM_WHWP(3); else BM_WHWP(2);
#undef BM_WHWP
                    BM_LAUNCH_CHECK();
                } else if (pc->nitems > 0) {
                    ScopedTimer timer(ctx, "matvec_white_f32");
#define BM_WF32(NC)                                                                                     \
    white_matvec_f32_kernel<NC, float><<<resident_grid(ctx, white_matvec_f32_kernel<NC, float>, kWhiteWarps * 32, wunits), kWhiteWarps * 32, 0, s>>>( \
        pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems, pc->wcs.get(), pc->w1.get(), x32,    \
        partial)
                    if (nc == 3) BM_WF32(3); else if (nc == 2) BM_WF32(2); else BM_WF32(1);
#undef BM_WF32
                    BM_LAUNCH_CHECK();
                }
            } else if (pc->nitems > 0) {
                ScopedTimer timer(ctx, "matvec_white_f64");
#define BM_WF64(NC)                                                                                      \
    white_matvec_f64_kernel<NC><<<resident_grid(ctx, white_matvec_f64_kernel<NC>, kWarps * 32, wunits), kWarps * 32, 0, s>>>(                                              \
        pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems, p->perm.get(),            \
        p->cs_hi_s.get(), p->cs_lo_s.get(), n->det_off32.get(), n->ndet, n->ns_uniform, n->inv_ns, n->white.get(), \
        n->kind == 2 ? pc->ws64.get() : nullptr, xr, partial)
                if (nc == 3) BM_WF64(3); else if (nc == 2) BM_WF64(2); else BM_WF64(1);
#undef BM_WF64
                BM_LAUNCH_CHECK();
            }
            finalize(ctx, pc->pitem.get(), partial, p->npix, nc, qr);
        } else if (n->kind == 3 && prec == BM_PREC_MIXED) {
            offset_matvec_mixed(p, n, pc, xr, qr);
        } else if (n->kind == 3 && prec == kPrecRefine) {
            offset_matvec_refine(p, n, pc, xr, qr);
        } else {
            if (prec == BM_PREC_MIXED) {
                // the transpose by time chunks over the chunk-major order when
                // it can be built (FFT form), else the pixel-sorted gather
                const bool cm = ensure_chunk_major(p, n, pc);
                float* z32 = workspace_as<float>(ctx, "z32", p->nsamples);
                {
                    ScopedTimer timer(ctx, "toeplitz_f32");
                    float4* x4 = workspace_as<float4>(ctx, "x4", p->npix);
                    float* y32 = workspace_as<float>(ctx, "y32", p->nsamples);
                    {
                        ScopedTimer timer_px(ctx, "toeplitz_px");
                        masked_copy4_kernel<<<grid_for(ctx, (p->npix + threads - 1) / threads, 16), threads, 0,
                                              s>>>(xr, pc->mask.get(), p->npix, nc, x4);
                        BM_LAUNCH_CHECK();
                        // y = P x in its own full-occupancy pass (formed inside
                        // the FFT filter's load stage instead, its dependent map
                        // gather left the filter latency-bound: 15.8 -> 23.7 ms
                        // at config 2)
                        const float2* trig_t = time_trig(p);  // built here on first use when deferred
                        const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
                        pointing_apply_f32_kernel<<<grid_for(ctx, (p->nsamples + threads - 1) / threads, 16),
                                                    threads, 0, s>>>(pix_t, trig_t, p->nsamples,
                                                                     x4, y32);
                        BM_LAUNCH_CHECK();
                    }
                    apply_filter_f32(n, pc, SrcPlainF32{y32}, z32);
                }
                // scatter with the same FP32 trig the gather used (symmetric operator)
                ScopedTimer timer(ctx, "toeplitz_pt");
                if (cm) pt_chunked(p, pc, z32, qr);
                else gather_reduce_f32(p, kept_items(pc), z32, qr);
            } else if (prec == kPrecRefine) {
                // the refinement operator: P x, the filter and the pixel sums
                // in double-float on the FP32 pipes, no FP64 per sample
                float4* x2 = workspace_as<float4>(ctx, "x_df", 2 * p->npix);
                float2* z2 = workspace_as<float2>(ctx, "z_df", p->nsamples);
                masked_copy_df_kernel<<<grid_for(ctx, (p->npix + threads - 1) / threads, 16), threads, 0, s>>>(
                    xr, pc->mask.get(), p->npix, nc, x2);
                BM_LAUNCH_CHECK();
                {
                    ScopedTimer timer(ctx, "toeplitz_refine");
                    float2* y2 = workspace_as<float2>(ctx, "y_df", p->nsamples);
                    {
                        ScopedTimer timer_px(ctx, "toeplitz_px_df");
                        const float2* trig_t = time_trig(p);  // built here on first use when deferred
                        const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
                        pointing_apply_df_kernel<<<grid_for(ctx, (p->nsamples + threads - 1) / threads, 16),
                                                   threads, 0, s>>>(pix_t, trig_t,
                                                                    p->cs_lo_t.get(), p->nsamples, x2, y2);
                        BM_LAUNCH_CHECK();
                    }
                    apply_toeplitz_df(n, SrcPlainDF{y2}, z2);
                }
                ScopedTimer timer(ctx, "toeplitz_pt_df");
                if (p->cs_lo_s.get() == nullptr && ensure_chunk_major(p, n, pc)) pt_chunked_df(p, pc, z2, qr);
                else gather_reduce<float2>(p, kept_items(pc), z2, nullptr, p->cs_lo_s.get(), true, qr);
            } else {
                // FP64: P x, the filter and the pixel sums in FP64
                double* xm = workspace_as<double>(ctx, "xm", nvec);
                double* z64 = workspace_as<double>(ctx, "z64", p->nsamples);
                masked_copy_kernel<double><<<vgrid, threads, 0, s>>>(xr, pc->mask.get(), p->npix, nc, xm);
                BM_LAUNCH_CHECK();
                {
                    ScopedTimer timer(ctx, "toeplitz_f64");
                    double* y64 = workspace_as<double>(ctx, "y64", p->nsamples);
                    const float2* trig_t = time_trig(p);  // built here on first use when deferred
                    const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
                    pointing_apply_kernel<<<grid_for(ctx, (p->nsamples + threads - 1) / threads, 16), threads, 0, s>>>(
                        pix_t, trig_t, p->cs_lo_t.get(), p->nsamples, nc, xm, y64);
                    BM_LAUNCH_CHECK();
                    apply_filter_f64(n, pc, SrcPlain{y64}, z64);
                }
                ScopedTimer timer(ctx, "toeplitz_pt");
                gather_reduce<double>(p, kept_items(pc), z64, nullptr, p->cs_lo_s.get(), false, qr);
            }
        }
        shard_reduce(ctx, qr, nvec);  // a shard's partial A x, summed over the ranks
    }
}

void rhs(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod, bm_dtype dt, int64_t nrhs,
         double* b, bool df) {
    bm_context* ctx = p->ctx;
    const int nc = p->ncomp;
    const int64_t nvec = p->npix * nc;
    ScopedTimer timer(ctx, "rhs");
    for (int64_t r = 0; r < nrhs; ++r) {
        double* br = b + r * nvec;
        if (diagonal_noise(n)) {
            if (!tod && df && pc->b_tod.get()) {  // assembled (and summed over the ranks) with the blocks
                BM_CUDA(cudaMemcpyAsync(br, pc->b_tod.get(), sizeof(double) * nvec, cudaMemcpyDeviceToDevice,
                                        ctx->stream));
                continue;
            } else if (!tod) {  // the TOD sorted along with the pointing
                gather_reduce<float>(p, kept_items(pc), nullptr, n, p->cs_lo_s.get(), df, br, p->tod_s.get(), pc);
            } else if (dt == BM_F32) {
                const float* d = static_cast<const float*>(tod) + r * p->nsamples;
                gather_reduce<float>(p, kept_items(pc), d, n, p->cs_lo_s.get(), df, br, nullptr, pc);
            } else {
                const double* d = static_cast<const double*>(tod) + r * p->nsamples;
                gather_reduce<double>(p, kept_items(pc), d, n, p->cs_lo_s.get(), df, br, nullptr, pc);
            }
        } else if (n->kind == 3 && df) {
            // the offset template's double-float RHS: z as double-float pairs
            float2* z2 = workspace_as<float2>(ctx, "z2", p->nsamples);
            if (dt == BM_F32) {
                SrcMaskedTod<float> src{time_pix(p), pc->mask.get(),
                                        static_cast<const float*>(tod) + r * p->nsamples};
                run_offset_filter<double, SrcMaskedTod<float>, float2>(n, src, pc->ofs_inv.get(), z2);
            } else {
                SrcMaskedTod<double> src{time_pix(p), pc->mask.get(),
                                         static_cast<const double*>(tod) + r * p->nsamples};
                run_offset_filter<double, SrcMaskedTod<double>, float2>(n, src, pc->ofs_inv.get(), z2);
            }
            gather_reduce<float2>(p, kept_items(pc), z2, nullptr, p->cs_lo_s.get(), true, br);
        } else if (df && n->kind == 1) {
            // the mixed path's Toeplitz RHS: filter and pixel sums in
            // double-float, z as (hi, lo) pairs
            float2* z2 = workspace_as<float2>(ctx, "z_df", p->nsamples);
            float2* y2 = workspace_as<float2>(ctx, "y_df", p->nsamples);
            const int tthreads = 256;
            const int tgrid = grid_for(ctx, (p->nsamples + tthreads - 1) / tthreads, 16);
            const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
            if (dt == BM_F32)
                masked_tod_df_kernel<float><<<tgrid, tthreads, 0, ctx->stream>>>(
                    pix_t, pc->mask.get(), static_cast<const float*>(tod) + r * p->nsamples, p->nsamples, y2);
            else
                masked_tod_df_kernel<double><<<tgrid, tthreads, 0, ctx->stream>>>(
                    pix_t, pc->mask.get(), static_cast<const double*>(tod) + r * p->nsamples, p->nsamples, y2);
            BM_LAUNCH_CHECK();
            apply_toeplitz_df(n, SrcPlainDF{y2}, z2);
            if (p->cs_lo_s.get() == nullptr && ensure_chunk_major(p, n, pc)) pt_chunked_df(p, pc, z2, br);
            else gather_reduce<float2>(p, kept_items(pc), z2, nullptr, p->cs_lo_s.get(), true, br);
        } else {
            double* z64 = workspace_as<double>(ctx, "z64", p->nsamples);
            if (dt == BM_F32) {
                SrcMaskedTod<float> src{time_pix(p), pc->mask.get(),
                                        static_cast<const float*>(tod) + r * p->nsamples};
                apply_filter_f64(n, pc, src, z64);
            } else {
                SrcMaskedTod<double> src{time_pix(p), pc->mask.get(),
                                         static_cast<const double*>(tod) + r * p->nsamples};
                apply_filter_f64(n, pc, src, z64);
            }
            gather_reduce<double>(p, kept_items(pc), z64, nullptr, p->cs_lo_s.get(), df, br);
        }
        shard_reduce(ctx, br, nvec);  // a shard's partial b, summed over the ranks
    }
}

void pointing_apply(bm_pointing* p, const double* x, double* y) {
    bm_context* ctx = p->ctx;
    const int threads = 256;
    const float2* trig_t = time_trig(p);  // built here on first use when deferred
    const int32_t* pix_t = time_pix(p);  // built here on first use when deferred
    pointing_apply_kernel<<<grid_for(ctx, (p->nsamples + threads - 1) / threads, 16), threads, 0, ctx->stream>>>(
        pix_t, trig_t, p->cs_lo_t.get(), p->nsamples, p->ncomp, x, y);
    BM_LAUNCH_CHECK();
}

void pointing_apply_transpose(bm_pointing* p, const double* y, double* x) {
    Items it;
    plan_items(p->ctx, p->off.get(), nullptr, p->npix, it);
    const ItemsView v{it.pix.get(), it.beg.get(), it.len.get(), it.n, it.pitem.get()};
    gather_reduce<double>(p, v, y, nullptr, p->cs_lo_s.get(), false, x);
    shard_reduce(p->ctx, x, p->npix * p->ncomp);
    BM_CUDA(cudaStreamSynchronize(p->ctx->stream));
}

// z_t = w_t y_t for a weight per sample.
__global__ void sample_weight_apply_kernel(const double* __restrict__ w, const double* __restrict__ y, int64_t n,
                                           double* __restrict__ z) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        z[t] = w[t] * y[t];
}

void inv_noise_apply(bm_inv_noise* n, const double* y, double* z) {
    bm_context* ctx = n->ctx;
    if (n->kind == 2) {
        sample_weight_apply_kernel<<<grid_for(ctx, (n->nsamples + 255) / 256, 16), 256, 0, ctx->stream>>>(
            n->wsamp.get(), y, n->nsamples, z);
        BM_LAUNCH_CHECK();
    } else if (n->kind == 0) {
        // z_t = w_d y_t: reuse the Toeplitz machinery with a single lag.
        DevBuf<double> c(n->ndet);
        BM_CUDA(cudaMemcpyAsync(c.get(), n->white.get(), sizeof(double) * n->ndet, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        bm_inv_noise tmp;
        tmp.ctx = ctx;
        tmp.ndet = n->ndet;
        tmp.nsamples = n->nsamples;
        tmp.h_det_off = n->h_det_off;
        tmp.det_off.alloc(n->ndet + 1);
        BM_CUDA(cudaMemcpyAsync(tmp.det_off.get(), n->det_off.get(), sizeof(int64_t) * (n->ndet + 1),
                                cudaMemcpyDeviceToDevice, ctx->stream));
        tmp.chunk_len = n->nsamples;
        tmp.nlags = 1;
        run_toeplitz<double, 4>(&tmp, SrcPlain{y}, c.get(), z);
    } else if (n->kind == 3) {
        run_offset_filter<double>(n, SrcPlain{y}, nullptr, z);
    } else {
        apply_toeplitz_f64(n, SrcPlain{y}, z);
    }
}

}  // namespace bm
