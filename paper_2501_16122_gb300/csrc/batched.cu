// Multi-RHS GLS solve for white noise: R right-hand sides that share one
// pointing (noise or signal realisations), solved together so that every
// pass over the pointing serves all R of them.
//
// Layout: vectors are RHS-interleaved, [npix][ncomp][R] (per pixel and
// Stokes component the R right-hand sides are contiguous, so a warp over
// right-hand sides reads and writes whole lines).  The caller's TOD
// [R][nsamples] is transposed group by group (G <= 32 * RPL right-hand sides,
// RPL = 1 or 2 a lane, the group size timed once per problem shape) into
// [nsamples][G], so that the pixel-sorted gather of one sample reads G
// contiguous values.
//
// Kernels (one warp per work item, lanes over right-hand sides, RPL per lane):
//   batched_rhs:    b_{p,r} = sum_{t in p} w_d d_r[t] v_t   (double-float,
//                   lazily renormalised as the single-RHS gather-reduce)
//   batched_matvec: q_{p,r} = sum_{t in p} u_t (u_t . x_{p,r}) with the FP32
//                   weighted stream u_t = sqrt(w)(1?, cos, sin): FP32 products,
//                   compensated (double-float) sums
// A pixel with a single work item writes its result directly; pixels with
// several items write item partials that a per-pixel pass sums in item order
// (deterministic).
//
// PCG: per-RHS FP64 scalars on the device, per-RHS done flags; the inner
// loop is one CUDA graph with a WHILE node (one inner iteration per pass,
// matvec + dots + updates, ended on the device when every RHS is done or an
// iteration limit is reached), captured once per solve on the context's side
// stream; the host reads the RHS states once per outer iteration.  Mixed
// precision with iterative refinement: outer residual r = b - B x per pixel
// in FP64 (for white noise
// A equals the block-diagonal matrix B of Eq. 7).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int kRB = 2048;  // most blocks of the per-pixel PCG kernels (a full wave: enough loads in flight for HBM)
constexpr int kRT = 256;   // threads per reduction block

struct RhsState {
    double rho, rr, bb, pq, alpha, beta, tol2;
    int done;   // 1 converged, 2 breakdown
    int iters;
};

// ---------------------------------------------------------------- transpose
template <typename T>
__global__ void transpose_group_kernel(const T* const* __restrict__ rows, int64_t n, int r0, int G,
                                       T* __restrict__ out) {
    __shared__ T tile[32][33];
    const int rt = blockIdx.y * 32;
    for (int64_t t0 = (int64_t)blockIdx.x * 32; t0 < n; t0 += (int64_t)gridDim.x * 32) {
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int r = rt + yy;
            const int64_t t = t0 + threadIdx.x;
            tile[yy][threadIdx.x] = (r < G && t < n) ? rows[r0 + r][t] : T(0);
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int64_t t = t0 + yy;
            const int r = rt + threadIdx.x;
            if (t < n && r < G) out[t * G + r] = tile[threadIdx.x][yy];
        }
        __syncthreads();
    }
}

// FP32 rows -> [n][G] (G <= 64) by tiles of kTT samples x G rows staged in
// shared memory: each row's samples are loaded as float4 runs (streaming,
// read once), and the tile's output, one contiguous block of kTT G floats,
// is stored as float4 runs.  Rows must start on 16-byte boundaries.
constexpr int kTT = 128;

__global__ void __launch_bounds__(256) transpose_f32x4_kernel(const float* const* __restrict__ rows, int64_t n, int r0,
                                                              int G, float* __restrict__ out) {
    __shared__ float tile[64][kTT + 1];
    for (int64_t t0 = (int64_t)blockIdx.x * kTT; t0 < n; t0 += (int64_t)gridDim.x * kTT) {
        const int cnt = (int)min((int64_t)kTT, n - t0);
        for (int i = threadIdx.x; i < G * (kTT / 4); i += blockDim.x) {
            const int r = i / (kTT / 4), c = (i % (kTT / 4)) * 4;
            const float* src = rows[r0 + r] + t0 + c;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c + 4 <= cnt) {
                v = __ldcs(reinterpret_cast<const float4*>(src));
            } else {
                if (c < cnt) v.x = src[0];
                if (c + 1 < cnt) v.y = src[1];
                if (c + 2 < cnt) v.z = src[2];
            }
            tile[r][c] = v.x;
            tile[r][c + 1] = v.y;
            tile[r][c + 2] = v.z;
            tile[r][c + 3] = v.w;
        }
        __syncthreads();
        float* dst = out + t0 * G;
        const int total = cnt * G;
        for (int j = threadIdx.x * 4; j < total; j += blockDim.x * 4) {
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = j + k;
                const int tt = G == 32 ? (e >> 5) : (G == 64 ? (e >> 6) : e / G);
                v[k] = e < total ? tile[e - tt * G][tt] : 0.f;
            }
            if (j + 4 <= total) {
                *reinterpret_cast<float4*>(dst + j) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                for (int k = 0; k < 4 && j + k < total; ++k) dst[j + k] = v[k];
            }
        }
        __syncthreads();
    }
}

// Destination of item k's values for RHS r: the output itself when the item
// is its pixel's only item, else the item's partial slot.
__device__ __forceinline__ double* item_dst(const int64_t* pitem, int64_t p, int64_t k, int R, int NC, int r,
                                            double* out, double* partial) {
    if (pitem[p + 1] - pitem[p] == 1) return out + (int64_t)p * NC * R + r;
    return partial + (int64_t)k * NC * R + r;
}

// ---------------------------------------------------------------- batched RHS
template <int NC, typename T, int RPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
batched_rhs_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                   const int32_t* __restrict__ item_len, int64_t nitems, const int64_t* __restrict__ pitem,
                   const uint32_t* __restrict__ perm, const float2* __restrict__ hi, const float2* __restrict__ lo,
                   const T* __restrict__ dT, int G, int r0, int R, DetTables dt, int ndet,
                   double* __restrict__ out, double* __restrict__ partial) {
    // the detector tables, staged when they fit (sized by the launch)
    extern __shared__ __align__(16) unsigned char rhs_smem[];
    float2* s_w = reinterpret_cast<float2*>(rhs_smem);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(rhs_smem + sizeof(float2) * (size_t)ndet);
    const bool in_smem = ndet <= kMaxDetSmem;
    if (in_smem) {
        for (int d = threadIdx.x; d <= ndet; d += blockDim.x) s_off[d] = dt.off[d];
        for (int d = threadIdx.x; d < ndet; d += blockDim.x) s_w[d] = dt.wdf[d];
    }
    __syncthreads();
    const uint32_t* offp = in_smem ? s_off : dt.off;
    const float2* wp = in_smem ? s_w : dt.wdf;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    for (int64_t k = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        df32 acc[RPL][NC];
#pragma unroll
        for (int q = 0; q < RPL; ++q)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[q][c] = {0.f, 0.f};
        int nadd = 0;
        for (int base = 0; base < len; base += 32) {
            const int j = base + lane;
            const bool valid = j < len;
            uint32_t tl = 0;
            float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f), wl = make_float2(0.f, 0.f);
            if (valid) {
                tl = perm[b + j];
                h = hi[b + j];
                if (lo) l = lo[b + j];
                wl = wp[det_of(offp, ndet, dt.ns, dt.inv_ns, tl)];
            }
            const int cnt = min(32, len - base);
            // sample kk of the chunk: its row of the G right-hand sides, added
            // in order in the lazily renormalised form (rhs_term_lazy)
            auto add = [&](int kk, const T (&dv)[RPL]) {
                const float2 w = {__shfl_sync(0xffffffffu, wl.x, kk), __shfl_sync(0xffffffffu, wl.y, kk)};
                const float2 hh = {__shfl_sync(0xffffffffu, h.x, kk), __shfl_sync(0xffffffffu, h.y, kk)};
                const float2 ll = {__shfl_sync(0xffffffffu, l.x, kk), __shfl_sync(0xffffffffu, l.y, kk)};
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    if (lane + 32 * q < G) {
                        df32 d;
                        if (sizeof(T) == 4) d = {(float)dv[q], 0.f};
                        else d = df_from((double)dv[q]);
                        rhs_term_lazy<NC>(acc[q], d.hi, d.lo, true, w, hh, ll);
                    }
                }
                if (++nadd == kLazyNorm) {
                    nadd = 0;
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
#pragma unroll
                        for (int c = 0; c < NC; ++c) acc_norm(acc[q][c]);
                }
            };
            auto row = [&](int kk, T (&dv)[RPL]) {
                const uint32_t t = __shfl_sync(0xffffffffu, tl, kk);
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const int r = lane + 32 * q;
                    dv[q] = r < G ? dT[(int64_t)t * G + r] : T(0);
                }
            };
            // sixteen (one RHS a lane) or eight rows in flight, then their
            // sums in sample order
            constexpr int U = 16 / RPL;
            int kk = 0;
            for (; kk + U <= cnt; kk += U) {
                T dv[U][RPL];
#pragma unroll
                for (int u = 0; u < U; ++u) row(kk + u, dv[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) add(kk + u, dv[u]);
            }
            for (; kk + 4 <= cnt; kk += 4) {
                T dv[4][RPL];
#pragma unroll
                for (int u = 0; u < 4; ++u) row(kk + u, dv[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) add(kk + u, dv[u]);
            }
            for (; kk < cnt; ++kk) {
                T dv[RPL];
                row(kk, dv);
                add(kk, dv);
            }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            if (r < G) {
                double* dst = item_dst(pitem, p, k, R, NC, r0 + r, out, partial);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    acc_norm(acc[q][c]);
                    dst[(int64_t)c * R] = df_to_double(acc[q][c]);
                }
            }
        }
    }
}

// ------------------------------------------------------------- batched matvec
template <int NC, int RPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
batched_matvec_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                      const int32_t* __restrict__ item_len, int64_t nitems, const int64_t* __restrict__ pitem,
                      const float2* __restrict__ wcs, const float* __restrict__ w1,
                      const float* __restrict__ x32, int r0, int G, int R, double* __restrict__ out,
                      double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    for (int64_t k = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        float xv[RPL][NC];
        float g[RPL][NC];
        df32 A[RPL][NC];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                xv[q][c] = r < G ? x32[((int64_t)p * NC + c) * R + r0 + r] : 0.f;
                g[q][c] = 0.f;
                A[q][c] = {0.f, 0.f};
            }
        }
        for (int base = 0; base < len; base += 32) {
            const int j = base + lane;
            float2 ul = make_float2(0.f, 0.f);
            float wl = 0.f;
            if (j < len) {
                if (NC == 1) wl = w1[b + j];
                else ul = wcs[b + j];
            }
            const int cnt = min(32, len - base);
            for (int kk = 0; kk < cnt; ++kk) {
                if (NC == 1) {
                    const float w = __shfl_sync(0xffffffffu, wl, kk);
#pragma unroll
                    for (int q = 0; q < RPL; ++q) g[q][0] = fmaf(w, xv[q][0], g[q][0]);
                } else {
                    const float ux = __shfl_sync(0xffffffffu, ul.x, kk);
                    const float uy = __shfl_sync(0xffffffffu, ul.y, kk);
                    float rr = 0.f;
                    if (NC == 3) {
                        const float u2 = fmaf(ux, ux, uy * uy);
                        rr = u2 > 0.f ? u2 * rsqrtf(u2) : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < RPL; ++q) {
                        float y = fmaf(ux, xv[q][NC - 2], uy * xv[q][NC - 1]);
                        if (NC == 3) {
                            y = fmaf(rr, xv[q][0], y);
                            g[q][0] = fmaf(y, rr, g[q][0]);
                        }
                        g[q][NC - 2] = fmaf(y, ux, g[q][NC - 2]);
                        g[q][NC - 1] = fmaf(y, uy, g[q][NC - 1]);
                    }
                }
                if ((kk & 7) == 7) {  // fold the FP32 group into the compensated sums
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
#pragma unroll
                        for (int c = 0; c < NC; ++c) { A[q][c] = df_add(A[q][c], g[q][c]); g[q][c] = 0.f; }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int r = lane + 32 * q;
            if (r < G) {
                double* dst = item_dst(pitem, p, k, R, NC, r0 + r, out, partial);
#pragma unroll
                for (int c = 0; c < NC; ++c) dst[(int64_t)c * R] = df_to_double(df_add(A[q][c], g[q][c]));
            }
        }
    }
}

// Pixels with several items: sum the partials (item order); pixels without
// items (masked or empty): zero.  Single-item pixels were written directly.
__global__ void batched_finalize_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ partial,
                                        int64_t npix, int RNC, double* __restrict__ out) {
    const int64_t n = npix * RNC;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / RNC;
        const int64_t e = i - p * RNC;
        const int64_t k0 = pitem[p], k1 = pitem[p + 1];
        if (k1 - k0 == 1) continue;
        double s = 0.0;
        for (int64_t k = k0; k < k1; ++k) s += partial[k * RNC + e];
        out[i] = s;
    }
}

// [npix][NC][R] FP64 -> FP32 with masked pixels zeroed.
__global__ void batched_masked_f32_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask,
                                          int64_t npix, int RNC, float* __restrict__ out) {
    const int64_t n = npix * RNC;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = mask[i / RNC] ? 0.f : (float)x[i];
}

// ---------------------------------------------------------------- PCG pieces
// Thread layout of the per-pixel kernels: blockDim = kRT, Rp = R rounded up
// to a power of two <= kRT, ppb = kRT / Rp pixels per block pass; thread
// (sub, r) handles RHS r of pixel blk * ppb + sub + pass * gridDim * ppb.
// Per-RHS partial sums go to part[blk * R + r] (fixed order everywhere).
struct BGeo {
    int R, Rp, ppb;
    int64_t npix;
};

__device__ __forceinline__ void block_rhs_reduce(double v, double* sh, const BGeo& g, double* part, int slot) {
    sh[threadIdx.x] = v;
    __syncthreads();
    const int r = threadIdx.x % g.Rp;
    const int sub = threadIdx.x / g.Rp;
    if (sub == 0 && r < g.R) {
        double s = 0.0;
        for (int q = 0; q < g.ppb; ++q) s += sh[q * g.Rp + r];
        part[((int64_t)slot * gridDim.x + blockIdx.x) * g.R + r] = s;
    }
    __syncthreads();
}

template <int NC>
__device__ __forceinline__ void apply_block(const double* __restrict__ M, int64_t p, const double* v, double* o) {
    const double* m = M + p * NC * NC;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NC; ++j) s += m[i * NC + j] * v[j];
        o[i] = s;
    }
}

// r = b - B x (masked pixels 0); XZ: x = 0 (the start: r = b, no block
// products, which cost GB300's FP64 pipe most of this kernel's time);
// part slot 0: r.r, slot 1: b.b
template <int NC, bool XZ>
__global__ void __launch_bounds__(kRT) b_residual_kernel(BGeo g, const double* __restrict__ B, const uint8_t* __restrict__ mask,
                                                        const double* __restrict__ b, const double* __restrict__ x,
                                                        double* __restrict__ r, double* __restrict__ part) {
    __shared__ double sh[kRT];
    const int rr_ = threadIdx.x % g.Rp, sub = threadIdx.x / g.Rp;
    double s_rr = 0.0, s_bb = 0.0;
    if (rr_ < g.R) {
        for (int64_t p = (int64_t)blockIdx.x * g.ppb + sub; p < g.npix; p += (int64_t)gridDim.x * g.ppb) {
            const int64_t o = p * NC * g.R + rr_;
            double bx[NC];
            if (XZ) {
#pragma unroll
                for (int c = 0; c < NC; ++c) bx[c] = 0.0;
            } else {
                double xv[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) xv[c] = x[o + c * g.R];
                apply_block<NC>(B, p, xv, bx);
            }
            const bool keep = mask[p] == 0;
            double bl[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) bl[c] = b[o + c * g.R];  // not behind the mask load
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const double bv = keep ? bl[c] : 0.0;
                const double v = keep ? bv - bx[c] : 0.0;
                r[o + c * g.R] = v;
                s_rr += v * v;
                s_bb += bv * bv;
            }
        }
    }
    block_rhs_reduce(s_rr, sh, g, part, 0);
    block_rhs_reduce(s_bb, sh, g, part, 1);
}

// Start of an inner PCG on A e = rin: e = 0, rcg = rin, z = M rin, p = z;
// part slots: 0 r.z, 1 r.r
template <int NC>
__global__ void __launch_bounds__(kRT) b_init_kernel(BGeo g, const double* __restrict__ M, const double* __restrict__ rin,
                                                    double* __restrict__ e, double* __restrict__ rcg, double* __restrict__ z,
                                                    double* __restrict__ pv, double* __restrict__ part) {
    __shared__ double sh[kRT];
    const int rr_ = threadIdx.x % g.Rp, sub = threadIdx.x / g.Rp;
    double s_rz = 0.0, s_rr = 0.0;
    if (rr_ < g.R) {
        for (int64_t p = (int64_t)blockIdx.x * g.ppb + sub; p < g.npix; p += (int64_t)gridDim.x * g.ppb) {
            const int64_t o = p * NC * g.R + rr_;
            double rv[NC], zv[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) rv[c] = rin[o + c * g.R];
            apply_block<NC>(M, p, rv, zv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                e[o + c * g.R] = 0.0;
                rcg[o + c * g.R] = rv[c];
                z[o + c * g.R] = zv[c];
                pv[o + c * g.R] = zv[c];
                s_rz += rv[c] * zv[c];
                s_rr += rv[c] * rv[c];
            }
        }
    }
    block_rhs_reduce(s_rz, sh, g, part, 0);
    block_rhs_reduce(s_rr, sh, g, part, 1);
}

// One thread per RHS: sum the per-block partials in block order.
__global__ void b_init_finalize(const double* __restrict__ part, int nblk, int R, const double* __restrict__ tolr,
                                RhsState* __restrict__ st) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double rz = 0.0, rr = 0.0;
    for (int b = 0; b < nblk; ++b) {
        rz += part[(int64_t)b * R + r];
        rr += part[((int64_t)nblk + b) * R + r];
    }
    RhsState s{};
    s.rho = rz;
    s.rr = rr;
    s.tol2 = tolr[r];
    s.done = (rr <= s.tol2) ? 1 : 0;
    s.iters = 0;
    st[r] = s;
}

__global__ void __launch_bounds__(kRT) b_dot_kernel(BGeo g, int NCr, const double* __restrict__ a, const double* __restrict__ b,
                                                   double* __restrict__ part) {
    __shared__ double sh[kRT];
    const int rr_ = threadIdx.x % g.Rp, sub = threadIdx.x / g.Rp;
    double s = 0.0;
    if (rr_ < g.R) {
        for (int64_t p = (int64_t)blockIdx.x * g.ppb + sub; p < g.npix; p += (int64_t)gridDim.x * g.ppb) {
            const int64_t o = p * NCr * g.R + rr_;
            for (int c = 0; c < NCr; ++c) s += a[o + c * g.R] * b[o + c * g.R];
        }
    }
    block_rhs_reduce(s, sh, g, part, 0);
}

__global__ void b_alpha_kernel(const double* __restrict__ part, int nblk, int R, RhsState* __restrict__ st) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || st[r].done) return;
    double pq = 0.0;
    for (int b = 0; b < nblk; ++b) pq += part[(int64_t)b * R + r];
    st[r].pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) st[r].done = 2;
    else st[r].alpha = st[r].rho / pq;
}

// e += alpha p; r -= alpha q; z = M r; slots 0 r.r, 1 r.z (done RHS untouched)
template <int NC>
__global__ void __launch_bounds__(kRT) b_update_kernel(BGeo g, const double* __restrict__ M, double* __restrict__ e,
                                                      double* __restrict__ rcg, double* __restrict__ z,
                                                      const double* __restrict__ pv, const double* __restrict__ q,
                                                      const RhsState* __restrict__ st, double* __restrict__ part) {
    __shared__ double sh[kRT];
    const int rr_ = threadIdx.x % g.Rp, sub = threadIdx.x / g.Rp;
    double s_rr = 0.0, s_rz = 0.0;
    if (rr_ < g.R && !st[rr_].done) {
        const double alpha = st[rr_].alpha;
        for (int64_t p = (int64_t)blockIdx.x * g.ppb + sub; p < g.npix; p += (int64_t)gridDim.x * g.ppb) {
            const int64_t o = p * NC * g.R + rr_;
            double rv[NC], zv[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                e[o + c * g.R] += alpha * pv[o + c * g.R];
                rv[c] = rcg[o + c * g.R] - alpha * q[o + c * g.R];
                rcg[o + c * g.R] = rv[c];
            }
            apply_block<NC>(M, p, rv, zv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                z[o + c * g.R] = zv[c];
                s_rr += rv[c] * rv[c];
                s_rz += rv[c] * zv[c];
            }
        }
    }
    block_rhs_reduce(s_rr, sh, g, part, 0);
    block_rhs_reduce(s_rz, sh, g, part, 1);
}

__global__ void b_beta_kernel(const double* __restrict__ part, int nblk, int R, RhsState* __restrict__ st) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || st[r].done) return;
    double rr = 0.0, rz = 0.0;
    for (int b = 0; b < nblk; ++b) {
        rr += part[(int64_t)b * R + r];
        rz += part[((int64_t)nblk + b) * R + r];
    }
    RhsState s = st[r];
    s.rr = rr;
    s.iters += 1;
    if (rr <= s.tol2) s.done = 1;
    else if (!isfinite(rr) || !isfinite(rz)) s.done = 2;
    else { s.beta = rz / s.rho; s.rho = rz; }
    st[r] = s;
}

__global__ void __launch_bounds__(kRT) b_pupdate_kernel(BGeo g, int NCr, double* __restrict__ pv, const double* __restrict__ z,
                                                       const RhsState* __restrict__ st) {
    const int rr_ = threadIdx.x % g.Rp, sub = threadIdx.x / g.Rp;
    if (rr_ >= g.R || st[rr_].done) return;
    const double beta = st[rr_].beta;
    for (int64_t p = (int64_t)blockIdx.x * g.ppb + sub; p < g.npix; p += (int64_t)gridDim.x * g.ppb) {
        const int64_t o = p * NCr * g.R + rr_;
        for (int c = 0; c < NCr; ++c) pv[o + c * g.R] = z[o + c * g.R] + beta * pv[o + c * g.R];
    }
}

__global__ void b_axpy_kernel(double* __restrict__ x, const double* __restrict__ e, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += e[i];
}

// Per-RHS sums of slots 0 and 1 into host-visible out[2R].
__global__ void b_sum2_kernel(const double* __restrict__ part, int nblk, int R, double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblk; ++k) {
        a += part[(int64_t)k * R + r];
        b += part[((int64_t)nblk + k) * R + r];
    }
    out[r] = a;
    out[R + r] = b;
}

// maps[r][p][c] = x[p][r][c] (NaN on masked pixels), by tiles of P pixels:
// the tile's block of x (P R NC contiguous values) is staged in shared memory
// and each map's P NC contiguous values are written as one run.
__global__ void b_write_map_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask, int64_t npix,
                                   int R, int NC, int P, double* const* __restrict__ maps) {
    extern __shared__ double map_tile[];  // [P R NC]
    const int per = R * NC;
    const int64_t ntiles = (npix + P - 1) / P;
    for (int64_t tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const int64_t p0 = tb * P;
        const int np = (int)(npix - p0 < P ? npix - p0 : P);
        const double* src = x + p0 * per;
        for (int i = threadIdx.x; i < np * per; i += blockDim.x) map_tile[i] = src[i];
        __syncthreads();
        const int run = np * NC;
        for (int i = threadIdx.x; i < R * run; i += blockDim.x) {
            const int r = i / run, j = i - r * run;
            const int pl = j / NC, c = j - pl * NC;
            maps[r][(p0 + pl) * NC + c] = mask[p0 + pl] ? NAN : map_tile[(pl * NC + c) * R + r];
        }
        __syncthreads();
    }
}

// Inner-loop control for the WHILE node of the batched solve: loop[0]
// counts the iterations run by the current graph launch (inc = 1 after an
// iteration, 0 before the first), loop[1] is their limit; the node goes on
// while any right-hand side is active and the limit is not reached.
__global__ void b_loop_kernel(const RhsState* __restrict__ st, int R, int* __restrict__ loop, int inc,
                              cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = loop[0] + inc;
    loop[0] = it;
    bool active = false;
    for (int r = 0; r < R; ++r) active = active || st[r].done == 0;
    cudaGraphSetConditional(h, (active && it < loop[1]) ? 1u : 0u);
}

// ------------------------------------------------------------------ launchers
struct Variant {
    int rpl, warps;
};

template <int NC, int RPL, int W>
void launch_matvec_v(bm_context* ctx, bm_precond* pc, const float* x32, int r0, int G, int R, double* q,
                     double* partial) {
    auto kern = batched_matvec_kernel<NC, RPL, W>;
    const int grid = resident_grid(ctx, kern, W * 32, (pc->nitems + W - 1) / W);
    kern<<<grid, W * 32, 0, ctx->stream>>>(pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems,
                                           pc->pitem.get(), pc->wcs.get(), pc->w1.get(), x32, r0, G, R, q, partial);
    BM_LAUNCH_CHECK();
}

template <int NC>
void launch_matvec(bm_context* ctx, bm_precond* pc, Variant v, const float* x32, int r0, int G, int R, double* q,
                   double* partial) {
    if (v.rpl == 1) {
        if (v.warps == 4) launch_matvec_v<NC, 1, 4>(ctx, pc, x32, r0, G, R, q, partial);
        else launch_matvec_v<NC, 1, 8>(ctx, pc, x32, r0, G, R, q, partial);
    } else if (v.rpl == 2) {
        if (v.warps == 4) launch_matvec_v<NC, 2, 4>(ctx, pc, x32, r0, G, R, q, partial);
        else launch_matvec_v<NC, 2, 8>(ctx, pc, x32, r0, G, R, q, partial);
    } else {
        if (v.warps == 4) launch_matvec_v<NC, 4, 4>(ctx, pc, x32, r0, G, R, q, partial);
        else launch_matvec_v<NC, 4, 8>(ctx, pc, x32, r0, G, R, q, partial);
    }
}

template <int NC, typename T, int RPL>
void launch_rhs_v(bm_context* ctx, bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const T* dT, int G, int r0,
                  int R, double* b, double* partial, bool exact_lo) {
    auto kern = batched_rhs_kernel<NC, T, RPL, 4>;
    const size_t smem = n->ndet <= kMaxDetSmem ? (sizeof(float2) + sizeof(uint32_t)) * (size_t)n->ndet + 4 : 0;
    const int grid = resident_grid(ctx, kern, 4 * 32, (pc->nitems + 3) / 4, smem);
    const DetTables dt{n->det_off32.get(), n->wdf.get(), n->wsqrt.get(), n->ns_uniform, n->inv_ns};
    kern<<<grid, 4 * 32, smem, ctx->stream>>>(pc->item_pix.get(), pc->item_beg.get(), pc->item_len.get(), pc->nitems,
                                          pc->pitem.get(), p->perm.get(), p->cs_hi_s.get(),
                                          exact_lo ? p->cs_lo_s.get() : nullptr, dT, G, r0, R, dt, n->ndet, b,
                                          partial);
    BM_LAUNCH_CHECK();
}

// Group size of the batched RHS for a problem shape: for more than 32
// right-hand sides, groups of 32 (one a lane) and of 64 (two a lane) are
// both run once per shape (pixels, kept samples, R, components, TOD type)
// and timed, and the faster is kept for the process; both give the same
// bits (each right-hand side's sums run in the same order either way).
// Returns the group size; b holds the RHS on return.
template <class F>
int rhs_autotune(bm_context* ctx, bm_pointing* p, int R, bm_dtype dt, F&& run) {
    static std::mutex mu;
    static std::map<std::tuple<int64_t, int64_t, int, int, int>, int> cache;
    if (R <= 32) {
        run(R);
        return R;
    }
    const auto key = std::make_tuple(p->npix, p->nvalid, R, p->ncomp, (int)dt);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            run(it->second);
            return it->second;
        }
    }
    cudaEvent_t a, b;
    BM_CUDA(cudaEventCreate(&a));
    BM_CUDA(cudaEventCreate(&b));
    float best_ms = 1e30f;
    int best = 32;
    for (int G : {32, std::min(R, 64)}) {
        BM_CUDA(cudaEventRecord(a, ctx->stream));
        run(G);
        BM_CUDA(cudaEventRecord(b, ctx->stream));
        BM_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        BM_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best_ms) {
            best_ms = ms;
            best = G;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return best;
}



// The batched solver's device buffers, all RHS-interleaved [npix][NC][R].
struct BatchBufs {
    double *b, *x, *r, *e, *rcg, *z, *pv, *q, *partial, *part, *tolr, *sums;
    float* x32;
    RhsState* st;
    int* loop;
};

template <int NC>
Variant autotune(bm_context* ctx, bm_precond* pc, int R, const BatchBufs& bb) {
    // Variant of the batched matvec (right-hand sides per lane, warps per
    // block) timed once per problem shape (npix, samples, R, components) and
    // cached for the process.
    static std::mutex mu;
    static std::map<std::tuple<int64_t, int64_t, int, int>, Variant> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(pc->p->npix, pc->p->nvalid, R, NC);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const Variant cands[] = {{1, 4}, {1, 8}, {2, 4}, {2, 8}, {4, 4}, {4, 8}};
    Variant best = {2, 4};
    float best_ms = 1e30f;
    cudaEvent_t a, b;
    BM_CUDA(cudaEventCreate(&a));
    BM_CUDA(cudaEventCreate(&b));
    for (const Variant& v : cands) {
        const int per = 32 * v.rpl;
        if (per > 32 && R <= per / 2) continue;  // lanes would idle
        float tot = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            BM_CUDA(cudaEventRecord(a, ctx->stream));
            for (int r0 = 0; r0 < R; r0 += per)
                launch_matvec<NC>(ctx, pc, v, bb.x32, r0, std::min(per, R - r0), R, bb.q, bb.partial);
            BM_CUDA(cudaEventRecord(b, ctx->stream));
            BM_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            BM_CUDA(cudaEventElapsedTime(&ms, a, b));
            if (rep == 1) tot = ms;
        }
        if (tot < best_ms) { best_ms = tot; best = v; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cache[key] = best;
    return best;
}

template <int NC>
bm_status batched_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* const* rows, bm_dtype dt,
                        int R, double* const* maps, double tol, int32_t maxiter, bm_solve_info* info) {
    bm_context* ctx = p->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t npix = p->npix;
    const int RNC = R * NC;
    const int64_t nv = npix * RNC;
    const int threads = 256;
    const int vgrid = grid_for(ctx, (nv + threads - 1) / threads, 16);

    BatchBufs bb;
    bb.b = workspace_as<double>(ctx, "bt_b", nv);
    bb.x = workspace_as<double>(ctx, "bt_x", nv);
    bb.r = workspace_as<double>(ctx, "bt_r", nv);
    bb.e = workspace_as<double>(ctx, "bt_e", nv);
    bb.rcg = workspace_as<double>(ctx, "bt_rcg", nv);
    bb.z = workspace_as<double>(ctx, "bt_z", nv);
    bb.pv = workspace_as<double>(ctx, "bt_p", nv);
    bb.q = workspace_as<double>(ctx, "bt_q", nv);
    bb.partial = workspace_as<double>(ctx, "bt_partial", (size_t)std::max<int64_t>(pc->nitems, 1) * RNC);
    bb.part = workspace_as<double>(ctx, "bt_part", (size_t)2 * kRB * R);
    bb.tolr = workspace_as<double>(ctx, "bt_tol", R);
    bb.sums = workspace_as<double>(ctx, "bt_sums", 2 * (size_t)R);
    bb.x32 = workspace_as<float>(ctx, "bt_x32", nv);
    bb.st = reinterpret_cast<RhsState*>(workspace_as<char>(ctx, "bt_state", sizeof(RhsState) * R));
    bb.loop = workspace_as<int>(ctx, "bt_loop", 2);
    // the caller's TOD rows and map outputs, as device arrays of pointers
    char* ptrs = workspace_as<char>(ctx, "bt_ptrs", 2 * sizeof(void*) * (size_t)R);
    {
        std::vector<const void*> h(2 * (size_t)R);
        for (int r = 0; r < R; ++r) {
            h[r] = rows[r];
            h[R + r] = maps[r];
        }
        BM_CUDA(cudaMemcpyAsync(ptrs, h.data(), 2 * sizeof(void*) * (size_t)R, cudaMemcpyHostToDevice, s));
        BM_CUDA(cudaStreamSynchronize(s));
    }
    const void* const* d_rows = reinterpret_cast<const void* const*>(ptrs);
    bool rows_aligned = true;
    for (int r = 0; r < R; ++r) rows_aligned = rows_aligned && (reinterpret_cast<uintptr_t>(rows[r]) % 16 == 0);
    double* const* d_maps = reinterpret_cast<double* const*>(ptrs + sizeof(void*) * (size_t)R);

    // --- batched RHS, TOD transposed group by group (groups of G <= 64 rows)
    auto batched_rhs = [&](int G) {
        const size_t esz = dt == BM_F32 ? 4 : 8;
        void* dT = workspace(ctx, "bt_todT", (size_t)p->nsamples * G * esz);
        for (int r0 = 0; r0 < R; r0 += G) {
            const int g = std::min(G, R - r0);
            const dim3 tgrid((unsigned)std::min<int64_t>((p->nsamples + 31) / 32, (int64_t)ctx->num_sms * 16),
                             (unsigned)((g + 31) / 32));
            const dim3 tblk(32, 8);
            if (dt == BM_F32 && rows_aligned)
                transpose_f32x4_kernel<<<resident_grid(ctx, transpose_f32x4_kernel, 256, (p->nsamples + kTT - 1) / kTT),
                                         256, 0, s>>>(reinterpret_cast<const float* const*>(d_rows), p->nsamples, r0,
                                                      g, static_cast<float*>(dT));
            else if (dt == BM_F32)
                transpose_group_kernel<float><<<tgrid, tblk, 0, s>>>(reinterpret_cast<const float* const*>(d_rows),
                                                                     p->nsamples, r0, g, static_cast<float*>(dT));
            else
                transpose_group_kernel<double><<<tgrid, tblk, 0, s>>>(
                    reinterpret_cast<const double* const*>(d_rows), p->nsamples, r0, g, static_cast<double*>(dT));
            BM_LAUNCH_CHECK();
            const bool lo = p->cs_lo_s.get() != nullptr;
            if (dt == BM_F32)
                (g > 32 ? launch_rhs_v<NC, float, 2> : launch_rhs_v<NC, float, 1>)(
                    ctx, p, n, pc, static_cast<float*>(dT), g, r0, R, bb.b, bb.partial, lo);
            else
                (g > 32 ? launch_rhs_v<NC, double, 2> : launch_rhs_v<NC, double, 1>)(
                    ctx, p, n, pc, static_cast<double*>(dT), g, r0, R, bb.b, bb.partial, lo);
        }
        batched_finalize_kernel<<<vgrid, threads, 0, s>>>(pc->pitem.get(), bb.partial, npix, RNC, bb.b);
        BM_LAUNCH_CHECK();
    };
    {
        const int G = rhs_autotune(ctx, p, R, dt, batched_rhs);  // runs the RHS at least once
        ScopedTimer timer(ctx, "rhs_batched");
        if (ctx->timing) batched_rhs(G);  // (timed on its own when kernel timing is on)
    }

    // --- geometry of the per-pixel PCG kernels
    int Rp = 1;
    while (Rp < R) Rp <<= 1;
    BGeo geo{R, Rp, kRT / Rp, npix};
    // per-pixel PCG kernels: one wave of resident blocks (at most kRB)
    int per_sm = 64;
    for (const void* k : {reinterpret_cast<const void*>(b_residual_kernel<NC, false>),
                          reinterpret_cast<const void*>(b_init_kernel<NC>),
                          reinterpret_cast<const void*>(b_update_kernel<NC>),
                          reinterpret_cast<const void*>(b_dot_kernel),
                          reinterpret_cast<const void*>(b_pupdate_kernel)})
        per_sm = std::min(per_sm, blocks_per_sm(k, kRT, 0));
    const int rgrid = std::min(kRB, std::max(per_sm, 1) * ctx->num_sms);
    const int sgrid = (R + 127) / 128;

    // x = 0; r = b (masked), per-RHS ||b||
    BM_CUDA(cudaMemsetAsync(bb.x, 0, sizeof(double) * nv, s));
    b_residual_kernel<NC, true><<<rgrid, kRT, 0, s>>>(geo, pc->B.get(), pc->mask.get(), bb.b, bb.x, bb.r, bb.part);
    BM_LAUNCH_CHECK();
    b_sum2_kernel<<<sgrid, 128, 0, s>>>(bb.part, rgrid, R, bb.sums);
    BM_LAUNCH_CHECK();
    std::vector<double> hs(2 * R);
    BM_CUDA(cudaMemcpyAsync(hs.data(), bb.sums, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bnorm(R), rr(hs.begin(), hs.begin() + R);
    for (int r = 0; r < R; ++r) bnorm[r] = std::sqrt(hs[R + r]);

    const Variant var = (pc->nitems > 0) ? autotune<NC>(ctx, pc, R, bb) : Variant{2, 4};
    const int per = 32 * var.rpl;
    if (ctx->timing && pc->nitems > 0) {  // one batched matvec timed on its own (its roofline)
        ScopedTimer timer(ctx, "matvec_batched");
        for (int r0 = 0; r0 < R; r0 += per)
            launch_matvec<NC>(ctx, pc, var, bb.x32, r0, std::min(per, R - r0), R, bb.q, bb.partial);
    }

    auto inner_iteration = [&](cudaStream_t st) {
        batched_masked_f32_kernel<<<vgrid, threads, 0, st>>>(bb.pv, pc->mask.get(), npix, RNC, bb.x32);
        BM_LAUNCH_CHECK();
        cudaStream_t saved = ctx->stream;
        ctx->stream = st;
        for (int r0 = 0; r0 < R; r0 += per)
            launch_matvec<NC>(ctx, pc, var, bb.x32, r0, std::min(per, R - r0), R, bb.q, bb.partial);
        ctx->stream = saved;
        batched_finalize_kernel<<<vgrid, threads, 0, st>>>(pc->pitem.get(), bb.partial, npix, RNC, bb.q);
        BM_LAUNCH_CHECK();
        b_dot_kernel<<<rgrid, kRT, 0, st>>>(geo, NC, bb.pv, bb.q, bb.part);
        BM_LAUNCH_CHECK();
        b_alpha_kernel<<<sgrid, 128, 0, st>>>(bb.part, rgrid, R, bb.st);
        BM_LAUNCH_CHECK();
        b_update_kernel<NC><<<rgrid, kRT, 0, st>>>(geo, pc->Minv.get(), bb.e, bb.rcg, bb.z, bb.pv, bb.q, bb.st, bb.part);
        BM_LAUNCH_CHECK();
        b_beta_kernel<<<sgrid, 128, 0, st>>>(bb.part, rgrid, R, bb.st);
        BM_LAUNCH_CHECK();
        b_pupdate_kernel<<<rgrid, kRT, 0, st>>>(geo, NC, bb.pv, bb.z, bb.st);
        BM_LAUNCH_CHECK();
    };

    // The inner PCG loop as one graph, built on first use: b_loop_kernel
    // decides whether to enter, then a WHILE node runs one inner iteration
    // followed by b_loop_kernel again, for as long as any right-hand side is
    // active and fewer iterations than the limit in loop[1] have run.  The
    // limit bounds the loop whatever the states hold.  The host reads the
    // states once per outer iteration, not after every inner one.
    cudaGraphExec_t gexec = nullptr;
    int64_t body_kernels = 0;
    bool graph_ok = true;
    auto build_loop_graph = [&]() {
        cudaGraph_t graph = nullptr;
        BM_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(ctx->side, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            b_loop_kernel<<<1, 32, 0, ctx->side>>>(bb.st, R, bb.loop, 0, h);
            e = cudaGetLastError();
            const cudaError_t e2 = cudaStreamEndCapture(ctx->side, &graph);
            if (e == cudaSuccess) e = e2;
        }
        cudaGraphNode_t first = nullptr;
        size_t nn = 1;
        if (e == cudaSuccess) e = cudaGraphGetNodes(graph, &first, &nn);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, graph, &first, nullptr, 1, &cp);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(ctx->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const int64_t before = bm_kernel_launches();
                try {
                    inner_iteration(ctx->side);
                } catch (...) {
                    cudaStreamEndCapture(ctx->side, &body);
                    cudaGraphDestroy(graph);
                    throw;
                }
                body_kernels = bm_kernel_launches() - before + 1;  // + the loop kernel
                count_launches(-(body_kernels - 1));  // counted from the iterations that ran
                b_loop_kernel<<<1, 32, 0, ctx->side>>>(bb.st, R, bb.loop, 1, h);
                e = cudaGetLastError();
                const cudaError_t e2 = cudaStreamEndCapture(ctx->side, &body);
                if (e == cudaSuccess) e = e2;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        BM_CUDA(e);
    };

    std::vector<bm_solve_info> inf(R);
    std::vector<RhsState> hst(R);
    int inner_total = 0, outer = 0;
    const int max_outer = 30;
    std::vector<double> tolr(R);
    auto all_done = [&]() {
        for (int r = 0; r < R; ++r)
            if (bnorm[r] > 0 && std::sqrt(rr[r]) > tol * bnorm[r]) return false;
        return true;
    };
    while (!all_done() && inner_total < maxiter && outer < max_outer) {
        // inner tolerance per RHS (absolute, squared): max(1e-5, 0.5 tol ||b|| / ||r||) relative to ||r||
        for (int r = 0; r < R; ++r) {
            const double nr = std::sqrt(rr[r]);
            const double rel = (nr > 0) ? std::max(1e-5, std::min(0.5, 0.5 * tol * bnorm[r] / nr)) : 0.5;
            const double t = rel * nr;
            tolr[r] = (bnorm[r] > 0 && nr > tol * bnorm[r]) ? t * t : 1e300;  // converged RHS start done
        }
        BM_CUDA(cudaMemcpyAsync(bb.tolr, tolr.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
        b_init_kernel<NC><<<rgrid, kRT, 0, s>>>(geo, pc->Minv.get(), bb.r, bb.e, bb.rcg, bb.z, bb.pv, bb.part);
        BM_LAUNCH_CHECK();
        b_init_finalize<<<sgrid, 128, 0, s>>>(bb.part, rgrid, R, bb.tolr, bb.st);
        BM_LAUNCH_CHECK();
        const int hloop[2] = {0, maxiter - inner_total};  // >= 1 here
        BM_CUDA(cudaMemcpyAsync(bb.loop, hloop, sizeof(hloop), cudaMemcpyHostToDevice, s));
        int loop_out[2] = {0, 0};
        if (ctx->side != nullptr && ctx->graphs && gexec == nullptr && graph_ok) {
            try {
                build_loop_graph();
            } catch (const Error&) {  // no conditional graph here: the host-driven loop below
                graph_ok = false;
                gexec = nullptr;
                cudaGetLastError();
                clear_error();
            }
        }
        if (gexec != nullptr) {
            BM_CUDA(cudaEventRecord(ctx->side_ev, s));
            BM_CUDA(cudaStreamWaitEvent(ctx->side, ctx->side_ev, 0));
            BM_CUDA(cudaGraphLaunch(gexec, ctx->side));
            BM_CUDA(cudaEventRecord(ctx->side_ev, ctx->side));
            BM_CUDA(cudaStreamWaitEvent(s, ctx->side_ev, 0));
            BM_CUDA(cudaMemcpyAsync(loop_out, bb.loop, sizeof(loop_out), cudaMemcpyDeviceToHost, s));
        } else {  // no side stream or no conditional graph: the same loop driven from the host
            for (int it = 0; it < hloop[1]; ++it) {
                BM_CUDA(cudaMemcpyAsync(hst.data(), bb.st, sizeof(RhsState) * R, cudaMemcpyDeviceToHost, s));
                BM_CUDA(cudaStreamSynchronize(s));
                bool any = false;
                for (int r = 0; r < R; ++r) any = any || !hst[r].done;
                if (!any) break;
                inner_iteration(s);
            }
        }
        BM_CUDA(cudaMemcpyAsync(hst.data(), bb.st, sizeof(RhsState) * R, cudaMemcpyDeviceToHost, s));
        BM_CUDA(cudaStreamSynchronize(s));
        if (gexec != nullptr) count_launches(1 + (int64_t)loop_out[0] * body_kernels);
        int itmax = 0;
        for (int r = 0; r < R; ++r) {
            inf[r].iterations += hst[r].iters;
            itmax = std::max(itmax, hst[r].iters);
        }
        inner_total += std::max(itmax, 1);
        ++outer;
        b_axpy_kernel<<<vgrid, threads, 0, s>>>(bb.x, bb.e, nv);
        BM_LAUNCH_CHECK();
        b_residual_kernel<NC, false><<<rgrid, kRT, 0, s>>>(geo, pc->B.get(), pc->mask.get(), bb.b, bb.x, bb.r,
                                                          bb.part);
        BM_LAUNCH_CHECK();
        b_sum2_kernel<<<sgrid, 128, 0, s>>>(bb.part, rgrid, R, bb.sums);
        BM_LAUNCH_CHECK();
        BM_CUDA(cudaMemcpyAsync(hs.data(), bb.sums, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
        BM_CUDA(cudaStreamSynchronize(s));
        bool improved = false;
        for (int r = 0; r < R; ++r) {
            if (hs[r] < rr[r]) improved = true;
            rr[r] = hs[r];
        }
        if (!improved) break;  // stagnation
    }
    if (gexec) cudaGraphExecDestroy(gexec);

    {
        const int P = std::max(1, 4096 / RNC);  // pixels a tile: at most 32 KB of x staged
        const size_t smem = sizeof(double) * (size_t)P * RNC;
        const int64_t ntiles = (npix + P - 1) / P;
        b_write_map_kernel<<<resident_grid(ctx, b_write_map_kernel, threads, ntiles, smem), threads, smem, s>>>(
            bb.x, pc->mask.get(), npix, R, NC, P, d_maps);
        BM_LAUNCH_CHECK();
    }
    BM_CUDA(cudaStreamSynchronize(s));
    bm_status first = BM_OK;
    for (int r = 0; r < R; ++r) {
        inf[r].outer_iterations = outer;
        inf[r].rel_residual = bnorm[r] > 0 ? std::sqrt(rr[r]) / bnorm[r] : 0.0;
        inf[r].status = (inf[r].rel_residual <= tol) ? BM_OK : BM_ERR_NOT_CONVERGED;
        if (hst[r].done == 2 && inf[r].status != BM_OK) inf[r].status = BM_ERR_BREAKDOWN;
        if (first == BM_OK && inf[r].status != BM_OK) first = (bm_status)inf[r].status;
        if (info) info[r] = inf[r];
    }
    return first;
}

}  // namespace

bm_status batched_white_solve_rows(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* const* rows,
                                   bm_dtype dt, int32_t nrhs, double* const* maps, double tol, int32_t maxiter,
                                   bm_solve_info* info) {
    const int nc = p->ncomp;
    bm_status first = BM_OK;
    // Groups of at most kBatchMax right-hand sides per batched solve.
    for (int32_t r0 = 0; r0 < nrhs; r0 += kBatchMax) {
        const int R = std::min<int32_t>(kBatchMax, nrhs - r0);
        bm_solve_info* ir = info ? info + r0 : nullptr;
        bm_status st;
        if (nc == 3) st = batched_solve<3>(p, n, pc, rows + r0, dt, R, maps + r0, tol, maxiter, ir);
        else if (nc == 2) st = batched_solve<2>(p, n, pc, rows + r0, dt, R, maps + r0, tol, maxiter, ir);
        else st = batched_solve<1>(p, n, pc, rows + r0, dt, R, maps + r0, tol, maxiter, ir);
        if (first == BM_OK && st != BM_OK) first = st;
    }
    return first;
}

bm_status batched_white_solve(bm_pointing* p, bm_inv_noise* n, bm_precond* pc, const void* tod, bm_dtype dt,
                              int32_t nrhs, double* map_out, double tol, int32_t maxiter, bm_solve_info* info) {
    const int64_t nvec = p->npix * p->ncomp;
    const size_t row_bytes = (size_t)p->nsamples * (dt == BM_F32 ? 4 : 8);
    std::vector<const void*> rows(nrhs);
    std::vector<double*> maps(nrhs);
    for (int32_t r = 0; r < nrhs; ++r) {
        rows[r] = static_cast<const char*>(tod) + (size_t)r * row_bytes;
        maps[r] = map_out + (int64_t)r * nvec;
    }
    return batched_white_solve_rows(p, n, pc, rows.data(), dt, nrhs, maps.data(), tol, maxiter, info);
}

}  // namespace bm
