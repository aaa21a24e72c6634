// Block-diagonal preconditioner (paper Eq. 7) and the pixel mask.
//
// B_p = sum_{t in p} w_d(t) v_t v_t^T is accumulated in FP64 over each pixel's
// pixel-sorted segment (one warp per work item of <= kItemMax samples, item
// partials summed in item order, so the result is deterministic).  Per pixel:
// eigenvalue extremes of the symmetric block, condition number, mask, and the
// FP64 inverse M_p = B_p^-1.  The same pass plans the work items over kept
// pixels used by every sorted-order kernel, and, for white noise, writes the
// weighted FP32 stream sqrt(w) (cos 2psi, sin 2psi) that the FP32 matvec reads.
#include "bm_internal.cuh"

namespace bm {

// ------------------------------------------------------------ item planning
namespace {

__global__ void item_count_kernel(const int64_t* __restrict__ off, const uint8_t* __restrict__ mask,
                                  int64_t npix, int64_t* __restrict__ cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = off[p + 1] - off[p];
        const bool keep = h > 0 && (mask == nullptr || mask[p] == 0);
        cnt[p] = keep ? (h + kItemMax - 1) / kItemMax : 0;
    }
}

__global__ void item_fill_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ pitem,
                                 int64_t npix, int32_t* __restrict__ item_pix,
                                 int64_t* __restrict__ item_beg, int32_t* __restrict__ item_len) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = pitem[p], k1 = pitem[p + 1];
        const int64_t a = off[p], e = off[p + 1];
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t b = a + (k - k0) * kItemMax;
            item_pix[k] = (int32_t)p;
            item_beg[k] = b;
            item_len[k] = (int32_t)((e - b) < kItemMax ? (e - b) : kItemMax);
        }
    }
}

}  // namespace

void plan_items(bm_context* ctx, const int64_t* off, const uint8_t* mask, int64_t npix, Items& it) {
    cudaStream_t s = ctx->stream;
    const int threads = 256;
    const int grid = grid_for(ctx, (npix + threads - 1) / threads, 16);
    DevBuf<int64_t> cnt(npix + 1);
    it.pitem.alloc(npix + 1);
    BM_CUDA(cudaMemsetAsync(cnt.get() + npix, 0, sizeof(int64_t), s));
    item_count_kernel<<<grid, threads, 0, s>>>(off, mask, npix, cnt.get());
    BM_LAUNCH_CHECK();
    exclusive_scan_i64(cnt.get(), it.pitem.get(), npix + 1, s);
    BM_CUDA(cudaMemcpyAsync(&it.n, it.pitem.get() + npix, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    const size_t m = it.n > 0 ? (size_t)it.n : 1;
    it.pix.alloc(m);
    it.beg.alloc(m);
    it.len.alloc(m);
    if (it.n > 0) {
        item_fill_kernel<<<grid, threads, 0, s>>>(off, it.pitem.get(), npix, it.pix.get(), it.beg.get(),
                                                  it.len.get());
        BM_LAUNCH_CHECK();
    }
}

// ------------------------------------------------------------------ blocks
namespace {

constexpr int kBlkWarps = 8;

// B_p partials per work item.  Unique entries of the symmetric block,
// row-major upper triangle: IQU (II, IQ, IU, QQ, QU, UU); QU (QQ, QU, UU); I (II).
// Every product and sum is double-float (w and the trig pair carry ~48 bits),
// so the block keeps FP64-level accuracy without FP64 instructions per sample;
// the warp total is converted to FP64 once per item (EXACT: the lazily
// renormalised sums of prod_u / acc_add).  For white noise the
// same pass writes the weighted FP32 stream sqrt(w) (cos, sin) (w for I-only)
// that the FP32 matvec reads.  With RHS (white noise and a TOD sorted along
// with the pointing) it also sums b = P^T N^-1 d per item into rpartial, with
// the double-float steps of the pixel-sorted gather-reduce of the RHS (the
// same operations in the same order, so the same bits).  EXACT: the trig
// pairs are exact FP32 values (no lo part), so the block products multiply
// by a float instead of a double-float.
template <int NC, bool WCS, bool RHS, bool EXACT>
__global__ void __launch_bounds__(kBlkWarps * 32)
blocks_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
              const int32_t* __restrict__ item_len, int64_t nitems, const uint32_t* __restrict__ perm,
              const float2* __restrict__ hi, const float2* __restrict__ lo, DetTables g, int ndet,
              double* __restrict__ partial, float2* __restrict__ wcs, float* __restrict__ w1,
              const float* __restrict__ tod_s, double* __restrict__ rpartial) {
    constexpr int NS = NC * (NC + 1) / 2;
    __shared__ uint32_t s_off[kMaxDetSmem + 1];
    __shared__ float2 s_w[kMaxDetSmem];
    __shared__ float s_sw[kMaxDetSmem];
    const bool in_smem = ndet <= kMaxDetSmem;
    if (in_smem) {
        for (int d = threadIdx.x; d <= ndet; d += blockDim.x) s_off[d] = g.off[d];
        for (int d = threadIdx.x; d < ndet; d += blockDim.x) { s_w[d] = g.wdf[d]; s_sw[d] = g.wsqrt[d]; }
    }
    __syncthreads();
    const uint32_t* offp = in_smem ? s_off : g.off;
    const float2* wp = in_smem ? s_w : g.wdf;
    const float* swp = in_smem ? s_sw : g.wsqrt;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kBlkWarps;
    for (int64_t k = (int64_t)blockIdx.x * kBlkWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t b = item_beg[k];
        const int len = item_len[k];
        df32 acc[NS], racc[NC];
#pragma unroll
        for (int j = 0; j < NS; ++j) acc[j] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < NC; ++j) racc[j] = {0.f, 0.f};
        // A lane's samples of one item are in increasing time order (the sort
        // is stable), so its detector changes only when t passes the current
        // detector's end: look the detector up only then.
        uint32_t dend = 0;
        float2 wv = make_float2(0.f, 0.f);
        float swv = 0.f;
        auto add = [&](int64_t si, uint32_t t, float2 h, float2 l, float dv) {
            if (g.wsort) {  // a weight per sample
                wv = g.wsort[si];
                if (WCS && NC > 1) swv = g.ssort[si];
            } else if (t >= dend) {
                const int d = det_of(offp, ndet, g.ns, g.inv_ns, t);
                dend = g.ns ? (uint32_t)(d + 1) * g.ns : offp[d + 1];
                wv = wp[d];
                if (WCS && NC > 1) swv = swp[d];
            }
            const df32 w = {wv.x, wv.y};
            const df32 c = {h.x, l.x}, s = {h.y, l.y};
            if (RHS) rhs_term_lazy<NC>(racc, dv, 0.f, true, wv, h, l);
            if (EXACT) {
                if (NC == 1) {
                    acc_add(acc[0], w.hi, w.lo);
                } else {
                    float wcp, wce, wsp, wse, p, e;
                    prod_u(w.hi, w.lo, h.x, wcp, wce);
                    prod_u(w.hi, w.lo, h.y, wsp, wse);
                    if (NC == 3) {
                        acc_add(acc[0], w.hi, w.lo);
                        acc_add(acc[1], wcp, wce);
                        acc_add(acc[2], wsp, wse);
                    }
                    prod_u(wcp, wce, h.x, p, e);
                    acc_add(acc[NS - 3], p, e);
                    prod_u(wcp, wce, h.y, p, e);
                    acc_add(acc[NS - 2], p, e);
                    prod_u(wsp, wse, h.y, p, e);
                    acc_add(acc[NS - 1], p, e);
                }
            } else if (NC == 3) {
                const df32 wc = df_mul(w, c), ws = df_mul(w, s);
                acc[0] = df_add(acc[0], w);
                acc[1] = df_add(acc[1], wc);
                acc[2] = df_add(acc[2], ws);
                acc[3] = df_add(acc[3], df_mul(wc, c));
                acc[4] = df_add(acc[4], df_mul(wc, s));
                acc[5] = df_add(acc[5], df_mul(ws, s));
            } else if (NC == 2) {
                const df32 wc = df_mul(w, c), ws = df_mul(w, s);
                acc[0] = df_add(acc[0], df_mul(wc, c));
                acc[1] = df_add(acc[1], df_mul(wc, s));
                acc[2] = df_add(acc[2], df_mul(ws, s));
            } else {
                acc[0] = df_add(acc[0], w);
            }
            if (WCS) {
                if (NC == 1) {
                    w1[si] = wv.x;
                } else {
                    wcs[si] = make_float2(swv * h.x, swv * h.y);
                }
            }
        };
        // kUnroll samples per lane in flight (their loads issued together);
        // the lane's samples are still added in order
        constexpr int kUnroll = 4;
        // the lazy sums are renormalised after every kLazyNorm samples of the
        // lane (at the end of every kLazyNorm / kUnroll groups) and at the end
        auto norm = [&]() {
            if (EXACT) {
#pragma unroll
                for (int j = 0; j < NS; ++j) acc_norm(acc[j]);
            }
            if (RHS) {
#pragma unroll
                for (int j = 0; j < NC; ++j) acc_norm(racc[j]);
            }
        };
        static_assert(kLazyNorm % kUnroll == 0, "renormalisation points fall at group ends");
        int nadd = 0;
        int i = lane;
        for (; i + 32 * (kUnroll - 1) < len; i += 32 * kUnroll) {
            uint32_t t[kUnroll];
            float2 h[kUnroll], l[kUnroll];
            float dv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t si = b + i + 32 * u;
                t[u] = perm[si];
                h[u] = hi[si];
                l[u] = (!EXACT && lo) ? lo[si] : make_float2(0.f, 0.f);
                dv[u] = RHS ? tod_s[si] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) add(b + i + 32 * u, t[u], h[u], l[u], dv[u]);
            nadd += kUnroll;
            if (nadd == kLazyNorm) {
                nadd = 0;
                norm();
            }
        }
        for (; i < len; i += 32) {
            const int64_t si = b + i;
            add(si, perm[si], hi[si], (!EXACT && lo) ? lo[si] : make_float2(0.f, 0.f), RHS ? tod_s[si] : 0.f);
            if (++nadd == kLazyNorm) {
                nadd = 0;
                norm();
            }
        }
        norm();
#pragma unroll
        for (int j = 0; j < NS; ++j) acc[j] = df_warp_sum(acc[j]);
        if (RHS) {
#pragma unroll
            for (int j = 0; j < NC; ++j) racc[j] = df_warp_sum(racc[j]);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < NS; ++j) partial[k * NS + j] = df_to_double(acc[j]);
            if (RHS) {
#pragma unroll
                for (int j = 0; j < NC; ++j) rpartial[NC * k + j] = df_to_double(racc[j]);
            }
        }
    }
}

// b_p = sum of the pixel's item partials in item order, 0 on masked pixels.
__global__ void finalize_rhs_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ rpartial,
                                    const uint8_t* __restrict__ mask, int64_t npix, int nc, double* __restrict__ b) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = mask[p] ? 0 : pitem[p], k1 = mask[p] ? 0 : pitem[p + 1];
        for (int c = 0; c < nc; ++c) {
            double s = 0.0;
            for (int64_t k = k0; k < k1; ++k) s += rpartial[k * nc + c];
            b[p * nc + c] = s;
        }
    }
}

// The weights of a noise model with a weight per sample, in pixel-sorted
// order: as a double-float pair, its square root in FP32, and in FP64.
__global__ void sort_weights_kernel(const uint32_t* __restrict__ perm, int64_t nvalid, const double* __restrict__ w,
                                    float2* __restrict__ wdf, float* __restrict__ wsq, double* __restrict__ w64) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvalid; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[perm[i]];
        const float hi = (float)x;
        wdf[i] = make_float2(hi, (float)(x - (double)hi));
        wsq[i] = sqrtf((float)x);
        w64[i] = x;
    }
}

// One Jacobi rotation in the (i, j) plane of the symmetric matrix m
// (row-major 3x3) that annihilates m[i][j]: with theta = (m_jj - m_ii) /
// (2 m_ij), t = tan of the rotation angle = sign(theta) / (|theta| +
// sqrt(theta^2 + 1)) (the smaller root), c = 1/sqrt(1 + t^2), s = t c.
__device__ __forceinline__ void jacobi_rotate(double m[3][3], int i, int j) {
    const double mij = m[i][j];
    if (mij == 0.0) return;
    const double theta = (m[j][j] - m[i][i]) / (2.0 * mij);
    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
    const int k = 3 - i - j;
    const double mik = m[i][k], mjk = m[j][k];
    m[i][i] -= t * mij;
    m[j][j] += t * mij;
    m[i][j] = m[j][i] = 0.0;
    m[i][k] = m[k][i] = c * mik - s * mjk;
    m[j][k] = m[k][j] = s * mik + c * mjk;
}

// Eigenvalue extremes of a symmetric 3x3 matrix a = (a00, a01, a02, a11,
// a12, a22) by cyclic Jacobi rotations (absolute error ~ eps ||a||, so the
// smallest eigenvalue keeps relative accuracy ~ eps * cond even when the
// two largest eigenvalues nearly coincide).
__device__ __forceinline__ void eig_sym3(const double a[6], double& lmin, double& lmax) {
    double m[3][3] = {{a[0], a[1], a[2]}, {a[1], a[3], a[4]}, {a[2], a[4], a[5]}};
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = m[0][1] * m[0][1] + m[0][2] * m[0][2] + m[1][2] * m[1][2];
        const double diag = m[0][0] * m[0][0] + m[1][1] * m[1][1] + m[2][2] * m[2][2];
        if (off <= 1e-36 * diag || off == 0.0) break;
        jacobi_rotate(m, 0, 1);
        jacobi_rotate(m, 0, 2);
        jacobi_rotate(m, 1, 2);
    }
    lmin = fmin(m[0][0], fmin(m[1][1], m[2][2]));
    lmax = fmax(m[0][0], fmax(m[1][1], m[2][2]));
}

// Eigenvalue extremes, condition number, mask, the block and its inverse of
// pixel p from its block sums a (the NS upper-triangle entries) and its hit
// count: Eq. 7 with the mask rule of the build's reading (hits < min_hits,
// or, for QU and IQU, lambda_min <= 0 or cond > max_cond).
template <int NC>
__device__ __forceinline__ void decide_block(int64_t p, const double* a, int32_t hits, int32_t min_hits,
                                             double max_cond, double* __restrict__ B, double* __restrict__ Minv,
                                             double* __restrict__ cond, uint8_t* __restrict__ mask) {
    double lmin, lmax;
    if (NC == 3) {
        eig_sym3(a, lmin, lmax);
    } else if (NC == 2) {
        const double m = 0.5 * (a[0] + a[2]);
        const double h = 0.5 * (a[0] - a[2]);
        const double rad = sqrt(h * h + a[1] * a[1]);
        lmax = m + rad;
        lmin = m - rad;
    } else {
        lmin = lmax = a[0];
    }
    const double c = lmin > 0.0 ? lmax / lmin : INFINITY;
    bool bad = hits < min_hits;
    if (NC > 1) bad = bad || !(lmin > 0.0) || c > max_cond;
    else bad = bad || !(a[0] > 0.0);
    cond[p] = c;
    mask[p] = bad ? 1 : 0;
    double* Bp = B + p * NC * NC;
    double* Mp = Minv + p * NC * NC;
    if (NC == 3) {
        const double b[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
#pragma unroll
        for (int j = 0; j < 9; ++j) Bp[j] = b[j];
        if (bad) {
#pragma unroll
            for (int j = 0; j < 9; ++j) Mp[j] = 0.0;
        } else {
            const double c00 = a[3] * a[5] - a[4] * a[4];
            const double c01 = a[2] * a[4] - a[1] * a[5];
            const double c02 = a[1] * a[4] - a[2] * a[3];
            const double c11 = a[0] * a[5] - a[2] * a[2];
            const double c12 = a[1] * a[2] - a[0] * a[4];
            const double c22 = a[0] * a[3] - a[1] * a[1];
            const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
            const double id = 1.0 / det;
            const double m[9] = {c00 * id, c01 * id, c02 * id, c01 * id, c11 * id,
                                 c12 * id, c02 * id, c12 * id, c22 * id};
#pragma unroll
            for (int j = 0; j < 9; ++j) Mp[j] = m[j];
        }
    } else if (NC == 2) {
        Bp[0] = a[0]; Bp[1] = a[1]; Bp[2] = a[1]; Bp[3] = a[2];
        if (bad) {
            Mp[0] = Mp[1] = Mp[2] = Mp[3] = 0.0;
        } else {
            const double id = 1.0 / (a[0] * a[2] - a[1] * a[1]);
            Mp[0] = a[2] * id; Mp[1] = -a[1] * id; Mp[2] = -a[1] * id; Mp[3] = a[0] * id;
        }
    } else {
        Bp[0] = a[0];
        Mp[0] = bad ? 0.0 : 1.0 / a[0];
    }
}

template <int NC>
__global__ void finalize_blocks_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ partial,
                                       const int32_t* __restrict__ hits, int64_t npix, int32_t min_hits,
                                       double max_cond, double* __restrict__ B, double* __restrict__ Minv,
                                       double* __restrict__ cond, uint8_t* __restrict__ mask) {
    constexpr int NS = NC * (NC + 1) / 2;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) a[j] = 0.0;
        for (int64_t k = pitem[p]; k < pitem[p + 1]; ++k)
#pragma unroll
            for (int j = 0; j < NS; ++j) a[j] += partial[k * NS + j];
        decide_block<NC>(p, a, hits[p], min_hits, max_cond, B, Minv, cond, mask);
    }
}

// Sharded build, first half: this rank's block sums of every pixel and its
// hit count, S[p] = (a_0 .. a_{NS-1}, hits), summed over the item partials in
// the same order as finalize_blocks_kernel.
template <int NC>
__global__ void block_sums_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ partial,
                                  const int32_t* __restrict__ hits, int64_t npix, double* __restrict__ S) {
    constexpr int NS = NC * (NC + 1) / 2;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) a[j] = 0.0;
        for (int64_t k = pitem[p]; k < pitem[p + 1]; ++k)
#pragma unroll
            for (int j = 0; j < NS; ++j) a[j] += partial[k * NS + j];
#pragma unroll
        for (int j = 0; j < NS; ++j) S[p * (NS + 1) + j] = a[j];
        S[p * (NS + 1) + NS] = (double)hits[p];
    }
}

// Sharded build, second half: the decision of every pixel from the block
// sums and hit counts summed over the ranks; the global hit counts are kept.
template <int NC>
__global__ void finalize_block_sums_kernel(const double* __restrict__ S, int64_t npix, int32_t min_hits,
                                           double max_cond, double* __restrict__ B, double* __restrict__ Minv,
                                           double* __restrict__ cond, uint8_t* __restrict__ mask,
                                           int32_t* __restrict__ hits_out) {
    constexpr int NS = NC * (NC + 1) / 2;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) a[j] = S[p * (NS + 1) + j];
        const int32_t h = (int32_t)S[p * (NS + 1) + NS];
        hits_out[p] = h;
        decide_block<NC>(p, a, h, min_hits, max_cond, B, Minv, cond, mask);
    }
}

}  // namespace

void build_precond(bm_precond* pc) {
    bm_context* ctx = pc->ctx;
    cudaStream_t s = ctx->stream;
    bm_pointing* p = pc->p;
    bm_inv_noise* n = pc->n;
    const int64_t npix = p->npix;
    const int nc = pc->ncomp;
    const int ns = pc->nsym;
    const int threads = 256;

    pc->B.alloc(npix * nc * nc);
    pc->Minv.alloc(npix * nc * nc);
    pc->cond.alloc(npix);
    pc->mask.alloc(npix);

    // Blocks over every non-empty pixel.
    {
        ScopedTimer timer(ctx, "blocks");
        Items all;
        plan_items(ctx, p->off.get(), nullptr, npix, all);
        DevBuf<double> partial((all.n > 0 ? all.n : 1) * ns);
        // the weighted sorted stream: white noise, and the offset template's
        // mixed operator (its white part)
        // (not for a half-wave-plate pointing with per-detector white noise
        // in QU or IQU: its FP32 matvec rebuilds the angle from the model)
        const bool white = (diagonal_noise(n) || n->kind == 3) && p->nvalid > 0 &&
                           !(p->hwp && n->kind == 0 && nc > 1);
        if (n->kind == 2 && p->nvalid > 0) {  // a weight per sample: gathered once into sorted order
            pc->ws_df.alloc(p->nvalid);
            pc->ws_sqrt.alloc(p->nvalid);
            pc->ws64.alloc(p->nvalid);
            sort_weights_kernel<<<grid_for(ctx, (p->nvalid + threads - 1) / threads, 16), threads, 0, s>>>(
                p->perm.get(), p->nvalid, n->wsamp.get(), pc->ws_df.get(), pc->ws_sqrt.get(), pc->ws64.get());
            BM_LAUNCH_CHECK();
        }
        if (white) {
            if (nc == 1) pc->w1.alloc(p->nvalid);
            else pc->wcs.alloc(p->nvalid);
        }
        // b = P^T N^-1 d of a TOD the pointing carries, in the same pass
        const bool with_rhs = white && diagonal_noise(n) && p->tod_s.get() != nullptr;
        DevBuf<double> rpartial;
        if (with_rhs) {
            rpartial.alloc((all.n > 0 ? all.n : 1) * nc);
            pc->b_tod.alloc(npix * nc);
        } else {
            pc->b_tod.release();
        }
        if (all.n > 0) {
            const int64_t wunits = (all.n + kBlkWarps - 1) / kBlkWarps;
            const DetTables g = det_tables(n, pc);
#define BM_BLOCKS3(NC, W, R, E)                                                                              \
    blocks_kernel<NC, W, R, E><<<resident_grid(ctx, blocks_kernel<NC, W, R, E>, kBlkWarps * 32, wunits), kBlkWarps * 32, 0, s>>>( \
        all.pix.get(), all.beg.get(), all.len.get(), all.n, p->perm.get(), p->cs_hi_s.get(), p->cs_lo_s.get(), g,     \
        n->ndet, partial.get(), pc->wcs.get(), pc->w1.get(), p->tod_s.get(), rpartial.get())
#define BM_BLOCKS(NC, W, R)                  \
    do {                                     \
        if (exact) BM_BLOCKS3(NC, W, R, true); \
        else BM_BLOCKS3(NC, W, R, false);    \
    } while (0)
            const bool exact = p->cs_lo_s.get() == nullptr;  // FP32 trig given: exact float multiplies
            if (with_rhs) {
                if (nc == 3) BM_BLOCKS(3, true, true); else if (nc == 2) BM_BLOCKS(2, true, true); else BM_BLOCKS(1, true, true);
            } else if (white) {
                if (nc == 3) BM_BLOCKS(3, true, false); else if (nc == 2) BM_BLOCKS(2, true, false); else BM_BLOCKS(1, true, false);
            } else {
                if (nc == 3) BM_BLOCKS(3, false, false); else if (nc == 2) BM_BLOCKS(2, false, false); else BM_BLOCKS(1, false, false);
            }
#undef BM_BLOCKS3
#undef BM_BLOCKS
            BM_LAUNCH_CHECK();
        }
        const int pgrid = grid_for(ctx, (npix + threads - 1) / threads, 16);
        if (!ctx->allreduce) {
#define BM_FIN(NC)                                                                                       \
    finalize_blocks_kernel<NC><<<pgrid, threads, 0, s>>>(all.pitem.get(), partial.get(), p->hits.get(),  \
                                                         npix, pc->min_hits, pc->max_cond, pc->B.get(), \
                                                         pc->Minv.get(), pc->cond.get(), pc->mask.get())
            if (nc == 3) BM_FIN(3);
            else if (nc == 2) BM_FIN(2);
            else BM_FIN(1);
#undef BM_FIN
            BM_LAUNCH_CHECK();
            pc->hits_global.release();
        } else {
            // a shard: this rank's block sums and hit counts, summed over
            // the ranks, then the decisions (the same on every rank)
            DevBuf<double> S(npix * (ns + 1));
            pc->hits_global.alloc(npix);
#define BM_SUMS(NC)                                                                                                   \
    block_sums_kernel<NC><<<pgrid, threads, 0, s>>>(all.pitem.get(), partial.get(), p->hits.get(), npix, S.get())
            if (nc == 3) BM_SUMS(3);
            else if (nc == 2) BM_SUMS(2);
            else BM_SUMS(1);
#undef BM_SUMS
            BM_LAUNCH_CHECK();
            shard_reduce(ctx, S.get(), npix * (ns + 1));
#define BM_FINS(NC)                                                                                                \
    finalize_block_sums_kernel<NC><<<pgrid, threads, 0, s>>>(S.get(), npix, pc->min_hits, pc->max_cond,             \
                                                             pc->B.get(), pc->Minv.get(), pc->cond.get(),         \
                                                             pc->mask.get(), pc->hits_global.get())
            if (nc == 3) BM_FINS(3);
            else if (nc == 2) BM_FINS(2);
            else BM_FINS(1);
#undef BM_FINS
            BM_LAUNCH_CHECK();
        }
        if (with_rhs) {
            finalize_rhs_kernel<<<pgrid, threads, 0, s>>>(all.pitem.get(), rpartial.get(), pc->mask.get(), npix, nc,
                                                          pc->b_tod.get());
            BM_LAUNCH_CHECK();
            shard_reduce(ctx, pc->b_tod.get(), npix * nc);
        }
        BM_CUDA(cudaStreamSynchronize(s));
    }

    // Work items over kept pixels.
    Items kept;
    plan_items(ctx, p->off.get(), pc->mask.get(), npix, kept);
    pc->nitems = kept.n;
    pc->item_pix = std::move(kept.pix);
    pc->item_beg = std::move(kept.beg);
    pc->item_len = std::move(kept.len);
    pc->pitem = std::move(kept.pitem);
    if (n->kind == 3) build_offset_counts(pc);

    BM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bm
