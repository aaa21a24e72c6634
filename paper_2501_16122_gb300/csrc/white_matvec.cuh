// The white-noise matvec with FP32 per-sample products (paper Eq. 6 with a
// diagonal N^-1, the operator of the mixed path's inner solve) and the
// per-pixel sum of its work-item partials.  Kept in a header so that every
// entry point that applies this operator compiles the same arithmetic and
// gives the same bits.
//
// The map x is read at the item's pixel and rounded to FP32 in registers:
// XT = float (a masked FP32 copy of x) or XT = double (x itself).  Work items
// exist only for kept pixels, so both read the same FP32 values.
#pragma once

#include "bm_internal.cuh"

namespace bm {

namespace {

constexpr int kWhiteWarps = 8;  // warps per block of white_matvec_f32_kernel

// ------------------------------------------------------- white, FP32 form
// One work item per warp.  Loads are 16 bytes per lane (two samples of the
// (u_c, u_s) stream, four of the I-only weight stream) after a scalar head
// that aligns the item start; each lane sums a group of samples in FP32 and
// folds the group into a compensated (double-float) accumulator, the warp
// combines the accumulators in double-float, and lane 0 writes the FP64 item
// partial.  sqrt(w) = |u| is formed as |u|^2 * rsqrt(|u|^2); the same value
// multiplies x_I and the I output, so the operator stays symmetric.
template <int NC, typename XT>
__global__ void __launch_bounds__(kWhiteWarps * 32)
white_matvec_f32_kernel(const int32_t* __restrict__ item_pix, const int64_t* __restrict__ item_beg,
                        const int32_t* __restrict__ item_len, int64_t nitems,
                        const float2* __restrict__ wcs, const float* __restrict__ w1,
                        const XT* __restrict__ x, double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWhiteWarps;
    for (int64_t k = (int64_t)blockIdx.x * kWhiteWarps + (threadIdx.x >> 5); k < nitems; k += nwarps) {
        const int64_t p = item_pix[k];
        int64_t b = item_beg[k];
        int len = item_len[k];
        if (NC == 1) {
            const float xi = (float)x[p];
            df32 A = {0.f, 0.f};
            const int head = (int)((4 - (b & 3)) & 3) < len ? (int)((4 - (b & 3)) & 3) : len;
            if (lane < head) A = df_add(A, __ldg(w1 + b + lane));
            b += head;
            len -= head;
            const float4* src4 = reinterpret_cast<const float4*>(w1 + b);
            const int nq = len >> 2;
            int j = lane;
            for (; j + 32 < nq; j += 64) {
                const float4 a = __ldg(src4 + j), c = __ldg(src4 + j + 32);
                A = df_add(A, ((a.x + a.y) + (a.z + a.w)) + ((c.x + c.y) + (c.z + c.w)));
            }
            for (; j < nq; j += 32) {
                const float4 a = __ldg(src4 + j);
                A = df_add(A, (a.x + a.y) + (a.z + a.w));
            }
            const int rem = len & 3;
            if (lane < rem) A = df_add(A, __ldg(w1 + b + 4 * nq + lane));
            A = df_warp_sum(A);
            if (lane == 0) partial[k] = df_to_double(A) * (double)xi;
        } else {
            float xI = 0.f, xQ, xU;
            if (NC == 3) { xI = (float)x[3 * p]; xQ = (float)x[3 * p + 1]; xU = (float)x[3 * p + 2]; }
            else { xQ = (float)x[2 * p]; xU = (float)x[2 * p + 1]; }
            float aI = 0.f, aQ = 0.f, aU = 0.f;  // FP32 group sums
            df32 AI = {0.f, 0.f}, AQ = {0.f, 0.f}, AU = {0.f, 0.f};
            auto step = [&](float2 u) {
                float r = 0.f;
                if (NC == 3) {
                    const float u2 = fmaf(u.x, u.x, u.y * u.y);
                    r = u2 > 0.f ? u2 * rsqrtf(u2) : 0.f;  // sqrt(w); a zero weight gives 0
                }
                const float y = fmaf(u.x, xQ, fmaf(u.y, xU, r * xI));
                if (NC == 3) aI = fmaf(y, r, aI);
                aQ = fmaf(y, u.x, aQ);
                aU = fmaf(y, u.y, aU);
            };
            auto fold = [&]() {
                if (NC == 3) AI = df_add(AI, aI);
                AQ = df_add(AQ, aQ);
                AU = df_add(AU, aU);
                aI = aQ = aU = 0.f;
            };
            if (b & 1) {  // align the stream to 16 bytes
                if (lane == 0) step(__ldg(wcs + b));
                ++b;
                --len;
            }
            const float4* src4 = reinterpret_cast<const float4*>(wcs + b);
            const int np = len >> 1;  // sample pairs
            int j = lane;
            for (; j + 96 < np; j += 128) {
                const float4 u0 = __ldg(src4 + j), u1 = __ldg(src4 + j + 32);
                const float4 u2 = __ldg(src4 + j + 64), u3 = __ldg(src4 + j + 96);
                step(make_float2(u0.x, u0.y)); step(make_float2(u0.z, u0.w));
                step(make_float2(u1.x, u1.y)); step(make_float2(u1.z, u1.w));
                step(make_float2(u2.x, u2.y)); step(make_float2(u2.z, u2.w));
                step(make_float2(u3.x, u3.y)); step(make_float2(u3.z, u3.w));
                fold();
            }
            for (; j < np; j += 32) {
                const float4 u0 = __ldg(src4 + j);
                step(make_float2(u0.x, u0.y)); step(make_float2(u0.z, u0.w));
            }
            if ((len & 1) && lane == 0) step(__ldg(wcs + b + len - 1));
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
}

// q_p = sum of the partials of pixel p's items (item order); 0 for pixels without items.
__global__ void finalize_pixels_kernel(const int64_t* __restrict__ pitem, const double* __restrict__ partial,
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

}  // namespace

}  // namespace bm
