// HEALPix RING ang2pix on the device (Gorski et al. 2005, ApJ 622:759, Sec. 4):
// the "sky pixel" of a direction in the paper's pointing matrix (Eq. 8).
//
// Every floating-point step is an explicit correctly rounded FP64 intrinsic
// (__dmul_rn, __dadd_rn, __dsub_rn, __dsqrt_rn), so the compiler cannot fuse
// a multiply into an add; the integer result is therefore a function of the
// IEEE inputs alone and matches any implementation that follows the same
// steps:
//   tt = phi * (2/pi) wrapped into [0, 4)
//   belt (|z| <= 2/3): jp = floor(n (0.5 + tt) - n (0.75 z)),
//                      jm = floor(n (0.5 + tt) + n (0.75 z)),
//                      ring ir = n + 1 + jp - jm, ip = (jp + jm - n + kshift + 1)/2
//   caps:              tp = frac(tt), tmp = n sqrt(3 (1 - |z|)),
//                      jp = floor(tp tmp), jm = floor((1 - tp) tmp), ir = jp + jm + 1
#include "bm_internal.cuh"

namespace bm {

namespace {

__device__ __forceinline__ int64_t ang2pix_one(int64_t nside, double z, double phi) {
    const double two_over_pi = 2.0 / 3.141592653589793;  // 2 / (FP64 pi), correctly rounded
    const double za = fabs(z);
    double tt = __dmul_rn(phi, two_over_pi);
    if (tt >= 4.0) tt = __dsub_rn(tt, 4.0);
    if (tt < 0.0) tt = __dadd_rn(tt, 4.0);
    const double nsd = (double)nside;
    if (za <= 2.0 / 3.0) {
        const double t1 = __dmul_rn(nsd, __dadd_rn(0.5, tt));
        const double t2 = __dmul_rn(nsd, __dmul_rn(z, 0.75));
        const int64_t jp = (int64_t)floor(__dsub_rn(t1, t2));
        const int64_t jm = (int64_t)floor(__dadd_rn(t1, t2));
        const int64_t ir = nside + 1 + jp - jm;
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift + 1) / 2;
        ip = ip % (4 * nside);
        return 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
    }
    const double tp = __dsub_rn(tt, floor(tt));
    const double tmp = __dmul_rn(nsd, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
    const int64_t jp = (int64_t)floor(__dmul_rn(tp, tmp));
    const int64_t jm = (int64_t)floor(__dmul_rn(__dsub_rn(1.0, tp), tmp));
    const int64_t ir = jp + jm + 1;
    int64_t ip = (int64_t)floor(__dmul_rn(tt, (double)ir));
    ip = ip % (4 * ir);
    if (z > 0.0) return 2 * ir * (ir - 1) + ip;
    return 12 * nside * nside - 2 * ir * (ir + 1) + ip;
}

__global__ void ang2pix_kernel(int64_t nside, int64_t n, const double* __restrict__ z,
                               const double* __restrict__ phi, int32_t* __restrict__ pix) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pix[i] = (int32_t)ang2pix_one(nside, z[i], phi[i]);
}

}  // namespace

void ang2pix_ring(bm_context* ctx, int64_t nside, int64_t n, const double* z, const double* phi,
                  int32_t* pix) {
    const int threads = 256;
    ang2pix_kernel<<<grid_for(ctx, (n + threads - 1) / threads, 16), threads, 0, ctx->stream>>>(
        nside, n, z, phi, pix);
    BM_LAUNCH_CHECK();
}

}  // namespace bm
