// Banded Toeplitz N^-1 applied by FFT overlap-save (the circulant/FFT route
// to correlated-noise weighting the paper names as future work, Sec. V),
// with an own radix-4/2 Stockham FFT in shared memory.
//
// For a block of H outputs of one chunk, the N = H + 2(L-1) inputs around it
// (zero outside the chunk) are transformed, multiplied by the spectrum of the
// symmetric band (real, because the band is real and even:
// K[k] = c_0 + 2 sum_{j>=1} c_j cos(2 pi j k / N)) and transformed back; the
// middle H values of the circular convolution are exactly the banded linear
// convolution (no wrap-around reaches them).  The real N-point transform is
// done as an N/2-point complex transform of the packed sequence
// y[2n] + i y[2n+1] with the usual even/odd split.  Per output sample this
// costs O(log N) flops instead of the 2L - 1 of the direct filter.
//
// Stockham stage (radix R, current sub-transform size Ns, M points):
//   for j in [0, M/R):  k = j mod Ns,  v_r = in[j + r M/R] * W_M^(r k M/(Ns R)),
//   X = R-point DFT of v,  out[(j - k) R + k + r Ns] = X_r
// which leaves the result in natural order after log_R(M) stages.
#pragma once

#include "bm_internal.cuh"

namespace bm {

template <typename T>
struct cpx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }

// One Stockham stage.  tw[e] = exp(-2 pi i e / (2M)) (the N-point table), so
// W_M^e = tw[2e].  INV conjugates the twiddles and the radix-4 rotation.
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_stage(const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out, int M,
                                          int Ns, const cpx<T>* __restrict__ tw) {
    const int Q = M / R;
    const int step = M / (Ns * R);
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
        const int k = j & (Ns - 1);
        const int e = k * step;
        cpx<T> v[R];
        v[0] = in[j];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            cpx<T> w = tw[2 * ((r * e) & (M - 1))];
            if (INV) w.y = -w.y;
            v[r] = cmul(in[j + r * Q], w);
        }
        const int idxD = (j - k) * R + k;
        if (R == 4) {
            const cpx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
            const cpx<T> a2 = cadd(v[1], v[3]), a3 = csub(v[1], v[3]);
            const cpx<T> mi3 = {a3.y, -a3.x};  // -i * a3
            out[idxD] = cadd(a0, a2);
            out[idxD + 2 * Ns] = csub(a0, a2);
            if (!INV) {
                out[idxD + Ns] = cadd(a1, mi3);
                out[idxD + 3 * Ns] = csub(a1, mi3);
            } else {
                out[idxD + Ns] = csub(a1, mi3);
                out[idxD + 3 * Ns] = cadd(a1, mi3);
            }
        } else {
            out[idxD] = cadd(v[0], v[1]);
            out[idxD + Ns] = csub(v[0], v[1]);
        }
    }
}

// M-point transform (M a power of two) from buf0; returns the buffer holding the result.
template <typename T, bool INV>
__device__ cpx<T>* fft_run(cpx<T>* buf0, cpx<T>* buf1, int M, const cpx<T>* __restrict__ tw) {
    cpx<T>* a = buf0;
    cpx<T>* b = buf1;
    for (int Ns = 1; Ns < M;) {
        if ((M / Ns) % 4 == 0) {
            fft_stage<T, 4, INV>(a, b, M, Ns, tw);
            Ns *= 4;
        } else {
            fft_stage<T, 2, INV>(a, b, M, Ns, tw);
            Ns *= 2;
        }
        __syncthreads();
        cpx<T>* t = a;
        a = b;
        b = t;
    }
    return a;
}

constexpr int kFftThreads = 512;

struct FftGeom {
    const int64_t* det_off;
    const int64_t* tile_start;  // [ndet + 1] prefix of output blocks per detector
    int ndet;
    int64_t chunk_len;
    int64_t tiles_per_chunk;
    int64_t ntiles;
};

__device__ __forceinline__ int fft_tile_det(const int64_t* ts, int ndet, int64_t tile) {
    int lo = 0, hi = ndet - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ts[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One block of H = N - 2(L-1) outputs per iteration (grid-stride over blocks).
// spec: [ndet][N/2 + 1] real band spectra; tw: [N] twiddles exp(-2 pi i e / N).
template <typename T, class Src>
__global__ void __launch_bounds__(kFftThreads)
toeplitz_fft_kernel(Src src, const T* __restrict__ spec, const cpx<T>* __restrict__ tw, int N, int L, FftGeom geo,
                    T* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char fft_smem[];
    const int M = N / 2;
    cpx<T>* buf0 = reinterpret_cast<cpx<T>*>(fft_smem);
    cpx<T>* buf1 = buf0 + M;
    const int H = N - 2 * (L - 1);
    const T inv_m = T(1) / T(M);
    for (int64_t tile = blockIdx.x; tile < geo.ntiles; tile += gridDim.x) {
        const int d = fft_tile_det(geo.tile_start, geo.ndet, tile);
        const int64_t local = tile - geo.tile_start[d];
        const int64_t c = local / geo.tiles_per_chunk, kk = local % geo.tiles_per_chunk;
        const int64_t cs = geo.det_off[d] + c * geo.chunk_len;
        const int64_t ce = min(cs + geo.chunk_len, geo.det_off[d + 1]);
        const int64_t t0 = cs + kk * H;
        if (t0 >= ce) continue;  // uniform across the block
        const int64_t t1 = min(t0 + (int64_t)H, ce);
        const int64_t b0 = t0 - (L - 1);
        __syncthreads();  // previous block done with the buffers
        // Gather the block's inputs: four independent sample pairs per
        // thread and pass, so their dependent loads (pixel, then map) overlap.
#pragma unroll 4
        for (int n = threadIdx.x; n < M; n += kFftThreads) {
            const int64_t ta = b0 + 2 * n, tb = ta + 1;
            const T ya = (ta >= cs && ta < ce) ? T(src(ta)) : T(0);
            const T yb = (tb >= cs && tb < ce) ? T(src(tb)) : T(0);
            buf0[n] = {ya, yb};
        }
        __syncthreads();
        cpx<T>* Z = fft_run<T, false>(buf0, buf1, M, tw);
        cpx<T>* Zo = (Z == buf0) ? buf1 : buf0;
        const T* K = spec + (int64_t)d * (M + 1);
        // Even/odd split, multiply by the real spectrum, re-pack for the inverse.
        for (int k = threadIdx.x; k <= M / 2; k += kFftThreads) {
            const int k2 = M - k;
            const cpx<T> zk = Z[k], zk2 = Z[k2 & (M - 1)];
            const cpx<T> wk = tw[k], wk2 = tw[k2];  // W_N^k, W_N^(M-k)
            // Y[k] = (zk + conj(zk2))/2 + W_N^k (zk - conj(zk2))/(2i)
            auto yval = [&](cpx<T> a, cpx<T> b, cpx<T> w) {
                const cpx<T> e = {T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y)};
                const cpx<T> dd = {T(0.5) * (a.x - b.x), T(0.5) * (a.y + b.y)};  // (a - conj b)/2
                const cpx<T> o = {dd.y, -dd.x};                                      // / i
                return cadd(e, cmul(w, o));
            };
            cpx<T> Yk = yval(zk, zk2, wk);
            cpx<T> Yk2 = yval(zk2, zk, wk2);
            const T Kk = K[k], Kk2 = K[k2];
            Yk = {Yk.x * Kk, Yk.y * Kk};
            Yk2 = {Yk2.x * Kk2, Yk2.y * Kk2};
            // Z'[k] = E' + i O', E' = (Y[k] + conj(Y[M-k]))/2, O' = (Y[k] - conj(Y[M-k])) conj(W_N^k)/2
            auto zval = [&](cpx<T> a, cpx<T> b, cpx<T> w) {
                const cpx<T> e = {T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y)};
                const cpx<T> dd = {T(0.5) * (a.x - b.x), T(0.5) * (a.y + b.y)};
                const cpx<T> o = cmul(dd, cconj(w));
                return cpx<T>{e.x - o.y, e.y + o.x};  // e + i o
            };
            Zo[k] = zval(Yk, Yk2, wk);
            if (k2 < M && k2 != k) Zo[k2] = zval(Yk2, Yk, wk2);
        }
        __syncthreads();
        cpx<T>* zo = fft_run<T, true>(Zo, Z, M, tw);
        const int nout = (int)(t1 - t0);
        for (int i = threadIdx.x; i < nout; i += kFftThreads) {
            const int m = L - 1 + i;
            const cpx<T> v = zo[m >> 1];
            z[t0 + i] = ((m & 1) ? v.y : v.x) * inv_m;
        }
    }
}

// K[d][k] = c_0 + 2 sum_{j=1}^{L-1} c_j cos(2 pi j k / N), k = 0..N/2, in FP64
// (the argument reduced exactly with the integer j k mod N).
__global__ void band_spectrum_kernel(const double* __restrict__ coeffs, int ndet, int L, int N,
                                     double* __restrict__ spec64, float* __restrict__ spec32) {
    const int M = N / 2;
    const int64_t total = (int64_t)ndet * (M + 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(i / (M + 1));
        const int k = (int)(i - (int64_t)d * (M + 1));
        const double* c = coeffs + (int64_t)d * L;
        double s = 0.0;
        for (int j = 1; j < L; ++j) {
            const int64_t e = ((int64_t)j * k) % N;
            s += c[j] * cospi(2.0 * (double)e / (double)N);
        }
        const double v = c[0] + 2.0 * s;
        if (spec64) spec64[i] = v;
        if (spec32) spec32[i] = (float)v;
    }
}

// tw[e] = exp(-2 pi i e / N), e = 0..N-1, in FP64 (rounded for FP32).
__global__ void twiddle_kernel(int N, double2* __restrict__ tw64, float2* __restrict__ tw32) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)e / (double)N, &s, &c);
        if (tw64) tw64[e] = make_double2(c, -s);
        if (tw32) tw32[e] = make_float2((float)c, (float)-s);
    }
}

}  // namespace bm
