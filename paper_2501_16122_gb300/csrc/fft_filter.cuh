// Banded Toeplitz N^-1 applied by FFT overlap-save (the circulant/FFT route
// to correlated-noise weighting the paper names as future work, Sec. IV),
// with an own shared-memory Stockham FFT.
//
// For a block of H outputs of one chunk, the N = H + 2(L-1) inputs around it
// (zero outside the chunk) are transformed, multiplied by the spectrum of the
// symmetric band (real, because the band is real and even:
// K[k] = c_0 + 2 sum_{j>=1} c_j cos(2 pi j k / N)) and transformed back; the
// middle H values of the circular convolution are exactly the banded linear
// convolution (no wrap-around reaches them).  The real N-point transform is
// done as an M = N/2-point complex transform of the packed sequence
// y[2n] + i y[2n+1] with the usual even/odd split.  Per output sample this
// costs O(log N) flops instead of the 2L - 1 of the direct filter.
//
// The M-point transform runs in place in shared memory as Stockham passes of
// radix 16 for FP32, 8 for double-float and 4 for FP64, then 8, 4 or 2 for
// the last one: a thread reads its R points, applies
// the pass twiddles, does the R-point DFT in registers, and after a barrier
// writes the R results.  For radix R, current sub-transform size Ns and
// j in [0, M/R), k = j mod Ns:
//   v_r = x[j + r M/R] * W_{Ns R}^(r k),  X = DFT_R(v),  x[(j - k) R + k + r Ns] = X_r,
// which leaves the result in natural order.  The twiddles come from one
// table of W_N^q (q = 0..M) in shared memory; the buffer is padded by one
// entry every 16 so that the first pass's stride-16 writes spread over the
// banks.
#pragma once

#include <type_traits>

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
// A value as it is stored between passes: normalised for double-float.
template <typename T>
__device__ __forceinline__ cpx<T> fnorm(cpx<T> a) { return a; }

// Double-float (a pair of FP32 numbers carrying ~48 bits) as an FFT element:
// the refinement operator of the mixed solve transforms in this type on the
// FP32 pipes instead of FP64, which runs at 1/64 of the FP32 rate here.
// Inside a pass the sums and products are left unnormalised (the leading
// part from an exact two_sum / two_prod, the rounding errors and cross terms
// added into the trailing part), and every value is renormalised once when
// the pass stores it (fnorm): the trailing part stays within a few units of
// the leading part's last place over a butterfly, at about 40% fewer FP32
// operations than normalising after each operation.
__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
    const df32 s = df_two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ df32 operator-(df32 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
    const df32 p = df_two_prod(a.hi, b.hi);
    return {p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo))};
}

template <>
__device__ __forceinline__ cpx<df32> fnorm(cpx<df32> a) {
    return {df_quick_two_sum(a.x.hi, a.x.lo), df_quick_two_sum(a.y.hi, a.y.lo)};
}

// A number of type V as element type T (no detour through FP64 for FP32).
template <typename T, typename V>
__device__ __forceinline__ T fnum(V v) { return (T)v; }
template <>
__device__ __forceinline__ df32 fnum<df32, double>(double v) { return df_from(v); }
template <>
__device__ __forceinline__ df32 fnum<df32, float>(float v) { return {v, 0.f}; }
template <>
__device__ __forceinline__ df32 fnum<df32, float2>(float2 v) { return {v.x, v.y}; }
// An element as the output type.
__device__ __forceinline__ float fout(float v) { return v; }
__device__ __forceinline__ double fout(double v) { return v; }
__device__ __forceinline__ float2 fout(df32 v) {
    const df32 n = df_quick_two_sum(v.hi, v.lo);
    return make_float2(n.hi, n.lo);
}

// Padded shared-memory index: one spare entry after every 16.
__device__ __forceinline__ int fpad(int a) { return a + (a >> 4); }
__host__ __device__ inline int fft_buf_len(int M) { return M + M / 16 + 1; }

// W_16^e (forward, e = 0..15) from the exact values cos(pi/8), sin(pi/8),
// sqrt(1/2); INV conjugates.
template <typename T>
__device__ __forceinline__ cpx<T> w16(int e, bool inv) {
    const double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, r2 = 0.70710678118654752440;
    double c, s;
    switch (e & 15) {
        case 0: c = 1; s = 0; break;
        case 1: c = c1; s = s1; break;
        case 2: c = r2; s = r2; break;
        case 3: c = s1; s = c1; break;
        case 4: c = 0; s = 1; break;
        case 5: c = -s1; s = c1; break;
        case 6: c = -r2; s = r2; break;
        case 7: c = -c1; s = s1; break;
        case 8: c = -1; s = 0; break;
        case 9: c = -c1; s = -s1; break;
        case 10: c = -r2; s = -r2; break;
        case 11: c = -s1; s = -c1; break;
        case 12: c = 0; s = -1; break;
        case 13: c = s1; s = -c1; break;
        case 14: c = r2; s = -r2; break;
        default: c = c1; s = -s1; break;
    }
    return {fnum<T>(c), fnum<T>(inv ? s : -s)};  // exp(-/+ 2 pi i e / 16)
}

template <typename T>
__device__ __forceinline__ void dft2(cpx<T>* v) {
    const cpx<T> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

// In place on v[0], v[s], v[2s], v[3s].
template <typename T, int S = 1>
__device__ __forceinline__ void dft4(cpx<T>* v, bool inv) {
    const cpx<T> t0 = cadd(v[0], v[2 * S]), t1 = csub(v[0], v[2 * S]);
    const cpx<T> t2 = cadd(v[S], v[3 * S]), t3 = csub(v[S], v[3 * S]);
    v[0] = cadd(t0, t2);
    v[2 * S] = csub(t0, t2);
    // forward: X1 = t1 - i t3, X3 = t1 + i t3; inverse swaps them
    const cpx<T> mi3 = inv ? cpx<T>{-t3.y, t3.x} : cpx<T>{t3.y, -t3.x};  // -i t3 (forward), +i t3 (inverse)
    v[S] = cadd(t1, mi3);
    v[3 * S] = csub(t1, mi3);
}

// 8 = 4 x 2: x[2 n1 + n2]; a[n2][k1] = DFT4_n1, times W_8^(n2 k1); X[k1 + 4 k2] = DFT2_n2.
// The result X[r] is left in v[slot8(r)] = v[2 (r mod 4) + r / 4].
template <typename T>
__device__ __forceinline__ void dft8(cpx<T>* v, bool inv) {
    dft4<T, 2>(v, inv);      // n2 = 0: v[0], v[2], v[4], v[6] -> a[0][k1] at v[2 k1]
    dft4<T, 2>(v + 1, inv);  // n2 = 1 -> a[1][k1] at v[2 k1 + 1]
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[2 * k1 + 1] = cmul(v[2 * k1 + 1], w16<T>(2 * k1, inv));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft2<T>(v + 2 * k1);  // X[k1 + 4 k2] at v[2 k1 + k2]
}
__host__ __device__ constexpr int slot8(int r) { return 2 * (r & 3) + (r >> 2); }

// 16 = 4 x 4 (done inside the pass): x[4 n1 + n2]; a[n2][k1] = DFT4_n1, times
// W_16^(n2 k1); X[k1 + 4 k2] = DFT4_n2, left in v[slot16(r)] = v[4 (r mod 4) + r / 4].
__host__ __device__ constexpr int slot16(int r) { return 4 * (r & 3) + (r >> 2); }

// W_M^e for e in [0, M) from the table tw[q] = W_N^q, q = 0..M (N = 2M).
template <typename T>
__device__ __forceinline__ cpx<T> twid(const cpx<T>* tws, int M, int e, bool inv) {
    const int q = 2 * e;
    cpx<T> w = q <= M ? tws[q] : cpx<T>{-tws[q - M].x, -tws[q - M].y};
    if (inv) w.y = -w.y;
    return w;
}

// One in-place Stockham pass of radix R; each thread owns up to NB
// butterflies (j = threadIdx.x + b blockDim.x), whose points it holds in
// registers across the barrier between the reads and the writes.
template <typename T, int R, int NB>
__device__ __forceinline__ void fft_pass(cpx<T>* buf, int M, int Ns, const cpx<T>* tws, bool inv,
                                         const cpx<T>* ptw = nullptr) {
    const int Q = M / R;
    cpx<T> v[NB][R];
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int j = threadIdx.x + bb * blockDim.x;
        if (j < Q) {
            const int k = j & (Ns - 1);
            const int step = (M / (Ns * R)) * k;  // W_{Ns R}^(r k) = W_M^(r step)
            auto load = [&](int r) {
                cpx<T> x = buf[fpad(j + r * Q)];
                if (r > 0 && Ns > 1) {
                    cpx<T> t;
                    if (ptw) {  // the pass's own table ptw[r - 1][k]
                        t = ptw[(r - 1) * Ns + k];
                        if (inv) t.y = -t.y;
                    } else {
                        t = twid<T>(tws, M, r * step, inv);
                    }
                    x = cmul(x, t);
                }
                return x;
            };
            cpx<T>* w = v[bb];
            if (R == 16 && sizeof(T) == 4 && Ns > 1) {
                // FP32: of the pass twiddles W^(r step) read only W^step,
                // W^(2 step), W^(4 step), W^(8 step) from the table and form
                // the others with at most two complex products (a few ulp;
                // a quarter fewer shared-memory loads in this pass)
                // from the pass's own table ptw[e][k] = W^(2^e step(k)) (rows
                // of Ns consecutive entries, so a warp's loads hit distinct
                // banks), else from the shared table
                cpx<T> t1, t2, t4, t8;
                if (ptw) {
                    t1 = ptw[k]; t2 = ptw[Ns + k]; t4 = ptw[2 * Ns + k]; t8 = ptw[3 * Ns + k];
                    if (inv) { t1.y = -t1.y; t2.y = -t2.y; t4.y = -t4.y; t8.y = -t8.y; }
                } else {
                    t1 = twid<T>(tws, M, step, inv); t2 = twid<T>(tws, M, 2 * step, inv);
                    t4 = twid<T>(tws, M, 4 * step, inv); t8 = twid<T>(tws, M, 8 * step, inv);
                }
                const cpx<T> t12 = cmul(t4, t8);
#pragma unroll
                for (int n2 = 0; n2 < 4; ++n2) {
                    // the group's twiddles W^((4 n1 + n2) step), n1 = 0..3
                    const cpx<T> base = n2 == 0 ? cpx<T>{fnum<T>(1.0f), fnum<T>(0.0f)}
                                      : n2 == 1 ? t1 : n2 == 2 ? t2 : cmul(t1, t2);
                    const cpx<T> g1 = n2 == 0 ? t4 : cmul(base, t4);
                    const cpx<T> g2 = n2 == 0 ? t8 : cmul(base, t8);
                    const cpx<T> g3 = n2 == 0 ? t12 : cmul(base, t12);
                    w[n2] = buf[fpad(j + n2 * Q)];
                    if (n2 > 0) w[n2] = cmul(w[n2], base);
                    w[n2 + 4] = cmul(buf[fpad(j + (4 + n2) * Q)], g1);
                    w[n2 + 8] = cmul(buf[fpad(j + (8 + n2) * Q)], g2);
                    w[n2 + 12] = cmul(buf[fpad(j + (12 + n2) * Q)], g3);
                    dft4<T, 4>(w + n2, inv);
#pragma unroll
                    for (int k1 = 1; k1 < 4; ++k1)
                        if (n2 > 0) w[n2 + 4 * k1] = cmul(w[n2 + 4 * k1], w16<T>(n2 * k1, inv));
                }
#pragma unroll
                for (int k1 = 0; k1 < 4; ++k1) dft4<T, 1>(w + 4 * k1, inv);
            } else if (R == 16) {
                // four groups x[4 n1 + n2] (n1 = 0..3): load, first DFT-4, inner twiddles
#pragma unroll
                for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
                    for (int n1 = 0; n1 < 4; ++n1) w[n2 + 4 * n1] = load(4 * n1 + n2);
                    dft4<T, 4>(w + n2, inv);
#pragma unroll
                    for (int k1 = 1; k1 < 4; ++k1)
                        if (n2 > 0) w[n2 + 4 * k1] = cmul(w[n2 + 4 * k1], w16<T>(n2 * k1, inv));
                }
#pragma unroll
                for (int k1 = 0; k1 < 4; ++k1) dft4<T, 1>(w + 4 * k1, inv);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) w[r] = load(r);
                if (R == 8) dft8<T>(w, inv);
                else if (R == 4) dft4<T, 1>(w, inv);
                else dft2<T>(w);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int j = threadIdx.x + bb * blockDim.x;
        if (j < Q) {
            const int k = j & (Ns - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int sl = R == 16 ? slot16(r) : (R == 8 ? slot8(r) : r);
                buf[fpad(base + r * Ns)] = fnorm(v[bb][sl]);
            }
        }
    }
    __syncthreads();
}

constexpr int kFftThreads = 256;

// Radix cap and largest transform per element type (the host sizes the
// FFT within these: N <= 8192 for FP32, N <= 4096 for FP64 and double-float).
template <typename T> constexpr int kFftRadix = sizeof(T) == 4 ? 16 : (std::is_same<T, double>::value ? 4 : 8);
template <typename T> constexpr int kFftMaxM = sizeof(T) == 4 ? 4096 : 2048;

// The passes' own twiddle tables, one after another in pass order: FP32
// (radix 16) has 4 Ns entries W^(2^e step), e = 0..3, for every radix-16
// pass after the first (the other twiddles are products of these; a shorter
// last pass reads the shared table); the 16-byte types have (R - 1) Ns
// entries W^(r step), r = 1..R-1, for every pass after the first.  Ns
// consecutive entries per row, so a warp's loads hit distinct banks.
// fft_pass_tw_len gives their total length; the kernel and fft_run walk the
// passes in the same order.
template <typename T>
__host__ __device__ inline int fft_next_radix(int rem) {
    if (sizeof(T) == 4) return rem >= 16 ? 16 : rem >= 8 ? 8 : rem >= 4 ? 4 : 2;
    if (kFftRadix<T> == 8 && rem >= 8) return 8;
    return rem >= 4 ? 4 : 2;
}
template <typename T>
__host__ __device__ inline int fft_pass_tw_rows(int R) {
    return sizeof(T) == 4 ? (R == 16 ? 4 : 0) : R - 1;
}
template <typename T>
__host__ __device__ inline int fft_pass_tw_len(int M) {
    int n = 0;
    for (int Ns = 1; Ns < M;) {
        const int R = fft_next_radix<T>(M / Ns);
        if (Ns > 1) n += fft_pass_tw_rows<T>(R) * Ns;
        Ns *= R;
    }
    return n;
}
// M-point transform in place (M a power of two, M <= MMAX), forward or
// inverse (unnormalised); ends with a barrier.  RMAX caps the radix: 16
// (FP32; M <= 4096, one butterfly per thread and pass), 8 (double-float)
// or 4 (FP64, whose radix-8 butterflies spill registers); up to
// MMAX / (RMAX kFftThreads) butterflies per thread.
template <typename T, int RMAX, int MMAX>
__device__ __forceinline__ void fft_run(cpx<T>* buf, int M, const cpx<T>* tws, bool inv,
                                        const cpx<T>* ptw = nullptr) {
    static_assert(RMAX == kFftRadix<T>, "the radix follows the element type");
    static_assert(RMAX != 16 || MMAX <= 16 * kFftThreads, "one radix-16 butterfly per thread");
    constexpr int NB8 = RMAX == 16 ? 1 : (MMAX / 8 + kFftThreads - 1) / kFftThreads;
    constexpr int NB4 = RMAX == 16 ? 1 : (MMAX / 4 + kFftThreads - 1) / kFftThreads;
    constexpr int NB2 = RMAX == 16 ? 1 : (MMAX / 2 + kFftThreads - 1) / kFftThreads;
    int Ns = 1;
    while (Ns < M) {
        const int R = fft_next_radix<T>(M / Ns);
        const int rows = fft_pass_tw_rows<T>(R);
        const cpx<T>* pt = (ptw && Ns > 1 && rows) ? ptw : nullptr;
        if (R == 16) fft_pass<T, 16, 1>(buf, M, Ns, tws, inv, pt);
        else if (R == 8) fft_pass<T, 8, NB8>(buf, M, Ns, tws, inv, pt);
        else if (R == 4) fft_pass<T, 4, NB4>(buf, M, Ns, tws, inv, pt);
        else fft_pass<T, 2, NB2>(buf, M, Ns, tws, inv, pt);
        if (pt) ptw += rows * Ns;
        Ns *= R;
    }
}

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

// Table, spectrum and output types per element type: FP32 runs on FP32
// tables; FP64 reads the FP64 tables and writes FP64; double-float reads its
// spectrum as (hi, lo) pairs and the FP64 twiddles (converted once per block)
// and writes (hi, lo) pairs.
template <typename T> struct FftIO {
    using spec_t = double;
    using tw_t = double;
    using out_t = double;
};
template <> struct FftIO<df32> {
    using spec_t = float2;
    using tw_t = double;
    using out_t = float2;  // the (hi, lo) pair itself: no FP64 conversion per sample
};
template <> struct FftIO<float> {
    using spec_t = float;
    using tw_t = float;
    using out_t = float;
};

// Shared memory of the filter kernel: the padded buffer and the table.
template <typename T>
inline size_t fft_smem(int N) {
    const int M = N / 2;
    return sizeof(cpx<T>) * ((size_t)fft_buf_len(M) + (size_t)M + 1 + (size_t)fft_pass_tw_len<T>(M));
}

// One block of H = N - 2(L-1) outputs per iteration (grid-stride over blocks).
// spec: [ndet][N/2 + 1] real band spectra; tw: [N] twiddles exp(-2 pi i e / N).
template <typename T, class Src>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 3 : 2)
toeplitz_fft_kernel(Src src, const typename FftIO<T>::spec_t* __restrict__ spec,
                    const cpx<typename FftIO<T>::tw_t>* __restrict__ tw, int N, int L, FftGeom geo,
                    typename FftIO<T>::out_t* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char fft_smem_raw[];
    const int M = N / 2;
    cpx<T>* buf = reinterpret_cast<cpx<T>*>(fft_smem_raw);
    cpx<T>* tws = buf + fft_buf_len(M);  // W_N^q, q = 0..M
    for (int q = threadIdx.x; q <= M; q += kFftThreads) tws[q] = {fnum<T>(tw[q].x), fnum<T>(tw[q].y)};
    // the passes' own twiddle tables (see fft_pass_tw_len), built once
    cpx<T>* ptw = tws + M + 1;
    __syncthreads();  // the shared table is complete
    {
        cpx<T>* t = ptw;
        for (int Ns = 1; Ns < M;) {
            const int R = fft_next_radix<T>(M / Ns);
            const int rows = fft_pass_tw_rows<T>(R);
            if (Ns > 1 && rows) {
                const int stepk = M / (Ns * R);  // step = stepk k
                for (int i = threadIdx.x; i < rows * Ns; i += kFftThreads) {
                    const int e = i / Ns, k = i % Ns;
                    const int r = sizeof(T) == 4 ? (1 << e) : e + 1;
                    t[i] = twid<T>(tws, M, r * stepk * k, false);
                }
                t += rows * Ns;
            }
            Ns *= R;
        }
    }
    const int H = N - 2 * (L - 1);
    const T inv_m = fnum<T>(typename FftIO<T>::tw_t(1) / typename FftIO<T>::tw_t(M));  // M = 2^k: exact
    const T half = fnum<T>(typename FftIO<T>::tw_t(0.5));
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
        __syncthreads();  // previous block done with the buffer (and the table loaded)
        // Gather the block's inputs: for FP32 all of a thread's sample pairs
        // in flight at once (one memory latency per block of outputs; the
        // transform is short next to it), for the 8-byte types four pairs at
        // a time (their registers are taken by the transform).
        {
            constexpr int GP = sizeof(T) == 4 ? kFftMaxM<T> / kFftThreads : 4;
            using V = decltype(src(b0));
            V va[GP], vb[GP];
            // (FP32: M <= GP kFftThreads, so the loop below runs once)
            for (int n0 = 0; n0 < (sizeof(T) == 4 ? 1 : M); n0 += GP * kFftThreads) {
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                    const int n = n0 + threadIdx.x + u * kFftThreads;
                    const int64_t ta = b0 + 2 * n, tb = ta + 1;
                    va[u] = (n < M && ta >= cs && ta < ce) ? src(ta) : V{};
                    vb[u] = (n < M && tb >= cs && tb < ce) ? src(tb) : V{};
                }
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                    const int n = n0 + threadIdx.x + u * kFftThreads;
                    if (n < M) buf[fpad(n)] = {fnum<T>(va[u]), fnum<T>(vb[u])};
                }
            }
        }
        __syncthreads();
        // forward transform, spectrum product, inverse transform: one copy of
        // the transform code serves both directions
        for (int dir = 0; dir < 2; ++dir) {
            fft_run<T, kFftRadix<T>, kFftMaxM<T>>(buf, M, tws, dir == 1, ptw);
            if (dir == 1) break;
            const typename FftIO<T>::spec_t* K = spec + (int64_t)d * (M + 1);
            // Even/odd split, multiply by the real spectrum, re-pack for the
            // inverse; each thread owns the pair (k, M - k), so this runs in place.
            for (int k = threadIdx.x; k <= M / 2; k += kFftThreads) {
                const int k2 = M - k;
                const cpx<T> zk = buf[fpad(k)], zk2 = buf[fpad(k2 & (M - 1))];
                const cpx<T> wk = tws[k], wk2 = tws[k2];  // W_N^k, W_N^(M-k)
                // Y[k] = (zk + conj(zk2))/2 + W_N^k (zk - conj(zk2))/(2i)
                auto yval = [&](cpx<T> a, cpx<T> b, cpx<T> w) {
                    const cpx<T> e = {half * (a.x + b.x), half * (a.y - b.y)};
                    const cpx<T> dd = {half * (a.x - b.x), half * (a.y + b.y)};  // (a - conj b)/2
                    const cpx<T> o = {dd.y, -dd.x};                                      // / i
                    return cadd(e, cmul(w, o));
                };
                cpx<T> Yk = yval(zk, zk2, wk);
                cpx<T> Yk2 = yval(zk2, zk, wk2);
                const T Kk = fnum<T>(K[k]), Kk2 = fnum<T>(K[k2]);
                Yk = {Yk.x * Kk, Yk.y * Kk};
                Yk2 = {Yk2.x * Kk2, Yk2.y * Kk2};
                // Z'[k] = E' + i O', E' = (Y[k] + conj(Y[M-k]))/2, O' = (Y[k] - conj(Y[M-k])) conj(W_N^k)/2
                auto zval = [&](cpx<T> a, cpx<T> b, cpx<T> w) {
                    const cpx<T> e = {half * (a.x + b.x), half * (a.y - b.y)};
                    const cpx<T> dd = {half * (a.x - b.x), half * (a.y + b.y)};
                    const cpx<T> o = cmul(dd, cconj(w));
                    return cpx<T>{e.x - o.y, e.y + o.x};  // e + i o
                };
                const cpx<T> zo = zval(Yk, Yk2, wk);
                const cpx<T> zo2 = zval(Yk2, Yk, wk2);
                buf[fpad(k)] = fnorm(zo);
                if (k2 < M && k2 != k) buf[fpad(k2)] = fnorm(zo2);
            }
            __syncthreads();
        }
        const int nout = (int)(t1 - t0);
        for (int i = threadIdx.x; i < nout; i += kFftThreads) {
            const int m = L - 1 + i;
            const cpx<T> v = buf[fpad(m >> 1)];
            z[t0 + i] = fout(((m & 1) ? v.y : v.x) * inv_m);
        }
    }
}

// cost[e] = cos(2 pi e / N), e = 0..N-1, in FP64.
__global__ void cos_table_kernel(int N, double* __restrict__ cost) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x)
        cost[e] = cospi(2.0 * (double)e / (double)N);
}

// K[d][k] = c_0 + 2 sum_{j=1}^{L-1} c_j cos(2 pi j k / N), k = 0..N/2, in FP64
// (the argument reduced exactly: the integer j k mod N, stepped by k, indexes
// the table cost of cos(2 pi e / N), staged in shared memory with the
// detector's band).  Block b handles detector b / kb_per_det and the
// kBandK values of k from (b mod kb_per_det) kBandK.
constexpr int kBandK = 1024;
__global__ void band_spectrum_kernel(const double* __restrict__ coeffs, const double* __restrict__ cost, int ndet,
                                     int L, int N, int kb_per_det, double* __restrict__ spec64,
                                     float* __restrict__ spec32, float2* __restrict__ spec_df) {
    extern __shared__ __align__(16) unsigned char band_smem[];
    double* tab = reinterpret_cast<double*>(band_smem);  // [N]
    double* c = tab + N;                                 // [L]
    const int M = N / 2;
    const int d = blockIdx.x / kb_per_det;
    const int k0 = (blockIdx.x % kb_per_det) * kBandK;
    if (d >= ndet) return;
    for (int e = threadIdx.x; e < N; e += blockDim.x) tab[e] = cost[e];
    for (int j = threadIdx.x; j < L; j += blockDim.x) c[j] = coeffs[(int64_t)d * L + j];
    __syncthreads();
    for (int k = k0 + threadIdx.x; k < min(k0 + kBandK, M + 1); k += blockDim.x) {
        double s = 0.0;
        int e = 0;  // j k mod N
        for (int j = 1; j < L; ++j) {
            e += k;
            if (e >= N) e -= N;
            s += c[j] * tab[e];
        }
        const double v = c[0] + 2.0 * s;
        const int64_t i = (int64_t)d * (M + 1) + k;
        if (spec64) spec64[i] = v;
        if (spec32) spec32[i] = (float)v;
        if (spec_df) {
            const float h = (float)v;
            spec_df[i] = make_float2(h, (float)(v - (double)h));
        }
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
