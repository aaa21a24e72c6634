/*
 * Seeded synthetic CMB experiment: the inputs that both the oracle and the
 * CUDA library consume.  Nothing in this file belongs to the map-making
 * solve itself; it simulates the data that a map-maker is handed:
 *
 *   - the scan: a spinning, precessing telescope (spin axis precessing about
 *     a fixed axis on the ecliptic equator), one unit vector per detector
 *     and time sample, expressed as (z = cos(theta), phi);
 *   - the pixel each sample falls in (HEALPix RING, Gorski et al. 2005,
 *     ApJ 622:759), i.e. the simulated pointing that the experiment would
 *     deliver together with its TOD;
 *   - the polarisation angle of each sample: a per-detector angle plus twice
 *     the rotation of a continuously spinning half-wave plate;
 *   - white Gaussian noise from a counter-based generator (Philox4x32-10,
 *     Salmon, Moraes, Dror & Shaw, SC'11) so that any sample can be drawn
 *     independently of the others and of the thread count;
 *   - the time-ordered data of the paper's data model, d = s + n with
 *     s = I + Q cos 2psi + U sin 2psi (paper Eq. 1-2).
 *
 * Every routine is a pure function of its arguments and of the sample index,
 * so the output does not depend on the number of OpenMP threads.  Compiled
 * with -ffp-contract=off so that x86 and Arm hosts give the same bits for
 * the arithmetic written here (libm calls aside).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define SYN_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of the 4x32 Philox S-box  */
/* with the published multipliers and Weyl key increments.                 */
/* ---------------------------------------------------------------------- */
static inline void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        if (r < 9) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Uniform in the open interval (0, 1) with 53 random bits. */
static inline double u53(uint32_t a, uint32_t b)
{
    const uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Standard normal number n of stream `stream` under `seed` (Box-Muller on
 * the Philox block n/2; even n takes the cosine branch, odd n the sine). */
static inline double normal_at(uint64_t seed, uint32_t stream, uint64_t n)
{
    const uint64_t blk = n >> 1;
    const uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), stream, 0x5EEDu};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    synth_philox4x32_10(ctr, key, o);
    const double u1 = u53(o[0], o[1]);
    const double u2 = u53(o[2], o[3]);
    const double r = sqrt(-2.0 * log(u1));
    const double a = 2.0 * SYN_PI * u2;
    return (n & 1) ? r * sin(a) : r * cos(a);
}

static inline double uniform_at(uint64_t seed, uint32_t stream, uint64_t n)
{
    const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), stream, 0x0F1Au};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    synth_philox4x32_10(ctr, key, o);
    return u53(o[0], o[1]);
}

/* Normals start .. start+n-1 of a stream, times scale. */
void synth_normal(uint64_t seed, uint32_t stream, int64_t start, int64_t n, double scale, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = scale * normal_at(seed, stream, (uint64_t)(start + i));
}

void synth_uniform(uint64_t seed, uint32_t stream, int64_t n, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = uniform_at(seed, stream, (uint64_t)i);
}

/* ---------------------------------------------------------------------- */
/* HEALPix RING pixel of a direction (Gorski et al. 2005, Sec. 4): the     */
/* simulated experiment's pixelisation of its own pointing.                */
/* ---------------------------------------------------------------------- */
static inline int64_t syn_ang2pix_ring(int64_t nside, double z, double phi)
{
    const double za = fabs(z);
    double tt = phi * (2.0 / SYN_PI);
    if (tt >= 4.0) tt -= 4.0;
    if (tt < 0.0) tt += 4.0;
    const double nsd = (double)nside;
    if (za <= 2.0 / 3.0) {
        const double t1 = nsd * (0.5 + tt);
        const double t2 = nsd * (z * 0.75);
        const int64_t jp = (int64_t)floor(t1 - t2);
        const int64_t jm = (int64_t)floor(t1 + t2);
        const int64_t ir = nside + 1 + jp - jm;
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift + 1) / 2;
        ip = ip % (4 * nside);
        return 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
    } else {
        const double tp = tt - floor(tt);
        const double tmp = nsd * sqrt(3.0 * (1.0 - za));
        const int64_t jp = (int64_t)floor(tp * tmp);
        const int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
        const int64_t ir = jp + jm + 1;
        int64_t ip = (int64_t)floor(tt * (double)ir);
        ip = ip % (4 * ir);
        if (z > 0.0) return 2 * ir * (ir - 1) + ip;
        return 12 * nside * nside - 2 * ir * (ir + 1) + ip;
    }
}

void synth_ang2pix_ring(int64_t nside, int64_t n, const double* z, const double* phi, int32_t* pix)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) pix[i] = (int32_t)syn_ang2pix_ring(nside, z[i], phi[i]);
}

/* ---------------------------------------------------------------------- */
/* Scan law                                                                 */
/* ---------------------------------------------------------------------- */
typedef struct {
    double fsamp;          /* sampling rate [Hz]                          */
    double spin_hz;        /* spin rate [Hz]                              */
    double prec_period_s;  /* precession period [s]                       */
    double alpha_rad;      /* precession opening angle                    */
    double beta_rad;       /* spin angle (boresight to spin axis)         */
    double hwp_hz;         /* half-wave-plate rotation rate [Hz]          */
    double hwp_phase0;     /* HWP phase at t = 0 [rad]                    */
    double spin_phase0;    /* spin phase at t = 0 [rad]                   */
    double prec_phase0;    /* precession phase at t = 0 [rad]             */
} synth_scan_params;

static inline void mat_mul3(const double a[9], const double b[9], double c[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}
static inline void rot_z(double ang, double m[9])
{
    const double c = cos(ang), s = sin(ang);
    m[0] = c; m[1] = -s; m[2] = 0; m[3] = s; m[4] = c; m[5] = 0; m[6] = 0; m[7] = 0; m[8] = 1;
}
static inline void rot_y(double ang, double m[9])
{
    const double c = cos(ang), s = sin(ang);
    m[0] = c; m[1] = 0; m[2] = s; m[3] = 0; m[4] = 1; m[5] = 0; m[6] = -s; m[7] = 0; m[8] = c;
}

/* Rotation from the focal-plane frame (boresight = +z) to the sky frame at
 * time t: R = Rfix * Rz(prec) * Ry(alpha) * Rz(spin) * Ry(beta), where Rfix
 * takes the precession axis (+z of the precessing frame) to +x, a direction
 * on the ecliptic equator. */
static void scan_rotation(const synth_scan_params* sp, double t, double R[9])
{
    double a[9], b[9], c[9], d[9];
    rot_y(0.5 * SYN_PI, a);                                           /* Rfix */
    rot_z(sp->prec_phase0 + 2.0 * SYN_PI * t / sp->prec_period_s, b); /* prec */
    mat_mul3(a, b, c);
    rot_y(sp->alpha_rad, b);
    mat_mul3(c, b, d);
    rot_z(sp->spin_phase0 + 2.0 * SYN_PI * sp->spin_hz * t, b);       /* spin */
    mat_mul3(d, b, c);
    rot_y(sp->beta_rad, b);
    mat_mul3(c, b, R);
}

/*
 * Pointing of ndet detectors for samples k0 .. k0+ns-1 (time t = k / fsamp).
 * Detector d sits at focal-plane offset (ox[d], oy[d]) radians from the
 * boresight and has polarisation angle psi_det[d].  Sample (d, k) is written
 * at index d*ns + (k - k0).  Outputs z/phi may be NULL.  A sample is flagged
 * (pix = -1) with probability flag_frac, drawn from Philox stream 7.
 */
void synth_scan(const synth_scan_params* sp, int64_t nside, int32_t ndet, int64_t k0, int64_t ns,
                const double* ox, const double* oy, const double* psi_det,
                double flag_frac, uint64_t flag_seed,
                int32_t* pix, double* psi, double* z_out, double* phi_out)
{
#pragma omp parallel for schedule(static)
    for (int64_t kk = 0; kk < ns; ++kk) {
        const int64_t k = k0 + kk;
        const double t = (double)k / sp->fsamp;
        double R[9];
        scan_rotation(sp, t, R);
        const double hwp = fmod(2.0 * SYN_PI * sp->hwp_hz * t + sp->hwp_phase0, 2.0 * SYN_PI);
        for (int32_t d = 0; d < ndet; ++d) {
            /* detector direction in the focal-plane frame */
            const double v0 = sin(ox[d]) * cos(oy[d]);
            const double v1 = sin(oy[d]);
            const double v2 = cos(ox[d]) * cos(oy[d]);
            const double x = R[0] * v0 + R[1] * v1 + R[2] * v2;
            const double y = R[3] * v0 + R[4] * v1 + R[5] * v2;
            double zz = R[6] * v0 + R[7] * v1 + R[8] * v2;
            if (zz > 1.0) zz = 1.0;
            if (zz < -1.0) zz = -1.0;
            double ph = atan2(y, x);
            if (ph < 0.0) ph += 2.0 * SYN_PI;
            if (ph >= 2.0 * SYN_PI) ph -= 2.0 * SYN_PI;
            const int64_t idx = (int64_t)d * ns + kk;
            int32_t p = (int32_t)syn_ang2pix_ring(nside, zz, ph);
            if (flag_frac > 0.0 && uniform_at(flag_seed, 7u, (uint64_t)d * 0x100000000ull + (uint64_t)k) < flag_frac)
                p = -1;
            pix[idx] = p;
            double ang = fmod(psi_det[d] + 2.0 * hwp, SYN_PI);
            if (ang < 0.0) ang += SYN_PI;
            psi[idx] = ang;
            if (z_out) z_out[idx] = zz;
            if (phi_out) phi_out[idx] = ph;
        }
    }
}

/* cos 2psi and sin 2psi rounded to FP32: the precomputed pointing entries an
 * experiment may deliver instead of the angle. */
void synth_trig32(int64_t n, const double* psi, float* c32, float* s32)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double a = 2.0 * psi[i];
        c32[i] = (float)cos(a);
        s32[i] = (float)sin(a);
    }
}

/*
 * Time-ordered data of the data model (paper Eq. 1-2): for sample i in
 * pixel p = pix[i] with angle psi[i],
 *     d_i = a_I * I_p + a_P * (Q_p cos 2psi_i + U_p sin 2psi_i) + n_i,
 * with the sky map laid out [npix][3] (I, Q, U).  a_I / a_P select which
 * Stokes parameters the simulated sky contains (1 or 0).  The noise is
 *     n_i = sigma_det[d] * N(0,1; seed, stream 1, i)  +  extra[i] (if extra),
 * where d is the detector owning sample i (samples are laid out [ndet][ns]).
 * Flagged samples (pix < 0) carry noise only.  Output in FP64 (out64) or
 * rounded to FP32 (out32); one of the two is non-NULL.
 */
void synth_tod(int64_t ndet, int64_t ns, const int32_t* pix, const double* psi, const double* map,
               double a_I, double a_P, const double* sigma_det, uint64_t noise_seed,
               const double* extra, double* out64, float* out32, const float* c32, const float* s32)
{
    const int64_t n = ndet * ns;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t d = i / ns;
        double s = 0.0;
        const int32_t p = pix[i];
        if (p >= 0) {
            const double* m = map + 3 * (int64_t)p;
            double c2, s2;
            if (c32) {  /* precomputed FP32 trig: the pointing entries as delivered */
                c2 = (double)c32[i];
                s2 = (double)s32[i];
            } else {
                const double a = 2.0 * psi[i];
                c2 = cos(a);
                s2 = sin(a);
            }
            s = a_I * m[0] + a_P * (m[1] * c2 + m[2] * s2);
        }
        double v = s;
        if (sigma_det) v += sigma_det[d] * normal_at(noise_seed, 1u, (uint64_t)i);
        if (extra) v += extra[i];
        if (out64) out64[i] = v;
        else out32[i] = (float)v;
    }
}
