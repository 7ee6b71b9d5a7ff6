/*
 * fram_oracle.c -- plain FP64 CPU oracle for FRAM-RIR (Luo & Gu, arXiv 2304.08052).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or constant generator
 * with the CUDA library: everything here is written straight from the paper's equations,
 * in the paper's order and notation, in double precision, with direct sin/cos evaluation
 * and no algebraic shortcuts.
 *
 * What each function follows:
 *   fo_philox4x32_10  Philox4x32-10 of Salmon, Moraes, Dror, Shaw, "Parallel random
 *                     numbers: as easy as 1, 2, 3" (SC'11): 10 rounds of the 2x(32x32->64)
 *                     multiply S-box with the Weyl key schedule.  The paper under study only
 *                     says "randomly sample" (Sec. III-B, III-C); the counter-based generator
 *                     is the chosen way to make the draws reproducible.
 *   fo_layout         RIR length L = ceil(T60 * fs) (Sec. III-D, with the output rate in place
 *                     of the paper's high rate r_h*fs) and the ragged offsets of the buffers.
 *   fo_room_stats     R = V/S of an empty rectangular room (Sec. III-A) and the Eyring
 *                     reflection coefficient r of Eq. 2.
 *   fo_sample         virtual-source sampler: Eq. 3 (quadratic distance-ratio PDF, sampled
 *                     by its inverse CDF), Eq. 4 (linear rescale to [1, c0*T60/D0]),
 *                     D_i = D0 * DR_i, azimuth/elevation on the sphere (Sec. III-B), Eq. 5
 *                     (RR_max) and Eq. 6 (reflection count with perturbation and clamp).
 *   fo_synthesize     Eq. 1 with each delta replaced by a fractional-delay Hann-windowed sinc
 *                     at the output rate; direct path with g = 0 (Sec. III-D); early RIR of
 *                     Eq. 9 as a mask on h.
 *   fo_backward       analytic gradient of a loss on h (and h_e) with respect to source, mic
 *                     and virtual-source positions, reflection counts and the coefficient.
 *   fo_sample_backward  the same gradient carried back through the sampler (Eq. 2-6): with
 *                     the random draws held fixed, images move with the source, the array and
 *                     T60, so source, mic, T60 and room-size gradients collect those paths.
 *   fo_synthesize_mr  the paper's own multi-rate output path (Sec. II-B, Eq. 7-9): impulses
 *                     quantised to the r_h fs grid, resampled to r_l fs, high-passed at 80 Hz,
 *                     resampled to fs (filter readings stated with the function).
 *   fo_spatialize     the training-data use of the RIRs (Sec. IV-A): each source signal
 *                     convolved with its RIRs, speakers scaled to a signal-to-interference
 *                     ratio against the first speaker, point-source noise to a signal-to-noise
 *                     ratio against the speech, summed into the microphone mixture; optional
 *                     per-speaker targets through a second RIR set (e.g. the early RIR, Eq. 9).
 *
 * Parity pins (what fixes each function independently of itself) live in the tests:
 *   Philox against the curand host generator; Eq. 2 against Eyring's reverberation formula;
 *   Eq. 3 by a Kolmogorov-Smirnov test; Eq. 4 end points; Eq. 5 by the 60 dB statement;
 *   Eq. 6 end points and clamp; synthesis by integer delays, band-limited interpolation of
 *   sinusoids, DTFT phase (TDOA), superposition, time shift and Schroeder decay; the
 *   gradient by central finite differences.  No function here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FO_PI 3.14159265358979323846

typedef struct {
    double alpha;         /* Eq. 3 support (alpha, beta] of the sampled distance ratio   */
    double beta;
    double a;             /* Eq. 6 perturbation p_i ~ U(a, b)                            */
    double b;
    double tau;           /* Eq. 6 distance shrinkage factor                             */
    double c0;            /* speed of sound, m/s                                         */
    double fs;            /* output sample rate, Hz                                      */
    double early_pre_ms;  /* Eq. 9 window: [-pre, +post] ms around the direct path       */
    double early_post_ms;
    int32_t half_len;     /* K: the windowed sinc spans |n - t| < K                      */
    int32_t pad_;
} fo_params;

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                                                 */
/* ------------------------------------------------------------------------------------ */
static const uint32_t FO_PHILOX_M0 = 0xD2511F53u;
static const uint32_t FO_PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t FO_PHILOX_W0 = 0x9E3779B9u;   /* golden ratio      */
static const uint32_t FO_PHILOX_W1 = 0xBB67AE85u;   /* sqrt(3) - 1       */

void fo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += FO_PHILOX_W0; k1 += FO_PHILOX_W1; }
        uint64_t p0 = (uint64_t)FO_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)FO_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void fo_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t j = 0; j < n; ++j) fo_philox4x32_10(ctr + 4 * j, key, out + 4 * j);
}

/* A 32-bit word to a uniform number in (0, 1): keep the top 23 bits and centre the
 * value in its cell, u = ((w >> 9) + 0.5) * 2^-23.  The result has at most 24 significant
 * bits, so it is exact in FP32 as well as FP64. */
static double fo_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------------------------------ */
/* Layout: L_b = ceil(T60_b * fs) samples per channel; room b holds S*M channels.        */
/* ------------------------------------------------------------------------------------ */
int fo_layout(int32_t B, int32_t S, int32_t M, double fs, const float* rt60, const int32_t* n_vs,
              int32_t* rir_len, int64_t* rir_off, int64_t* vs_off)
{
    if (B < 0 || S < 1 || M < 1 || !(fs > 0)) return -1;
    rir_off[0] = 0; vs_off[0] = 0;
    for (int32_t b = 0; b < B; ++b) {
        double t60 = (double)rt60[b];
        if (!(t60 > 0) || n_vs[b] < 0) return -1;
        double len = ceil(t60 * fs);
        if (len < 1 || len > 2147483647.0) return -1;
        rir_len[b] = (int32_t)len;
        rir_off[b + 1] = rir_off[b] + (int64_t)S * M * (int64_t)rir_len[b];
        vs_off[b + 1] = vs_off[b] + (int64_t)S * (int64_t)n_vs[b];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Room statistics (Sec. III-A) and Eyring reflection coefficient (Eq. 2).               */
/* ------------------------------------------------------------------------------------ */
static void fo_room(const double dims[3], double t60, double* R, double* r)
{
    double V = dims[0] * dims[1] * dims[2];
    double Sarea = 2.0 * (dims[0] * dims[1] + dims[0] * dims[2] + dims[1] * dims[2]);
    *R = V / Sarea;
    double e = 1.0 - exp(-0.16 * (*R) / t60);
    *r = sqrt(1.0 - e * e);
}

int fo_room_stats(int32_t B, const double* dims, const double* rt60, double* R_out, double* r_out)
{
    for (int32_t b = 0; b < B; ++b) fo_room(dims + 3 * b, rt60[b], R_out + b, r_out + b);
    return 0;
}

/* Array centre: the sphere of Sec. III-B is centred on the mean of the microphones. */
static void fo_centre(int32_t M, const double* mic_b, double c[3])
{
    c[0] = c[1] = c[2] = 0.0;
    for (int32_t m = 0; m < M; ++m) { c[0] += mic_b[3 * m]; c[1] += mic_b[3 * m + 1]; c[2] += mic_b[3 * m + 2]; }
    c[0] /= M; c[1] /= M; c[2] /= M;
}

static double fo_dist(const double* p, const double* q)
{
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Eq. 5: the reflection count at which the farthest image (distance c0*T60) is 60 dB
 * below the direct path. */
static double fo_rrmax(double c0, double t60, double d0, double r)
{
    return (log10(c0 * t60) - log10(d0) - 3.0) / log10(r);
}

/* ------------------------------------------------------------------------------------ */
/* Virtual-source sampler (Sec. III-B, III-C).                                           */
/* For room b, source s, image i: one Philox call with counter (i, s, b, 0) and key      */
/* (b replaced by room_ids[b] when given)                                                */
/* (seed_lo, seed_hi) gives u0..u3.  u0 -> distance ratio, u1 -> azimuth, u2 ->          */
/* elevation, u3 -> perturbation.                                                        */
/* Outputs per image: position (FP64), g_i; optionally the raw words, D_i, x, DR.        */
/* Per room: r; per (room, source): RR_max and D0.                                       */
/* ------------------------------------------------------------------------------------ */
int fo_sample(int32_t B, int32_t S, int32_t M,
              const double* dims, const double* rt60, const double* src, const double* mic,
              const int32_t* n_vs, const int64_t* vs_off, const fo_params* P, uint64_t seed,
              double* vs_pos, double* vs_g, double* r_out,
              uint32_t* words, double* vs_dist, double* vs_x, double* rrmax_out, double* d0_out,
              const int32_t* room_ids)
{
    const double alpha = P->alpha, beta = P->beta, c0 = P->c0;
    if (!(alpha > 0) || !(beta > alpha) || !(beta <= 1.0) || !(c0 > 0) || !(P->tau > 0)) return -1;
    const uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t b = 0; b < B; ++b) {
        const double t60 = rt60[b];
        double R, r;
        fo_room(dims + 3 * b, t60, &R, &r);
        if (r_out) r_out[b] = r;
        double c[3];
        fo_centre(M, mic + (int64_t)3 * M * b, c);
        for (int32_t s = 0; s < S; ++s) {
            const double* ps = src + 3 * ((int64_t)b * S + s);
            /* d0 in Eq. 4 and Eq. 5 is the direct-path distance D0 to the sphere centre. */
            const double D0 = fo_dist(ps, c);
            const double cT = c0 * t60;
            if (!(cT > D0) || !(D0 > 0)) { bad = 1; continue; }
            const double RRmax = fo_rrmax(c0, t60, D0, r);
            if (rrmax_out) rrmax_out[(int64_t)b * S + s] = RRmax;
            if (d0_out) d0_out[(int64_t)b * S + s] = D0;
            for (int32_t i = 0; i < n_vs[b]; ++i) {
                const int64_t v = vs_off[b] + (int64_t)s * n_vs[b] + i;
                /* room_ids (nullable) gives the room's index in a larger batch, so a subset of
                 * rooms draws exactly what it draws inside the full batch. */
                const uint32_t rid = room_ids ? (uint32_t)room_ids[b] : (uint32_t)b;
                const uint32_t ctr[4] = { (uint32_t)i, (uint32_t)s, rid, 0u };
                uint32_t w[4];
                fo_philox4x32_10(ctr, key, w);
                if (words) memcpy(words + 4 * v, w, sizeof w);
                const double u0 = fo_uniform(w[0]), u1 = fo_uniform(w[1]);
                const double u2 = fo_uniform(w[2]), u3 = fo_uniform(w[3]);
                /* Eq. 3: P(x) = 3x^2/(beta^3 - alpha^3) on (alpha, beta]; inverse CDF. */
                const double x = cbrt(alpha * alpha * alpha + u0 * (beta * beta * beta - alpha * alpha * alpha));
                /* Eq. 4: linear rescale of x from [alpha, beta] to DR in [1, c0*T60/D0]. */
                const double DR = 1.0 + alpha / (beta - alpha) * (x / alpha - 1.0) * (cT / D0 - 1.0);
                const double Di = D0 * DR;
                /* Sec. III-B: azimuth U[0, 2pi], elevation U[-pi/2, pi/2]. */
                const double theta = 2.0 * FO_PI * u1;
                const double phi = FO_PI * (u2 - 0.5);
                double* pos = vs_pos + 3 * v;
                pos[0] = c[0] + Di * cos(phi) * cos(theta);
                pos[1] = c[1] + Di * cos(phi) * sin(theta);
                pos[2] = c[2] + Di * sin(phi);
                /* Eq. 6. */
                const double p = P->a + (P->b - P->a) * u3;
                double g = 1.0 + (Di / cT) * (Di / cT) * (RRmax - 1.0) + p * pow(DR, P->tau);
                g = fmax(fmin(g, RRmax), 1.0);
                vs_g[v] = g;
                if (vs_dist) vs_dist[v] = Di;
                if (vs_x) vs_x[v] = x;
            }
        }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* Fractional-delay Hann-windowed sinc.                                                  */
/* tap(x) = sinc(x) * w(x) for |x| < K, with sinc(x) = sin(pi x)/(pi x) (1 at 0) and     */
/* w(x) = (1 + cos(pi x / K)) / 2; zero elsewhere.                                       */
/* ------------------------------------------------------------------------------------ */
static double fo_sinc(double x) { return x == 0.0 ? 1.0 : sin(FO_PI * x) / (FO_PI * x); }
static double fo_dsinc(double x) { return x == 0.0 ? 0.0 : (cos(FO_PI * x) - fo_sinc(x)) / x; }
static double fo_hann(double x, int K) { return 0.5 * (1.0 + cos(FO_PI * x / K)); }
static double fo_dhann(double x, int K) { return -0.5 * (FO_PI / K) * sin(FO_PI * x / K); }

/* Add A * tap(n - t) for every n in [0, L) with |n - t| < K. */
static void fo_add_impulse(double* h, int32_t L, int K, double t, double A)
{
    int64_t n0 = (int64_t)ceil(t - K), n1 = (int64_t)floor(t + K);
    if (n0 < 0) n0 = 0;
    if (n1 > L - 1) n1 = L - 1;
    for (int64_t n = n0; n <= n1; ++n) {
        double x = (double)n - t;
        if (fabs(x) < K) h[n] += A * fo_sinc(x) * fo_hann(x, K);
    }
}

/* Eq. 9 window, per mic: n0 = ceil(D_{0,m} fs/c0), keep -ceil(pre*fs/1000) <= n - n0 <=
 * ceil(post*fs/1000). */
static void fo_early_window(const fo_params* P, double d0m, int64_t* lo, int64_t* hi)
{
    int64_t n0 = (int64_t)ceil(d0m * P->fs / P->c0);
    *lo = n0 - (int64_t)ceil(P->early_pre_ms * P->fs / 1000.0);
    *hi = n0 + (int64_t)ceil(P->early_post_ms * P->fs / 1000.0);
}

/*
 * h^m[n] for every room b, source s, mic m (Eq. 1 with windowed sincs):
 *   direct path: amplitude 1/D_{0,m}, delay D_{0,m} fs/c0 (g = 0);
 *   image i:     amplitude r^{g_i}/D_{i,m}, delay D_{i,m} fs/c0.
 * Images are summed after the direct path in ascending i.  Layout: rir[rir_off[b] +
 * ((s*M)+m)*L_b + n].  early (nullable) receives h_e of Eq. 9.
 */
int fo_synthesize(int32_t B, int32_t S, int32_t M, const double* src, const double* mic,
                  const int32_t* n_vs, const int64_t* vs_off, const int32_t* rir_len, const int64_t* rir_off,
                  const double* vs_pos, const double* vs_g, const double* r, const fo_params* P,
                  double* rir, double* early)
{
    const int K = P->half_len;
    if (K < 1) return -1;
    const double q = P->fs / P->c0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t b = 0; b < B; ++b) {
        const int32_t L = rir_len[b];
        for (int32_t s = 0; s < S; ++s) {
            const double* ps = src + 3 * ((int64_t)b * S + s);
            for (int32_t m = 0; m < M; ++m) {
                const double* pm = mic + 3 * ((int64_t)b * M + m);
                double* h = rir + rir_off[b] + ((int64_t)s * M + m) * L;
                memset(h, 0, sizeof(double) * (size_t)L);
                const double D0m = fo_dist(ps, pm);
                fo_add_impulse(h, L, K, D0m * q, 1.0 / D0m);
                for (int32_t i = 0; i < n_vs[b]; ++i) {
                    const int64_t v = vs_off[b] + (int64_t)s * n_vs[b] + i;
                    const double D = fo_dist(vs_pos + 3 * v, pm);
                    fo_add_impulse(h, L, K, D * q, pow(r[b], vs_g[v]) / D);
                }
                if (early) {
                    double* he = early + rir_off[b] + ((int64_t)s * M + m) * L;
                    int64_t lo, hi;
                    fo_early_window(P, D0m, &lo, &hi);
                    for (int64_t n = 0; n < L; ++n) he[n] = (n >= lo && n <= hi) ? h[n] : 0.0;
                }
            }
        }
    }
    return 0;
}

/*
 * Gradient of a scalar loss given dL/dh (grad_rir, same layout as h) and optionally
 * dL/dh_e (grad_early).  h_e = mask * h, so the effective upstream gradient is
 * G = grad_rir + mask * grad_early.  For each impulse with delay t = D fs/c0 and
 * amplitude A:
 *   dL/dt = sum_n G[n] * A * d/dt[tap(n - t)] = -A sum_n G[n] tap'(n - t)
 *   dL/dA = sum_n G[n] * tap(n - t)
 *   dL/dD = dL/dt * fs/c0 + dL/dA * dA/dD,   dA/dD = -A/D
 *   images: dL/dr += dL/dA * g * A / r   (A = r^g / D)
 *   dD/d(position) = (position - mic)/D = -dD/d(mic).
 * Images are leaves: they do not move with the source, so the source gradient comes from
 * the direct path only.  Outputs are overwritten (each nullable).
 */
int fo_backward(int32_t B, int32_t S, int32_t M, const double* src, const double* mic,
                const int32_t* n_vs, const int64_t* vs_off, const int32_t* rir_len, const int64_t* rir_off,
                const double* vs_pos, const double* vs_g, const double* r, const fo_params* P,
                const double* grad_rir, const double* grad_early,
                double* grad_vs, double* grad_mic, double* grad_src, double* grad_r, double* grad_g)
{
    const int K = P->half_len;
    if (K < 1) return -1;
    const double q = P->fs / P->c0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t b = 0; b < B; ++b) {
        const int32_t L = rir_len[b];
        double* G = (double*)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
        double gr = 0.0;
        if (grad_mic) for (int j = 0; j < 3 * M; ++j) grad_mic[(int64_t)3 * M * b + j] = 0.0;
        if (grad_vs) for (int64_t v = 3 * vs_off[b]; v < 3 * vs_off[b + 1]; ++v) grad_vs[v] = 0.0;
        if (grad_g) for (int64_t v = vs_off[b]; v < vs_off[b + 1]; ++v) grad_g[v] = 0.0;
        for (int32_t s = 0; s < S; ++s) {
            const double* ps = src + 3 * ((int64_t)b * S + s);
            double gsrc[3] = { 0.0, 0.0, 0.0 };
            for (int32_t m = 0; m < M; ++m) {
                const double* pm = mic + 3 * ((int64_t)b * M + m);
                const int64_t base = rir_off[b] + ((int64_t)s * M + m) * L;
                const double D0m = fo_dist(ps, pm);
                int64_t lo, hi;
                fo_early_window(P, D0m, &lo, &hi);
                for (int64_t n = 0; n < L; ++n) {
                    G[n] = grad_rir ? grad_rir[base + n] : 0.0;
                    if (grad_early && n >= lo && n <= hi) G[n] += grad_early[base + n];
                }
                for (int32_t i = -1; i < n_vs[b]; ++i) {
                    const double* pp;
                    double A, g = 0.0;
                    int64_t v = -1;
                    double D;
                    if (i < 0) { pp = ps; D = D0m; A = 1.0 / D; }
                    else {
                        v = vs_off[b] + (int64_t)s * n_vs[b] + i;
                        pp = vs_pos + 3 * v; D = fo_dist(pp, pm); g = vs_g[v];
                        A = pow(r[b], g) / D;
                    }
                    const double t = D * q;
                    double dLdt = 0.0, dLdA = 0.0;
                    int64_t n0 = (int64_t)ceil(t - K), n1 = (int64_t)floor(t + K);
                    if (n0 < 0) n0 = 0;
                    if (n1 > L - 1) n1 = L - 1;
                    for (int64_t n = n0; n <= n1; ++n) {
                        const double x = (double)n - t;
                        if (!(fabs(x) < K)) continue;
                        const double tap = fo_sinc(x) * fo_hann(x, K);
                        const double dtap = fo_dsinc(x) * fo_hann(x, K) + fo_sinc(x) * fo_dhann(x, K);
                        dLdA += G[n] * tap;
                        dLdt += -A * G[n] * dtap;
                    }
                    const double dLdD = dLdt * q - dLdA * A / D;
                    const double e[3] = { (pp[0] - pm[0]) / D, (pp[1] - pm[1]) / D, (pp[2] - pm[2]) / D };
                    for (int k = 0; k < 3; ++k) {
                        if (grad_mic) grad_mic[3 * ((int64_t)b * M + m) + k] -= dLdD * e[k];
                        if (i < 0) gsrc[k] += dLdD * e[k];
                        else if (grad_vs) grad_vs[3 * v + k] += dLdD * e[k];
                    }
                    if (i >= 0) gr += dLdA * g * A / r[b];
                    if (i >= 0 && grad_g) grad_g[v] += dLdA * A * log(r[b]);   /* dA/dg = A ln r */
                }
            }
            if (grad_src) for (int k = 0; k < 3; ++k) grad_src[3 * ((int64_t)b * S + s) + k] = gsrc[k];
        }
        if (grad_r) grad_r[b] = gr;
        free(G);
    }
    return 0;
}

/*
 * Reparameterised gradient through the sampler (Sec. III-B, III-C; Eq. 2-6), for the continuous
 * synthesis.  With the Philox draws (u0..u3) of every image held fixed, an image is
 *   p_i = c + D_i nu_i,  D_i = D0 DR_i,  DR_i = 1 + k_i (c0 T60 / D0 - 1),  k_i = (x_i - alpha)/(beta - alpha),
 *   g_i = clamp(1 + (D_i / (c0 T60))^2 (RR_max - 1) + p_i DR_i^tau, 1, RR_max),
 * with c the mean of the mics, D0 = |src - c|, RR_max from Eq. 5 and r from Eq. 2 (R = V/S).
 * Inputs: dL/dp_i (grad_vs), dL/dg_i (grad_g), dL/dr through the amplitudes (grad_r_amp) and the
 * direct-path source and mic gradients (grad_src_dir, grad_mic_dir), all from fo_backward.
 * Outputs (each overwritten): total source and mic gradients, dL/dT60 and dL/d(room size).
 */
int fo_sample_backward(int32_t B, int32_t S, int32_t M,
                       const double* dims, const double* rt60, const double* src, const double* mic,
                       const int32_t* n_vs, const int64_t* vs_off, const fo_params* P, uint64_t seed,
                       const int32_t* room_ids,
                       const double* grad_vs, const double* grad_g, const double* grad_r_amp,
                       const double* grad_src_dir, const double* grad_mic_dir,
                       double* grad_src, double* grad_mic, double* grad_t60, double* grad_dims)
{
    const double alpha = P->alpha, beta = P->beta, c0 = P->c0, tau = P->tau;
    if (!(alpha > 0) || !(beta > alpha) || !(beta <= 1.0) || !(c0 > 0) || !(tau > 0)) return -1;
    const uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t b = 0; b < B; ++b) {
        const double t60 = rt60[b];
        const double* d = dims + 3 * b;
        double R, r;
        fo_room(d, t60, &R, &r);
        double c[3];
        fo_centre(M, mic + (int64_t)3 * M * b, c);
        const double cT = c0 * t60, lnr = log(r);
        double dLdc[3] = { 0.0, 0.0, 0.0 };
        double dLdcT = 0.0, dLdr = grad_r_amp ? grad_r_amp[b] : 0.0;
        for (int32_t s = 0; s < S; ++s) {
            const double* ps = src + 3 * ((int64_t)b * S + s);
            const double D0 = fo_dist(ps, c);
            if (!(cT > D0) || !(D0 > 0)) { bad = 1; continue; }
            const double RRmax = fo_rrmax(c0, t60, D0, r);
            double dLdD0 = 0.0, dLdRR = 0.0;
            for (int32_t i = 0; i < n_vs[b]; ++i) {
                const int64_t v = vs_off[b] + (int64_t)s * n_vs[b] + i;
                const uint32_t rid = room_ids ? (uint32_t)room_ids[b] : (uint32_t)b;
                const uint32_t ctr[4] = { (uint32_t)i, (uint32_t)s, rid, 0u };
                uint32_t w[4];
                fo_philox4x32_10(ctr, key, w);
                const double u0 = fo_uniform(w[0]), u1 = fo_uniform(w[1]);
                const double u2 = fo_uniform(w[2]), u3 = fo_uniform(w[3]);
                const double x = cbrt(alpha * alpha * alpha + u0 * (beta * beta * beta - alpha * alpha * alpha));
                const double k = (x - alpha) / (beta - alpha);
                const double DR = 1.0 + alpha / (beta - alpha) * (x / alpha - 1.0) * (cT / D0 - 1.0);
                const double Di = D0 * DR;
                const double theta = 2.0 * FO_PI * u1, phi = FO_PI * (u2 - 0.5);
                const double nu[3] = { cos(phi) * cos(theta), cos(phi) * sin(theta), sin(phi) };
                const double p = P->a + (P->b - P->a) * u3;
                const double graw = 1.0 + (Di / cT) * (Di / cT) * (RRmax - 1.0) + p * pow(DR, tau);
                const double* gp = grad_vs + 3 * v;
                const double gg = grad_g ? grad_g[v] : 0.0;
                /* position path: p_i = c + D_i nu_i */
                double dLdDi = gp[0] * nu[0] + gp[1] * nu[1] + gp[2] * nu[2];
                for (int j = 0; j < 3; ++j) dLdc[j] += gp[j];
                /* reflection-count path (Eq. 6), zero where the clamp holds g at 1 */
                double dLdD0_g = 0.0, dLdcT_g = 0.0;
                if (graw > RRmax) {
                    dLdRR += gg;
                } else if (graw >= 1.0) {
                    dLdDi += gg * (2.0 * Di / (cT * cT) * (RRmax - 1.0) + p * tau * pow(DR, tau - 1.0) / D0);
                    dLdD0_g = gg * (-p * tau * pow(DR, tau - 1.0) * Di / (D0 * D0));
                    dLdcT_g = gg * (-2.0 * Di * Di / (cT * cT * cT) * (RRmax - 1.0));
                    dLdRR += gg * (Di / cT) * (Di / cT);
                }
                /* D_i = D0 (1 - k) + k c0 T60 (Eq. 4) */
                dLdD0 += dLdDi * (1.0 - k) + dLdD0_g;
                dLdcT += dLdDi * k + dLdcT_g;
            }
            /* Eq. 5: RR_max = (log10(c0 T60) - log10(D0) - 3) / log10(r) */
            dLdD0 += dLdRR * (-1.0 / (D0 * lnr));
            dLdcT += dLdRR * (1.0 / (cT * lnr));
            dLdr += dLdRR * (-RRmax / (r * lnr));
            /* D0 = |src - c| */
            for (int j = 0; j < 3; ++j) {
                const double u = (ps[j] - c[j]) / D0;
                grad_src[3 * ((int64_t)b * S + s) + j] = (grad_src_dir ? grad_src_dir[3 * ((int64_t)b * S + s) + j] : 0.0)
                                                         + dLdD0 * u;
                dLdc[j] -= dLdD0 * u;
            }
        }
        /* c = mean of the mics */
        for (int32_t m = 0; m < M; ++m)
            for (int j = 0; j < 3; ++j)
                grad_mic[3 * ((int64_t)b * M + m) + j] = (grad_mic_dir ? grad_mic_dir[3 * ((int64_t)b * M + m) + j] : 0.0)
                                                         + dLdc[j] / M;
        /* Eq. 2: r = sqrt(1 - e^2), e = 1 - exp(-0.16 R / T60), R = V / S */
        const double ex = exp(-0.16 * R / t60);
        const double e = 1.0 - ex;
        const double dr_de = -e / r;
        const double dLde = dLdr * dr_de;
        grad_t60[b] = dLdcT * c0 + dLde * (-ex * 0.16 * R / (t60 * t60));
        const double dLdR = dLde * (ex * 0.16 / t60);
        const double V = d[0] * d[1] * d[2];
        const double Sa = 2.0 * (d[0] * d[1] + d[0] * d[2] + d[1] * d[2]);
        const double dVd[3] = { d[1] * d[2], d[0] * d[2], d[0] * d[1] };
        const double dSd[3] = { 2.0 * (d[1] + d[2]), 2.0 * (d[0] + d[2]), 2.0 * (d[0] + d[1]) };
        for (int j = 0; j < 3; ++j) grad_dims[3 * b + j] = dLdR * (dVd[j] / Sa - V * dSd[j] / (Sa * Sa));
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* Multi-rate output path as the paper prints it (Sec. II-B, Eq. 7-9): impulses on a grid  */
/* at the high rate r_h fs, q = min(ceil(D r_h fs / c0), L_h - 1), L_h = ceil(T60 r_h fs),  */
/* h[q] += r^g / D; then down to r_l fs, an 80 Hz high-pass, and down to fs, with          */
/* r_h = floor(1e6 / fs), r_l = floor(sqrt(r_h)).  The paper does not specify the filters;  */
/* the readings used here:                                                                 */
/*   resampling by up/down (reduced): y[k] = sum_n x[n] F(k down - n up), F centred (zero   */
/*     phase), F(m) = lowpass with cutoff pi / max(up, down) times a Kaiser window (beta 5) */
/*     on |m| <= HL = 10 max(up, down), scaled so that sum_m F(m) = up;                     */
/*   the high-pass: 2nd-order Butterworth at 80 Hz, bilinear transform with the cutoff     */
/*     pre-warped, run forward from a zero state over the intermediate signal;             */
/*   signal lengths: intermediate L_m = ceil(L_h up / down) (zero outside), output L =      */
/*     ceil(T60 fs) as in the continuous path.                                              */
/* ------------------------------------------------------------------------------------ */

void fo_mr_rates(double fs, int32_t* rh, int32_t* rl)
{
    *rh = (int32_t)floor(1.0e6 / fs);
    *rl = (int32_t)floor(sqrt((double)*rh));
}

static int32_t fo_gcd(int32_t a, int32_t b)
{
    while (b) { int32_t t = a % b; a = b; b = t; }
    return a;
}

/* Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2. */
static double fo_bessel_i0(double x)
{
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= (x / (2.0 * k)) * (x / (2.0 * k));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* The resampling filter for a reduced ratio up/down: F[m + HL] for |m| <= HL.  Returns HL. */
int32_t fo_resample_filter(int32_t up, int32_t down, double* F /* [2 HL + 1], may be NULL */)
{
    const int32_t mx = up > down ? up : down;
    const int32_t HL = 10 * mx;
    if (!F) return HL;
    const double beta = 5.0, i0b = fo_bessel_i0(beta);
    double sum = 0.0;
    for (int32_t m = -HL; m <= HL; ++m) {
        const double x = (double)m / (double)mx;                   /* lowpass, cutoff pi / mx */
        const double lp = fo_sinc(x) / (double)mx;
        const double rr = (double)m / (double)HL;
        const double w = fo_bessel_i0(beta * sqrt(fmax(0.0, 1.0 - rr * rr))) / i0b;
        F[m + HL] = lp * w;
        sum += F[m + HL];
    }
    for (int32_t m = 0; m <= 2 * HL; ++m) F[m] *= (double)up / sum;
    return HL;
}

/* 2nd-order Butterworth high-pass at fc for sample rate fsr (bilinear, pre-warped):
 * H(z) = (b0 + b1 z^-1 + b2 z^-2) / (1 + a1 z^-1 + a2 z^-2). */
void fo_hpf_coeffs(double fc, double fsr, double b[3], double a[3])
{
    const double k = tan(FO_PI * fc / fsr);
    const double s2 = sqrt(2.0);
    const double den = 1.0 + s2 * k + k * k;
    b[0] = 1.0 / den;
    b[1] = -2.0 / den;
    b[2] = 1.0 / den;
    a[0] = 1.0;
    a[1] = 2.0 * (k * k - 1.0) / den;
    a[2] = (1.0 - s2 * k + k * k) / den;
}

/* One channel: the high-rate impulses (q_j, A_j) -> y[0, L) at fs. */
static void fo_mr_channel(int64_t nimp, const int64_t* q, const double* A, int64_t Lh, int32_t upA, int32_t downA,
                          const double* FA, int32_t HLA, int32_t rl, const double* FC, int32_t HLC,
                          const double hb[3], const double ha[3], int32_t L, double* y, double* z /* [Lm] */)
{
    const int64_t Lm = (Lh * upA + downA - 1) / downA;
    for (int64_t k = 0; k < Lm; ++k) z[k] = 0.0;
    /* stage A: y1[k] = sum_j A_j F_A(k downA - q_j upA) */
    for (int64_t j = 0; j < nimp; ++j) {
        const int64_t c = q[j] * upA;
        int64_t k0 = (c - HLA + downA - 1) / downA;     /* ceil for c - HLA >= 0 */
        if (c - HLA < 0) k0 = -((HLA - c) / downA);      /* ceil of a negative ratio */
        for (int64_t k = k0; k * downA - c <= HLA; ++k) {
            if (k < 0 || k >= Lm) continue;
            const int64_t m = k * downA - c;
            if (m >= -HLA) z[k] += A[j] * FA[m + HLA];
        }
    }
    /* the high-pass, in place */
    double x1 = 0.0, x2 = 0.0, y1 = 0.0, y2 = 0.0;
    for (int64_t k = 0; k < Lm; ++k) {
        const double x0 = z[k];
        const double y0 = hb[0] * x0 + hb[1] * x1 + hb[2] * x2 - ha[1] * y1 - ha[2] * y2;
        x2 = x1; x1 = x0; y2 = y1; y1 = y0;
        z[k] = y0;
    }
    /* stage C: y[n] = sum_k z[k] F_C(n rl - k) */
    for (int32_t n = 0; n < L; ++n) {
        double acc = 0.0;
        for (int64_t k = (int64_t)n * rl - HLC; k <= (int64_t)n * rl + HLC; ++k)
            if (k >= 0 && k < Lm) acc += z[k] * FC[(int64_t)n * rl - k + HLC];
        y[n] = acc;
    }
}

/*
 * The multi-rate RIRs (and early RIRs, Eq. 9 applied on the high-rate grid around
 * n0 = ceil(D_{0,m} r_h fs / c0)) in the layout of fo_synthesize.  Returns -1 on bad
 * parameters, -2 when out of memory.
 */
int fo_synthesize_mr(int32_t B, int32_t S, int32_t M, const double* src, const double* mic, const double* rt60,
                     const int32_t* n_vs, const int64_t* vs_off, const int32_t* rir_len, const int64_t* rir_off,
                     const double* vs_pos, const double* vs_g, const double* r, const fo_params* P,
                     double* rir, double* early)
{
    int32_t rh, rl;
    fo_mr_rates(P->fs, &rh, &rl);
    if (rh < 1 || rl < 1) return -1;
    const int32_t g = fo_gcd(rh, rl), upA = rl / g, downA = rh / g;
    const int32_t HLA = fo_resample_filter(upA, downA, NULL), HLC = fo_resample_filter(1, rl, NULL);
    double* FA = (double*)malloc(sizeof(double) * (size_t)(2 * HLA + 1));
    double* FC = (double*)malloc(sizeof(double) * (size_t)(2 * HLC + 1));
    if (!FA || !FC) { free(FA); free(FC); return -2; }
    fo_resample_filter(upA, downA, FA);
    fo_resample_filter(1, rl, FC);
    double hb[3], ha[3];
    fo_hpf_coeffs(80.0, (double)rl * P->fs, hb, ha);
    const double fh = (double)rh * P->fs;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t b = 0; b < B; ++b) {
        const int32_t L = rir_len[b];
        const int64_t Lh = (int64_t)ceil(rt60[b] * fh);
        const int64_t Lm = (Lh * upA + downA - 1) / downA;
        const int64_t n = n_vs[b] + 1;
        int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        int64_t* qe = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        double* A = (double*)malloc(sizeof(double) * (size_t)n);
        double* Ae = (double*)malloc(sizeof(double) * (size_t)n);
        double* z = (double*)malloc(sizeof(double) * (size_t)(Lm > 0 ? Lm : 1));
        if (!q || !qe || !A || !Ae || !z) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int32_t s = 0; s < S; ++s) {
                const double* ps = src + 3 * ((int64_t)b * S + s);
                for (int32_t m = 0; m < M; ++m) {
                    const double* pm = mic + 3 * ((int64_t)b * M + m);
                    /* Eq. 7-8: the direct path (g = 0), then the images in ascending i */
                    const double D0m = fo_dist(ps, pm);
                    int64_t cnt = 0;
                    q[cnt] = (int64_t)ceil(D0m / P->c0 * fh);
                    if (q[cnt] > Lh - 1) q[cnt] = Lh - 1;
                    A[cnt++] = 1.0 / D0m;
                    for (int32_t i = 0; i < n_vs[b]; ++i) {
                        const int64_t v = vs_off[b] + (int64_t)s * n_vs[b] + i;
                        const double D = fo_dist(vs_pos + 3 * v, pm);
                        int64_t qi = (int64_t)ceil(D / P->c0 * fh);
                        if (qi > Lh - 1) qi = Lh - 1;
                        q[cnt] = qi;
                        A[cnt++] = pow(r[b], vs_g[v]) / D;
                    }
                    double* h = rir + rir_off[b] + ((int64_t)s * M + m) * L;
                    fo_mr_channel(cnt, q, A, Lh, upA, downA, FA, HLA, rl, FC, HLC, hb, ha, L, h, z);
                    if (early) {
                        /* Eq. 9 on the high-rate grid */
                        const int64_t n0 = (int64_t)ceil(D0m / P->c0 * fh);
                        const int64_t lo = n0 - (int64_t)ceil(P->early_pre_ms * fh / 1000.0);
                        const int64_t hi = n0 + (int64_t)ceil(P->early_post_ms * fh / 1000.0);
                        int64_t ce = 0;
                        for (int64_t j = 0; j < cnt; ++j)
                            if (q[j] >= lo && q[j] <= hi) { qe[ce] = q[j]; Ae[ce++] = A[j]; }
                        double* he = early + rir_off[b] + ((int64_t)s * M + m) * L;
                        fo_mr_channel(ce, qe, Ae, Lh, upA, downA, FA, HLA, rl, FC, HLC, hb, ha, L, he, z);
                    }
                }
            }
        }
        free(q); free(qe); free(A); free(Ae); free(z);
    }
    free(FA);
    free(FC);
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* Spatialisation (Sec. IV-A).  Readings (the paper names the quantities, not the formulas): */
/*   image   y_{s,m}[n] = sum_{k=0}^{min(L-1, n)} h_{s,m}[k] x_s[n - k],  n in [0, N)       */
/*           (causal convolution kept on the mixture's N samples);                           */
/*   energy  E_s = sum_n y_{s,0}[n]^2 at the reference mic 0;                                 */
/*   gains   g_0 = 1; speaker s in [1, n_speech): g_s = sqrt(E_0 / E_s * 10^(-l_s/10)), so    */
/*           10 log10(E_0 / (g_s^2 E_s)) = l_s (the SIR in dB); the speech at mic 0           */
/*           v[n] = sum_{s < n_speech} g_s y_{s,0}[n]; noise s >= n_speech:                     */
/*           g_s = sqrt(E_v / E_s * 10^(-l_s/10)), E_v = sum_n v[n]^2 (l_s = the SNR in dB);   */
/*           a silent image (E_s = 0) gets g_s = 0;                                             */
/*   outputs mix_m[n] = sum_s g_s y_{s,m}[n]; targets t_{s,m}[n] = g_s (h'_{s,m} * x_s)[n] for */
/*           s < n_speech with a second RIR set h' (the early RIR of Eq. 9, or h itself).      */
/* ------------------------------------------------------------------------------------ */
static void fo_conv_trunc(const double* h, int32_t L, const double* x, int64_t N, double* y)
{
    for (int64_t n = 0; n < N; ++n) {
        double acc = 0.0;
        const int64_t kmax = n < (int64_t)L - 1 ? n : (int64_t)L - 1;
        for (int64_t k = 0; k <= kmax; ++k) acc += h[k] * x[n - k];
        y[n] = acc;
    }
}

int fo_spatialize(int32_t B, int32_t S, int32_t M, const int32_t* rir_len, const int64_t* rir_off,
                  const double* rir, const double* target_rir, int64_t N, const double* x, int32_t n_speech,
                  const double* level_db, double* mix, double* targets, double* gains)
{
    if (B < 0 || S < 1 || M < 1 || N < 0 || n_speech < 1 || n_speech > S) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int32_t b = 0; b < B; ++b) {
        const int32_t L = rir_len[b];
        double* y = (double*)malloc(sizeof(double) * (size_t)(S * (int64_t)M * N + N + 1));
        double* E = (double*)malloc(sizeof(double) * (size_t)S);
        if (!y || !E) { err = 1; free(y); free(E); continue; }
        double* v = y + (int64_t)S * M * N;
        for (int32_t s = 0; s < S; ++s)
            for (int32_t m = 0; m < M; ++m)
                fo_conv_trunc(rir + rir_off[b] + ((int64_t)s * M + m) * L, L, x + ((int64_t)b * S + s) * N, N,
                              y + ((int64_t)s * M + m) * N);
        for (int32_t s = 0; s < S; ++s) {
            double e = 0.0;
            const double* y0 = y + (int64_t)s * M * N;
            for (int64_t n = 0; n < N; ++n) e += y0[n] * y0[n];
            E[s] = e;
        }
        double* g = gains + (int64_t)b * S;
        g[0] = 1.0;
        for (int32_t s = 1; s < n_speech; ++s)
            g[s] = E[s] > 0.0 ? sqrt(E[0] / E[s] * pow(10.0, -level_db[(int64_t)b * S + s] / 10.0)) : 0.0;
        double Ev = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double acc = 0.0;
            for (int32_t s = 0; s < n_speech; ++s) acc += g[s] * y[(int64_t)s * M * N + n];
            v[n] = acc;
            Ev += acc * acc;
        }
        for (int32_t s = n_speech; s < S; ++s)
            g[s] = E[s] > 0.0 ? sqrt(Ev / E[s] * pow(10.0, -level_db[(int64_t)b * S + s] / 10.0)) : 0.0;
        for (int32_t m = 0; m < M; ++m) {
            double* out = mix + ((int64_t)b * M + m) * N;
            for (int64_t n = 0; n < N; ++n) {
                double acc = 0.0;
                for (int32_t s = 0; s < S; ++s) acc += g[s] * y[((int64_t)s * M + m) * N + n];
                out[n] = acc;
            }
        }
        if (targets) {
            for (int32_t s = 0; s < n_speech; ++s)
                for (int32_t m = 0; m < M; ++m) {
                    double* t = targets + (((int64_t)b * n_speech + s) * M + m) * N;
                    fo_conv_trunc(target_rir + rir_off[b] + ((int64_t)s * M + m) * L, L,
                                  x + ((int64_t)b * S + s) * N, N, t);
                    for (int64_t n = 0; n < N; ++n) t[n] *= g[s];
                }
        }
        free(y);
        free(E);
    }
    return err ? -2 : 0;
}

int fo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void fo_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
