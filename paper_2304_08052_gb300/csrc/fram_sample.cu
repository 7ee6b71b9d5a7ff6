// fram_sample.cu -- virtual-image sampler kernel (FRAM-RIR Sec. III-A to III-C, Eq. 2-6) and
// the gradient through it (sample_backward_kernel, sample_backward_room).
//
// sample_prologue evaluates the per-(room, source) constants in FP64 (one thread each, a few
// dozen double operations) into the workspace; then one CTA per (room, source) draws images
// i = tid, tid +
// blockDim, ... with one Philox4x32-10 call each and maps the four words to
//   u0 -> distance ratio x (inverse CDF of Eq. 3) -> D_i = D0 + (c0 T60 - D0)(x - alpha)/(beta - alpha)
//         (Eq. 4 written as a single affine map: x = alpha gives D0, x = beta gives c0 T60),
//   u1, u2 -> azimuth 2 pi u1 and elevation pi (u2 - 1/2) (Sec. III-B),
//   u3 -> perturbation a + (b - a) u3 of the reflection count (Eq. 6).
// The distance chain and the final position are carried as float pairs so that each image's
// distance to the array centre is exact to ~1e-13 relative; the direction is computed in FP32
// and renormalised in float-pair arithmetic, so its error only tilts the image (a ~1e-7 rad
// tilt moves per-mic delays by |mic - c| * 1e-7, below 1e-8 m).
#include <cmath>

#include "fram_internal.cuh"

namespace fram {
namespace {

struct SampleConst {
    f2 d0, c2, alpha2, a3, w3;  // D0, (c0T60 - D0)/(beta - alpha), alpha, alpha^3, beta^3 - alpha^3
    f2 inv_ct, rr, rrm1, inv_d0;
    f2 cx, cy, cz;              // array centre
    float alpha, a, bma, tau, inv_bma;
    int valid;
};

// cbrt of a positive pair: one Newton step from the float cube root.
__device__ __forceinline__ f2 f2_cbrt(f2 v)
{
    float x0 = cbrtf(v.hi);
    f2 sq = two_prod(x0, x0);
    f2 cu = two_prod(x0, sq.hi);
    cu.lo = __fmaf_rn(x0, sq.lo, cu.lo);
    float res = __fadd_rn(__fsub_rn(v.hi, cu.hi), __fsub_rn(v.lo, cu.lo));
    float dx = __fdiv_rn(res, __fmul_rn(3.0f, sq.hi));
    return fast_two_sum(x0, dx);
}

// One image from its Philox words: position (float pairs), reflection count, and what the
// gradient through the sampler needs (shared by the sampler and its adjoint, so both take the
// same clamp decision).
struct SampledImage {
    f2 p0, p1, p2;          // position
    float gf;               // g after the clamp
    int clamp;              // 0: inside [1, RR_max]; 1: held at RR_max; -1: held at 1
    float nx, ny, nz;       // unit direction of the image from the array centre
    float k;                // (x - alpha) / (beta - alpha)
    float D, DR, pert;      // D_i, D_i / D0, a + (b - a) u3
    float DRt;              // DR^tau
};

__device__ __forceinline__ SampledImage sample_image(const SampleConst& C, u4 w)
{
    SampledImage im;
    const float u0 = uniform_from_word(w.x), u1 = uniform_from_word(w.y);
    const float u2 = uniform_from_word(w.z), u3 = uniform_from_word(w.w);
    // Eq. 3 inverse CDF: x = cbrt(alpha^3 + u0 (beta^3 - alpha^3)).
    f2 vv = f2_add(C.a3, f2_mul_f(C.w3, u0));
    f2 x = f2_cbrt(vv);
    // Eq. 4 and D_i = D0 * DR_i:  D_i = D0 + c2 (x - alpha).
    f2 xa = f2_add(x, f2_neg(C.alpha2));
    f2 D = f2_add(C.d0, f2_mul(C.c2, xa));
    // Sec. III-B: direction from azimuth theta = 2 pi u1 and elevation phi = pi (u2 - 1/2).
    float st, ct, sp, cp;
    sincospif(2.0f * u1, &st, &ct);
    sincospif(u2 - 0.5f, &sp, &cp);
    const float d0 = cp * ct, d1 = cp * st, d2 = sp;
    // Renormalise the float direction in pair arithmetic: |dir| = 1 to ~1e-13.
    f2 nn = f2_add(f2_add(two_prod(d0, d0), two_prod(d1, d1)), two_prod(d2, d2));
    float y0 = rsqrtf(nn.hi);
    // Newton step for 1/sqrt: y = y0 + y0 (1 - nn y0^2) / 2, residual in pair arithmetic.
    f2 y02 = two_prod(y0, y0);
    f2 t = f2_mul(nn, y02);
    float res = __fadd_rn(__fsub_rn(1.0f, t.hi), -t.lo);
    f2 inv = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), res));
    f2 Dinv = f2_mul(D, inv);
    im.p0 = f2_add(C.cx, f2_mul_f(Dinv, d0));
    im.p1 = f2_add(C.cy, f2_mul_f(Dinv, d1));
    im.p2 = f2_add(C.cz, f2_mul_f(Dinv, d2));
    // Eq. 6: g = clamp(1 + (D/(c0 T60))^2 (RR_max - 1) + p DR^tau, 1, RR_max).
    f2 ratio = f2_mul(D, C.inv_ct);
    f2 trend = f2_add_f(f2_mul(f2_mul(ratio, ratio), C.rrm1), 1.0f);
    const float DR = __fadd_rn(f2_mul(D, C.inv_d0).hi, 0.0f);
    const float pp = __fmaf_rn(C.bma, u3, C.a);
    const float DRt = exp2f(C.tau * log2f(DR));
    const float pert = __fmul_rn(pp, DRt);
    f2 g = f2_add_f(trend, pert);
    float gf = __fadd_rn(g.hi, g.lo);
    // Clamp in pair precision against RR_max and 1.
    im.clamp = 0;
    const bool above = (g.hi > C.rr.hi) || (g.hi == C.rr.hi && g.lo > C.rr.lo);
    if (above) { gf = __fadd_rn(C.rr.hi, C.rr.lo); im.clamp = 1; }
    if (g.hi < 1.0f || (g.hi == 1.0f && g.lo < 0.0f)) { gf = 1.0f; im.clamp = -1; }
    im.gf = gf;
    const float ivf = inv.hi + inv.lo;
    im.nx = d0 * ivf; im.ny = d1 * ivf; im.nz = d2 * ivf;
    im.k = (xa.hi + xa.lo) * C.inv_bma;
    im.D = D.hi + D.lo;
    im.DR = DR;
    im.pert = pp;
    im.DRt = DRt;
    return im;
}

// Per-(room, source) constants in FP64 (thread 0), shared by the sampler and its adjoint.
__device__ void sample_consts(const LaunchArgs& a, int b, int s, double alpha, double beta, double pa, double pb,
                              double tau, double c0, SampleConst& C, double* r_out_d, double* extra)
{
    // Sec. III-A: R = V/S of the empty shoebox; Eq. 2: Eyring coefficient.
    const double lx = a.dims[3 * b], ly = a.dims[3 * b + 1], lz = a.dims[3 * b + 2];
    const double t60 = a.rt60[b];
    const double V = lx * ly * lz;
    const double Sarea = 2.0 * (lx * ly + lx * lz + ly * lz);
    const double R = V / Sarea;
    const double e = 1.0 - exp(-0.16 * R / t60);
    const double r = sqrt(1.0 - e * e);
    if (r_out_d) *r_out_d = r;
    double cx = 0, cy = 0, cz = 0;
    for (int m = 0; m < a.M; ++m) {
        const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
        cx += pm[0]; cy += pm[1]; cz += pm[2];
    }
    cx /= a.M; cy /= a.M; cz /= a.M;
    const float* ps = a.src + 3 * ((size_t)b * a.S + s);
    const double dx = ps[0] - cx, dy = ps[1] - cy, dz = ps[2] - cz;
    const double D0 = sqrt(dx * dx + dy * dy + dz * dz);
    const double cT = c0 * t60;
    const bool ok = (lx > 0) && (ly > 0) && (lz > 0) && (t60 > 0) && (D0 > 0) && (cT > D0) && (r > 0) && (r < 1);
    // Eq. 5.
    const double RR = (log10(cT) - log10(D0) - 3.0) / log10(r);
    C.d0 = f2_from_double(D0);
    C.c2 = f2_from_double((cT - D0) / (beta - alpha));
    C.alpha2 = f2_from_double(alpha);
    C.a3 = f2_from_double(alpha * alpha * alpha);
    C.w3 = f2_from_double(beta * beta * beta - alpha * alpha * alpha);
    C.inv_ct = f2_from_double(1.0 / cT);
    C.rr = f2_from_double(RR);
    C.rrm1 = f2_from_double(RR - 1.0);
    C.inv_d0 = f2_from_double(1.0 / D0);
    C.cx = f2_from_double(cx);
    C.cy = f2_from_double(cy);
    C.cz = f2_from_double(cz);
    C.alpha = (float)alpha;
    C.a = (float)pa;
    C.bma = (float)(pb - pa);
    C.tau = (float)tau;
    C.inv_bma = (float)(1.0 / (beta - alpha));
    C.valid = ok ? 1 : 0;
    if (extra) {    // D0, c0 T60, RR_max, r, unit (src - c) / D0, R, exp(-0.16 R / T60), e
        extra[0] = D0; extra[1] = cT; extra[2] = RR; extra[3] = r;
        extra[4] = dx / D0; extra[5] = dy / D0; extra[6] = dz / D0;
        extra[7] = R; extra[8] = 1.0 - e; extra[9] = e;
    }
}

// Record of (room, source) bs in the workspace: SampleConst, then the 10 doubles of `extra`.
static_assert(sizeof(SampleConst) <= 128 && sizeof(SampleConst) % 4 == 0, "sampler record layout");
static_assert(128 + 10 * sizeof(double) <= kSampleRec, "sampler record size");

// The per-(room, source) constants, one thread each, so the image kernels need not wait on a
// serial FP64 prologue per CTA.
__global__ void __launch_bounds__(128) sample_prologue(LaunchArgs a, double alpha, double beta, double pa, double pb,
                                                       double tau, double c0, float* __restrict__ r_out)
{
    const int bs = blockIdx.x * blockDim.x + threadIdx.x;
    if (bs >= a.B * a.S) return;
    const int b = bs / a.S, s = bs % a.S;
    SampleConst C;
    double X[10];
    double r;
    sample_consts(a, b, s, alpha, beta, pa, pb, tau, c0, C, &r, X);
    if (s == 0 && r_out) r_out[b] = (float)r;
    if (!C.valid) atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
    char* rec = a.sconst + (int64_t)bs * kSampleRec;
    *reinterpret_cast<SampleConst*>(rec) = C;
    double* xr = reinterpret_cast<double*>(rec + 128);
    for (int k = 0; k < 10; ++k) xr[k] = X[k];
}

// Copies record bs into shared memory (C and, if X is given, the extras); the caller syncs.
__device__ __forceinline__ void load_record(const LaunchArgs& a, int bs, SampleConst* C, double* X)
{
    const int* src = reinterpret_cast<const int*>(a.sconst + (int64_t)bs * kSampleRec);
    constexpr int nc = (int)(sizeof(SampleConst) / 4);
    if (threadIdx.x < nc) reinterpret_cast<int*>(C)[threadIdx.x] = src[threadIdx.x];
    if (X && threadIdx.x >= 32 && threadIdx.x < 52) reinterpret_cast<int*>(X)[threadIdx.x - 32] = src[32 + threadIdx.x - 32];
}

__global__ void __launch_bounds__(256) sample_kernel(LaunchArgs a, uint64_t seed, const uint64_t* d_seed,
                                                     float* __restrict__ pos_hi, float* __restrict__ pos_lo,
                                                     float* __restrict__ g_out, uint32_t* __restrict__ words)
{
    const int bs = blockIdx.x;
    const int b = bs / a.S, s = bs % a.S;
    __shared__ SampleConst C;
    __shared__ uint32_t key_s[2];
    load_record(a, bs, &C, nullptr);
    if (threadIdx.x == 0) {
        const uint64_t sd = d_seed ? *d_seed : seed;
        key_s[0] = (uint32_t)(sd & 0xffffffffu);
        key_s[1] = (uint32_t)(sd >> 32);
    }
    __syncthreads();
    int n = a.n_vs[b];
    const int64_t row0 = a.vs_off[b] + (int64_t)s * n;
    if (n < 0 || row0 < 0 || row0 + n > a.n_vs_total) {   // offsets disagree with the host sizes
        if (threadIdx.x == 0) atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
        n = 0;
    }
    const uint32_t k0 = key_s[0], k1 = key_s[1];
    const float nanf_ = __int_as_float(0x7fc00000);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t v = row0 + i;
        const u4 w = philox4x32_10(u4{(uint32_t)i, (uint32_t)s, a.room_base + (uint32_t)b, 0u}, k0, k1);
        if (words) {
            reinterpret_cast<uint4*>(words)[v] = make_uint4(w.x, w.y, w.z, w.w);
        }
        if (!C.valid) {
            for (int k = 0; k < 3; ++k) { pos_hi[3 * v + k] = nanf_; if (pos_lo) pos_lo[3 * v + k] = nanf_; }
            g_out[v] = nanf_;
            continue;
        }
        const SampledImage im = sample_image(C, w);
        pos_hi[3 * v + 0] = im.p0.hi; pos_hi[3 * v + 1] = im.p1.hi; pos_hi[3 * v + 2] = im.p2.hi;
        if (pos_lo) { pos_lo[3 * v + 0] = im.p0.lo; pos_lo[3 * v + 1] = im.p1.lo; pos_lo[3 * v + 2] = im.p2.lo; }
        const float gf = im.gf;
        g_out[v] = gf;
    }
}

// ---- Gradient through the sampler (reparameterised: every image's draws held fixed) ----------
// An image is p_i = c + D_i nu_i with D_i = D0 (1 - k_i) + k_i c0 T60 and g_i from Eq. 6 (zero
// derivative where the clamp holds it at 1, derivative 1 in RR_max where it holds it at RR_max).
// Per (room, source): sums over images of dL/dD0, dL/d(c0 T60), dL/dRR_max and dL/dc, then Eq. 5
// (RR_max from c0 T60, D0 and r) and D0 = |src - c|.  Per room: Eq. 2 (r from T60 and R = V/S)
// and c = the mean of the mics.  Sums run in a fixed order (deterministic).
__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

constexpr int kSbParts = 5;     // per (room, source): dL/dc (3), dL/d(c0 T60), dL/dr via RR_max

__global__ void __launch_bounds__(256) sample_backward_kernel(LaunchArgs a, uint64_t seed, const uint64_t* d_seed,
                                                              const float* __restrict__ grad_vs,
                                                              const float* __restrict__ grad_g,
                                                              const float* __restrict__ grad_src_dir,
                                                              float* __restrict__ grad_src, double* __restrict__ part)
{
    const int bs = blockIdx.x;
    const int b = bs / a.S, s = bs % a.S;
    __shared__ SampleConst C;
    __shared__ double X[10];
    __shared__ uint32_t key_s[2];
    __shared__ double red[8][6];
    load_record(a, bs, &C, X);
    if (threadIdx.x == 0) {
        const uint64_t sd = d_seed ? *d_seed : seed;
        key_s[0] = (uint32_t)(sd & 0xffffffffu);
        key_s[1] = (uint32_t)(sd >> 32);
    }
    __syncthreads();
    int n = a.n_vs[b];
    const int64_t row0 = a.vs_off[b] + (int64_t)s * n;
    if (n < 0 || row0 < 0 || row0 + n > a.n_vs_total || !C.valid) n = 0;
    const float D0 = (float)X[0], cT = (float)X[1], RR = (float)X[2];
    const float inv_cT2 = 1.0f / (cT * cT), rrm1 = RR - 1.0f;
    // Per-thread sums in FP32 over the thread's images (a few dozen), then FP64 across threads.
    float dD0 = 0.f, dcT = 0.f, dRR = 0.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t v = row0 + i;
        const u4 w = philox4x32_10(u4{(uint32_t)i, (uint32_t)s, a.room_base + (uint32_t)b, 0u}, key_s[0], key_s[1]);
        const SampledImage im = sample_image(C, w);
        const float gx = grad_vs[3 * v], gy = grad_vs[3 * v + 1], gz = grad_vs[3 * v + 2];
        const float gg = grad_g ? grad_g[v] : 0.0f;
        float dDi = gx * im.nx + gy * im.ny + gz * im.nz;          // p_i = c + D_i nu_i
        dc0 += gx; dc1 += gy; dc2 += gz;
        float dD0g = 0.0f, dcTg = 0.0f;
        if (im.clamp == 1) {
            dRR += gg;
        } else if (im.clamp == 0) {                                // Eq. 6 inside the clamp
            const float drt = C.tau * im.DRt / im.DR;                  // d(DR^tau)/dDR
            dDi += gg * (2.0f * im.D * inv_cT2 * rrm1 + im.pert * drt / D0);
            dD0g = gg * (-im.pert * drt * im.D / (D0 * D0));
            dcTg = gg * (-2.0f * im.D * im.D * inv_cT2 / cT * rrm1);
            dRR += gg * (im.D * im.D * inv_cT2);
        }
        dD0 += dDi * (1.0f - im.k) + dD0g;                        // Eq. 4 as D_i = D0 (1-k) + k c0 T60
        dcT += dDi * im.k + dcTg;
    }
    double v6[6] = {(double)dD0, (double)dcT, (double)dRR, (double)dc0, (double)dc1, (double)dc2};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) v6[k] = warp_sum_d(v6[k]);
    if (lane == 0)
        for (int k = 0; k < 6; ++k) red[wid][k] = v6[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8)
            for (int k = 0; k < 6; ++k) t[k] += red[w8][k];
        const double r = X[3], lnr = log(r);
        const double D0d = X[0], cTd = X[1], RRd = X[2];
        double gD0 = t[0] + t[2] * (-1.0 / (D0d * lnr));          // Eq. 5
        const double gcT = t[1] + t[2] * (1.0 / (cTd * lnr));
        const double gr = t[2] * (-RRd / (r * lnr));
        if (!C.valid) gD0 = 0.0;
        double* pp = part + (int64_t)bs * kSbParts;
        for (int j = 0; j < 3; ++j) {                               // D0 = |src - c|
            const double u = X[4 + j];
            if (grad_src) {
                const double dir = grad_src_dir ? (double)grad_src_dir[3 * (int64_t)bs + j] : 0.0;
                grad_src[3 * (int64_t)bs + j] = (float)(dir + (C.valid ? gD0 * u : 0.0));
            }
            pp[j] = C.valid ? t[3 + j] - gD0 * u : 0.0;
        }
        pp[3] = C.valid ? gcT : 0.0;
        pp[4] = C.valid ? gr : 0.0;
    }
}

__global__ void sample_backward_room(LaunchArgs a, double c0, const float* __restrict__ grad_r_amp,
                                     const float* __restrict__ grad_mic_dir, const double* __restrict__ part,
                                     float* __restrict__ grad_mic, float* __restrict__ grad_t60,
                                     float* __restrict__ grad_dims)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    double dc[3] = {0, 0, 0}, dcT = 0.0, dr = grad_r_amp ? (double)grad_r_amp[b] : 0.0;
    for (int s = 0; s < a.S; ++s) {
        const double* pp = part + ((int64_t)b * a.S + s) * kSbParts;
        dc[0] += pp[0]; dc[1] += pp[1]; dc[2] += pp[2];
        dcT += pp[3];
        dr += pp[4];
    }
    if (grad_mic)
        for (int m = 0; m < a.M; ++m)
            for (int j = 0; j < 3; ++j) {
                const int64_t o = 3 * ((int64_t)b * a.M + m) + j;
                grad_mic[o] = (float)((grad_mic_dir ? (double)grad_mic_dir[o] : 0.0) + dc[j] / a.M);
            }
    // Eq. 2: r = sqrt(1 - e^2), e = 1 - exp(-0.16 R / T60), R = V / S.
    const double lx = a.dims[3 * b], ly = a.dims[3 * b + 1], lz = a.dims[3 * b + 2];
    const double t60 = a.rt60[b];
    const double V = lx * ly * lz, Sa = 2.0 * (lx * ly + lx * lz + ly * lz), R = V / Sa;
    const double ex = exp(-0.16 * R / t60), e = 1.0 - ex, r = sqrt(1.0 - e * e);
    const double dLde = dr != 0.0 ? dr * (-e / r) : 0.0;    // r = 0 (no reverberation tail): no r path
    if (grad_t60) grad_t60[b] = (float)(dcT * c0 + dLde * (-ex * 0.16 * R / (t60 * t60)));
    if (grad_dims) {
        const double dLdR = dLde * (ex * 0.16 / t60);
        const double dV[3] = {ly * lz, lx * lz, lx * ly};
        const double dS[3] = {2.0 * (ly + lz), 2.0 * (lx + lz), 2.0 * (lx + ly)};
        for (int j = 0; j < 3; ++j) grad_dims[3 * b + j] = (float)(dLdR * (dV[j] / Sa - V * dS[j] / (Sa * Sa)));
    }
}

}  // namespace

cudaError_t launch_sample(const LaunchArgs& a, const fram_params& p, uint64_t seed, const uint64_t* d_seed,
                          float* pos_hi, float* pos_lo, float* g, float* r, uint32_t* words, cudaStream_t st)
{
    const int nblocks = a.B * a.S;
    if (nblocks == 0) return cudaSuccess;
    sample_prologue<<<(nblocks + 127) / 128, 128, 0, st>>>(a, p.alpha, p.beta, p.a, p.b, p.tau, p.c0, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sample_kernel<<<nblocks, 256, 0, st>>>(a, seed, d_seed, pos_hi, pos_lo, g, words);
    return cudaGetLastError();
}

}  // namespace fram

namespace fram {

cudaError_t launch_sample_backward(const LaunchArgs& a, const fram_params& p, uint64_t seed, const uint64_t* d_seed,
                                   const float* grad_vs, const float* grad_g, const float* grad_r,
                                   const float* grad_src_dir, const float* grad_mic_dir, float* grad_src,
                                   float* grad_mic, float* grad_t60, float* grad_dims, double* part, cudaStream_t st)
{
    const int nblocks = a.B * a.S;
    if (nblocks == 0) return cudaSuccess;
    sample_prologue<<<(nblocks + 127) / 128, 128, 0, st>>>(a, p.alpha, p.beta, p.a, p.b, p.tau, p.c0, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sample_backward_kernel<<<nblocks, 256, 0, st>>>(a, seed, d_seed, grad_vs, grad_g, grad_src_dir, grad_src, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sample_backward_room<<<(a.B + 127) / 128, 128, 0, st>>>(a, p.c0, grad_r, grad_mic_dir, part, grad_mic, grad_t60,
                                                            grad_dims);
    return cudaGetLastError();
}

}  // namespace fram
