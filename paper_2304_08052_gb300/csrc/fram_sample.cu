// fram_sample.cu -- virtual-image sampler kernel (FRAM-RIR Sec. III-A to III-C, Eq. 2-6).
//
// One CTA per (room, source).  Thread 0 evaluates the per-(room, source) constants in FP64
// (a few dozen double operations per CTA); every thread then draws images i = tid, tid +
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
    float alpha, a, bma, tau;
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

__global__ void __launch_bounds__(256) sample_kernel(LaunchArgs a, double alpha, double beta, double pa, double pb,
                                                     double tau, double c0, uint64_t seed, const uint64_t* d_seed,
                                                     float* __restrict__ pos_hi, float* __restrict__ pos_lo,
                                                     float* __restrict__ g_out, float* __restrict__ r_out,
                                                     uint32_t* __restrict__ words)
{
    const int bs = blockIdx.x;
    const int b = bs / a.S, s = bs % a.S;
    __shared__ SampleConst C;
    __shared__ uint32_t key_s[2];
    if (threadIdx.x == 0) {
        const uint64_t sd = d_seed ? *d_seed : seed;
        key_s[0] = (uint32_t)(sd & 0xffffffffu);
        key_s[1] = (uint32_t)(sd >> 32);
        // Sec. III-A: R = V/S of the empty shoebox; Eq. 2: Eyring coefficient.
        const double lx = a.dims[3 * b], ly = a.dims[3 * b + 1], lz = a.dims[3 * b + 2];
        const double t60 = a.rt60[b];
        const double V = lx * ly * lz;
        const double Sarea = 2.0 * (lx * ly + lx * lz + ly * lz);
        const double R = V / Sarea;
        const double e = 1.0 - exp(-0.16 * R / t60);
        const double r = sqrt(1.0 - e * e);
        if (s == 0 && r_out) r_out[b] = (float)r;
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
        C.valid = ok ? 1 : 0;
        if (!ok) atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
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
        const u4 w = philox4x32_10(u4{(uint32_t)i, (uint32_t)s, (uint32_t)b, 0u}, k0, k1);
        if (words) {
            reinterpret_cast<uint4*>(words)[v] = make_uint4(w.x, w.y, w.z, w.w);
        }
        if (!C.valid) {
            for (int k = 0; k < 3; ++k) { pos_hi[3 * v + k] = nanf_; if (pos_lo) pos_lo[3 * v + k] = nanf_; }
            g_out[v] = nanf_;
            continue;
        }
        const float u0 = uniform_from_word(w.x), u1 = uniform_from_word(w.y);
        const float u2 = uniform_from_word(w.z), u3 = uniform_from_word(w.w);
        // Eq. 3 inverse CDF: x = cbrt(alpha^3 + u0 (beta^3 - alpha^3)).
        f2 vv = f2_add(C.a3, f2_mul_f(C.w3, u0));
        f2 x = f2_cbrt(vv);
        // Eq. 4 and D_i = D0 * DR_i:  D_i = D0 + c2 (x - alpha).
        f2 D = f2_add(C.d0, f2_mul(C.c2, f2_add(x, f2_neg(C.alpha2))));
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
        f2 p0 = f2_add(C.cx, f2_mul_f(Dinv, d0));
        f2 p1 = f2_add(C.cy, f2_mul_f(Dinv, d1));
        f2 p2 = f2_add(C.cz, f2_mul_f(Dinv, d2));
        pos_hi[3 * v + 0] = p0.hi; pos_hi[3 * v + 1] = p1.hi; pos_hi[3 * v + 2] = p2.hi;
        if (pos_lo) { pos_lo[3 * v + 0] = p0.lo; pos_lo[3 * v + 1] = p1.lo; pos_lo[3 * v + 2] = p2.lo; }
        // Eq. 6: g = clamp(1 + (D/(c0 T60))^2 (RR_max - 1) + p DR^tau, 1, RR_max).
        f2 ratio = f2_mul(D, C.inv_ct);
        f2 trend = f2_add_f(f2_mul(f2_mul(ratio, ratio), C.rrm1), 1.0f);
        const float DR = __fadd_rn(f2_mul(D, C.inv_d0).hi, 0.0f);
        const float pert = __fmul_rn(__fmaf_rn(C.bma, u3, C.a), exp2f(C.tau * log2f(DR)));
        f2 g = f2_add_f(trend, pert);
        float gf = __fadd_rn(g.hi, g.lo);
        // Clamp in pair precision against RR_max and 1.
        const bool above = (g.hi > C.rr.hi) || (g.hi == C.rr.hi && g.lo > C.rr.lo);
        if (above) gf = __fadd_rn(C.rr.hi, C.rr.lo);
        if (g.hi < 1.0f || (g.hi == 1.0f && g.lo < 0.0f)) gf = 1.0f;
        g_out[v] = gf;
    }
}

}  // namespace

cudaError_t launch_sample(const LaunchArgs& a, const fram_params& p, uint64_t seed, const uint64_t* d_seed,
                          float* pos_hi, float* pos_lo, float* g, float* r, uint32_t* words, cudaStream_t st)
{
    const int nblocks = a.B * a.S;
    if (nblocks == 0) return cudaSuccess;
    sample_kernel<<<nblocks, 256, 0, st>>>(a, p.alpha, p.beta, p.a, p.b, p.tau, p.c0, seed, d_seed, pos_hi, pos_lo,
                                          g, r, words);
    return cudaGetLastError();
}

}  // namespace fram
