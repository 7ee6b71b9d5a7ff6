// fram_backward.cu -- adjoint of the windowed-sinc synthesis (gradients of a loss on the RIR
// with respect to source, mic and image positions and the reflection coefficient).
//
// Ownership instead of scattering: every image belongs to exactly one (room, source, tile)
// work item -- the tile its binning key (delay to the array centre) falls in -- and the
// direct path of a (room, source) belongs to the tile of the source's key.  A persistent CTA
// takes an item, and for each mic stages the upstream gradient
//   G[n] = dL/dh[n] + [n in Eq. 9 window] dL/dh_e[n]
// over the tile plus a halo of 2K + margin samples in shared memory; each thread then owns one
// image, recomputes its arrival (float-pair delay, amplitude) and gathers its 2K+1 taps:
//   dL/dA = sum_k G[n_c + k] s(x) w(x),   dL/dt = -A sum_k G[n_c + k] (s'(x) w(x) + s(x) w'(x)),
// with x = k - delta, s = sinc, s'(x) = (cos(pi x) - s(x)) / x (a Taylor series on the centre
// tap, where the difference cancels), w = (1 + cos(pi x/K))/2, w' = -(pi/2K) sin(pi x/K).
// The chain rule gives dL/dD = dL/dt fs/c0 - dL/dA A/D and dD/dp = (p - mic)/D.
// Image gradients are summed over mics in mic order inside the owning thread; mic, source and
// r gradients are reduced per item in a fixed tree and then per room in item order, so the
// result does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <utility>

#include "fram_internal.cuh"

namespace fram {
namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.31830988618379067f;
constexpr float kTinyDelta = 9.313225746154785e-10f;

// d/dx sinc(x) for |x| <= 1/2: odd Taylor series sum_j (-1)^j 2j pi^(2j) x^(2j-1) / (2j+1)!.
__device__ __forceinline__ float dsinc_small(float x)
{
    const float x2 = x * x;
    // Coefficients of x^1, x^3, ..., x^11.
    const float c1 = -3.2898681336964524f;     // -pi^2/3
    const float c2 = 3.2469697011334144f;      //  pi^4/30
    const float c3 = -1.1445173762772416f;     // -pi^6/840
    const float c4 = 0.20918381538538052f;     //  pi^8/45360
    const float c5 = -0.023460744224286495f;   // -pi^10/3991680
    const float c6 = 0.0017807474713398848f;   //  pi^12/518918400
    float p = __fmaf_rn(c6, x2, c5);
    p = __fmaf_rn(p, x2, c4);
    p = __fmaf_rn(p, x2, c3);
    p = __fmaf_rn(p, x2, c2);
    p = __fmaf_rn(p, x2, c1);
    return p * x;
}

// cos and sin(pi k / K) for k = -K..K, evaluated at compile time (Taylor series in double on
// [-pi, pi]) and written into the unrolled tap loop as literal FMA operands.
__host__ __device__ constexpr double cx_term(double x, int n)
{
    double t = 1.0;
    for (int i = 1; i <= n; ++i) t *= x / i;
    return t;
}

__host__ __device__ constexpr double cx_sin(double x)
{
    double acc = 0.0;
    for (int j = 0; j < 30; ++j) acc += ((j & 1) ? -1.0 : 1.0) * cx_term(x, 2 * j + 1);
    return acc;
}

__host__ __device__ constexpr double cx_cos(double x)
{
    double acc = 0.0;
    for (int j = 0; j < 30; ++j) acc += ((j & 1) ? -1.0 : 1.0) * cx_term(x, 2 * j);
    return acc;
}

struct TrigTab {
    float c[2 * kMaxHalfLen + 1];
    float s[2 * kMaxHalfLen + 1];
};

template <int K>
constexpr TrigTab make_trig_tab()
{
    TrigTab t{};
    for (int i = 0; i <= 2 * K; ++i) {
        const double x = 3.14159265358979323846 * (double)(i - K) / (double)K;
        t.c[i] = (float)cx_cos(x);
        t.s[i] = (float)cx_sin(x);
    }
    return t;
}

__constant__ TrigTab c_trig40 = make_trig_tab<40>();
__constant__ TrigTab c_trig63 = make_trig_tab<63>();

// Taps of one arrival against staged G (Gs points at G[n_c - K]): gA = sum G tap, gT = sum G tap'
// with tap(x) = sinc(x) (1 + cos(pi x/K))/2, x = k - delta.  With W2 = 1 + cos(pi x/K):
//   2 tap = s W2,   2 tap' = s' W2 - (pi/K) s sin(pi x/K),
//   s = -(-1)^k sin(pi delta)/(pi x),  s' = ((-1)^k cos(pi delta) - s)/x.
// The loop is fully unrolled and the constant tables are named directly, so their entries are
// read as constant-bank operands of the FMAs.
template <int KT>
__device__ __forceinline__ void gather_taps_ct(const float* __restrict__ Gs, float delta, float& gA, float& gT)
{
    const float sd = sinpi_poly(delta), cd = cospi_poly(delta);
    const float y = delta * (1.0f / (float)KT);
    const float sk = sinpi_poly(y), ck = cospi_poly(y);
    const float spi = sd * kInvPi;                     // sin(pi delta) / pi
    const float spic = spi * (-kPi / (float)KT);       // -(pi/K) sin(pi delta) / pi
    float a = 0.f, t = 0.f;
#pragma unroll
    for (int kk = 0; kk <= 2 * KT; ++kk) {
        const int k = kk - KT;
        const float Ck = (KT == 40) ? c_trig40.c[kk] : c_trig63.c[kk];
        const float Sk = (KT == 40) ? c_trig40.s[kk] : c_trig63.s[kk];
        const float G = Gs[kk];
        const float x = __fsub_rn((float)k, delta);
        const float r = rcp_approx(x);
        const bool even = (k & 1) == 0;
        const float s = (even ? -spi : spi) * r;
        const float sc = (even ? -spic : spic) * r;
        const float sp = (k == 0) ? dsinc_small(x) : ((even ? cd : -cd) - s) * r;
        const float W2 = __fmaf_rn(Ck, ck, __fmaf_rn(Sk, sk, 1.0f));
        const float sw = __fmaf_rn(Sk, ck, -(Ck * sk));
        float tap2 = s * W2;
        float dtap2 = __fmaf_rn(sp, W2, sc * sw);
        if ((kk == 0 || kk == 2 * KT) && !(fabsf(x) < (float)KT)) { tap2 = 0.f; dtap2 = 0.f; }
        a = __fmaf_rn(G, tap2, a);
        t = __fmaf_rn(G, dtap2, t);
    }
    gA = 0.5f * a;
    gT = 0.5f * t;
}

// Any K: the same taps with the trigonometric table in shared memory.
__device__ __forceinline__ void gather_taps_rt(const float* __restrict__ Gs, int K, float delta, const float2* tab,
                                               float& gA, float& gT)
{
    const float sd = sinpi_poly(delta), cd = cospi_poly(delta);
    const float y = delta / (float)K;
    const float sk = sinpi_poly(y), ck = cospi_poly(y);
    const float spi = sd * kInvPi;
    const float spic = spi * (-kPi / (float)K);
    float a = 0.f, t = 0.f;
    for (int kk = 0; kk <= 2 * K; ++kk) {
        const int k = kk - K;
        const float G = Gs[kk];
        const float x = __fsub_rn((float)k, delta);
        const float r = rcp_approx(x);
        const bool even = (k & 1) == 0;
        const float s = (even ? -spi : spi) * r;
        const float sc = (even ? -spic : spic) * r;
        const float sp = (k == 0) ? dsinc_small(x) : ((even ? cd : -cd) - s) * r;
        const float2 cs = tab[kk];
        const float W2 = __fmaf_rn(cs.x, ck, __fmaf_rn(cs.y, sk, 1.0f));
        const float sw = __fmaf_rn(cs.y, ck, -(cs.x * sk));
        float tap2 = s * W2;
        float dtap2 = __fmaf_rn(sp, W2, sc * sw);
        if ((kk == 0 || kk == 2 * K) && !(fabsf(x) < (float)K)) { tap2 = 0.f; dtap2 = 0.f; }
        a = __fmaf_rn(G, tap2, a);
        t = __fmaf_rn(G, dtap2, t);
    }
    gA = 0.5f * a;
    gT = 0.5f * t;
}

template <int KT>
__device__ __forceinline__ void gather_taps(const float* __restrict__ Gs, int K, float delta, const float2* tab,
                                            float& gA, float& gT)
{
    if constexpr (KT > 0) gather_taps_ct<KT>(Gs, delta, gA, gT);
    else gather_taps_rt(Gs, K, delta, tab, gA, gT);
}

struct BwdSmemPlan {
    int gs, tab, red, total, glen;
};

// Two staging buffers of the upstream gradient, the table for a run-time K, and the per-warp
// mic partials.
__host__ __device__ inline BwdSmemPlan bwd_smem(int T, int K, int margin_i, int M, int nwarps)
{
    BwdSmemPlan p;
    p.glen = T + 4 * K + 2 * margin_i + 8;
    p.gs = 0;
    p.tab = ((8 * p.glen) + 15) & ~15;
    p.red = p.tab + (((8 * (2 * K + 1)) + 15) & ~15);
    p.total = p.red + 4 * 3 * M * nwarps;
    return p;
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int NT, int KT>
__global__ void __launch_bounds__(NT, 4) bwd_kernel(LaunchArgs a, int margin_i, const float* __restrict__ pos_hi,
                                                     const float* __restrict__ pos_lo, const float* __restrict__ gref,
                                                     const float* __restrict__ grad_rir,
                                                     const float* __restrict__ grad_early, float* __restrict__ grad_vs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = NT / 32;
    const int T = a.tile, K = a.K, M = a.M;
    const BwdSmemPlan P = bwd_smem(T, K, margin_i, M, NW);
    float* Gs0 = reinterpret_cast<float*>(smem + P.gs);
    float2* tab = reinterpret_cast<float2*>(smem + P.tab);
    float* red = reinterpret_cast<float*>(smem + P.red);   // [NW][M][3]
    __shared__ int s_item;
    __shared__ float s_r[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (KT == 0)
        for (int j = tid; j <= 2 * K; j += NT) {
            float sn, cs;
            sincospif((float)(j - K) / (float)K, &sn, &cs);
            tab[j] = make_float2(cs, sn);
        }
    const int n_items = a.hdr->n_items;
    const float qf = a.q;
    __syncthreads();

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.hdr->queue_bwd, 1);
        __syncthreads();
        const int qi = s_item;
        if (qi >= n_items) break;
        const int2 it = a.items[qi];
        const int b = it.x, s = it.y >> 16, tau = it.y & 0xffff;
        const RoomConst rc = a.room[b];
        const int T0 = tau * T;
        const int Lb = rc.len;
        const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
        const int* bo = a.bin_off + ((int64_t)b * a.S + s) * (a.max_tiles + 1);
        const int o_lo = bo[tau], o_hi = bo[tau + 1];
        const int gbase = T0 - 2 * K - margin_i - 4;
        const bool own_direct = a.src_tile[(int64_t)b * a.S + s] == tau;
        const int64_t chan0 = rc.rir_off + (int64_t)s * M * Lb;
        for (int k = lane; k < 3 * M; k += 32) red[(wid * M) * 3 + k] = 0.f;
        __syncwarp();
        float pr = 0.f;                          // this thread's share of dL/dr
        float dsx = 0.f, dsy = 0.f, dsz = 0.f;   // direct-path source gradient (thread 0)
        const int nown = o_hi - o_lo;
        const int nch = nown > 0 ? (nown + NT - 1) / NT : 1;
        int iter = 0;
        for (int ch = 0; ch < nch; ++ch) {
            const int slot = ch * NT + tid;
            const bool has = slot < nown;
            int64_t v = 0;
            float phx = 0, phy = 0, phz = 0, plx = 0, ply = 0, plz = 0, gg = 0;
            if (has) {
                v = v0 + a.perm[v0 + o_lo + slot];
                phx = pos_hi[3 * v]; phy = pos_hi[3 * v + 1]; phz = pos_hi[3 * v + 2];
                if (pos_lo) { plx = pos_lo[3 * v]; ply = pos_lo[3 * v + 1]; plz = pos_lo[3 * v + 2]; }
                gg = gref[v];
            }
            const float A_g = has ? exp2f(gg * rc.log2r) : 0.f;   // r^g
            float gvx = 0.f, gvy = 0.f, gvz = 0.f;
            for (int m = 0; m < M; ++m, ++iter) {
                const DirectConst dc = a.direct[((int64_t)b * a.S + s) * M + m];
                const int64_t ch0 = chan0 + (int64_t)m * Lb;
                float* Gs = Gs0 + (iter & 1) * P.glen;
                for (int j = tid; j < P.glen; j += NT) {
                    const int n = gbase + j;
                    float Gv = 0.f;
                    if (n >= 0 && n < Lb) {
                        if (grad_rir) Gv = grad_rir[ch0 + n];
                        if (grad_early && n >= dc.early_lo && n <= dc.early_hi) Gv += grad_early[ch0 + n];
                    }
                    Gs[j] = Gv;
                }
                __syncthreads();
                const float* pm = a.mic + 3 * ((size_t)b * M + m);
                const float mx = pm[0], my = pm[1], mz = pm[2];
                float mpx = 0.f, mpy = 0.f, mpz = 0.f;
                if (has) {
                    f2 dx = two_sum(phx, -mx); dx.lo = __fadd_rn(dx.lo, plx);
                    f2 dy = two_sum(phy, -my); dy.lo = __fadd_rn(dy.lo, ply);
                    f2 dz = two_sum(phz, -mz); dz.lo = __fadd_rn(dz.lo, plz);
                    f2 sx = two_prod(dx.hi, dx.hi); sx.lo = __fmaf_rn(__fmul_rn(2.0f, dx.hi), dx.lo, sx.lo);
                    f2 sy = two_prod(dy.hi, dy.hi); sy.lo = __fmaf_rn(__fmul_rn(2.0f, dy.hi), dy.lo, sy.lo);
                    f2 sz = two_prod(dz.hi, dz.hi); sz.lo = __fmaf_rn(__fmul_rn(2.0f, dz.hi), dz.lo, sz.lo);
                    f2 ss = f2_add(f2_add(fast_two_sum(sx.hi, sx.lo), fast_two_sum(sy.hi, sy.lo)),
                                   fast_two_sum(sz.hi, sz.lo));
                    f2 D = f2_sqrt_fast(ss);
                    f2 t = f2_mul(D, a.q2);
                    const int nc = __float2int_rn(t.hi);
                    float delta = __fadd_rn(__fsub_rn(t.hi, (float)nc), t.lo);
                    if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
                    const float invD = rcp_approx(D.hi);
                    const float A = A_g * invD;
                    const int j0 = nc - K - gbase;
                    if ((nc + K >= 0) && (nc - K < Lb)) {
                        if (j0 >= 0 && j0 + 2 * K < P.glen) {
                            float gA, gT;
                            gather_taps<KT>(Gs + j0, K, delta, tab, gA, gT);
                            const float dLdD = __fmaf_rn(-A * gT, qf, -gA * A * invD);
                            const float ex = (dx.hi + dx.lo) * invD, ey = (dy.hi + dy.lo) * invD,
                                        ez = (dz.hi + dz.lo) * invD;
                            gvx = __fmaf_rn(dLdD, ex, gvx);
                            gvy = __fmaf_rn(dLdD, ey, gvy);
                            gvz = __fmaf_rn(dLdD, ez, gvz);
                            mpx = -dLdD * ex; mpy = -dLdD * ey; mpz = -dLdD * ez;
                            pr = __fmaf_rn(gA * A * gg, rc.inv_r, pr);
                        } else {
                            atomicOr(&a.hdr->status, FRAM_DEV_CAPACITY);
                        }
                    }
                }
                // Direct path of (b, s, m): owned by one tile; thread 0 adds it after its image.
                if (own_direct && ch == 0 && tid == 0) {
                    const int nc = __float2int_rn(dc.t_hi);
                    float delta = __fadd_rn(__fsub_rn(dc.t_hi, (float)nc), dc.t_lo);
                    if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
                    const int j0 = nc - K - gbase;
                    if ((nc + K >= 0) && (nc - K < Lb)) {
                        if (j0 >= 0 && j0 + 2 * K < P.glen) {
                            float gA, gT;
                            gather_taps<KT>(Gs + j0, K, delta, tab, gA, gT);
                            const float A = dc.amp;
                            const float dLdD = __fmaf_rn(-A * gT, qf, -gA * A * A);
                            dsx += dLdD * dc.ex; dsy += dLdD * dc.ey; dsz += dLdD * dc.ez;
                            mpx -= dLdD * dc.ex; mpy -= dLdD * dc.ey; mpz -= dLdD * dc.ez;
                        } else {
                            atomicOr(&a.hdr->status, FRAM_DEV_CAPACITY);
                        }
                    }
                }
                // Mic partials: a fixed-order warp sum; each warp keeps its own slot.
                mpx = warp_sum(mpx); mpy = warp_sum(mpy); mpz = warp_sum(mpz);
                if (lane == 0) {
                    float* rw = red + (wid * M + m) * 3;
                    rw[0] += mpx; rw[1] += mpy; rw[2] += mpz;
                }
            }
            if (has && grad_vs) {
                grad_vs[3 * v] = gvx; grad_vs[3 * v + 1] = gvy; grad_vs[3 * v + 2] = gvz;
            }
        }
        pr = warp_sum(pr);
        if (lane == 0) s_r[wid] = pr;
        __syncthreads();
        for (int k = tid; k < 3 * M; k += NT) {
            float acc = 0.f;
            for (int w = 0; w < NW; ++w) acc += red[w * M * 3 + k];
            a.part_mic[(int64_t)qi * 3 * M + k] = acc;
        }
        if (tid == 0) {
            float acc = 0.f;
            for (int w = 0; w < NW; ++w) acc += s_r[w];
            a.part_r[qi] = acc;
            a.part_src[3 * (int64_t)qi] = dsx;
            a.part_src[3 * (int64_t)qi + 1] = dsy;
            a.part_src[3 * (int64_t)qi + 2] = dsz;
        }
        __syncthreads();
    }
}

// Per-room reductions of the item partials, in item order.
__global__ void bwd_reduce(LaunchArgs a, float* __restrict__ grad_mic, float* __restrict__ grad_src,
                           float* __restrict__ grad_r)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nm = (int64_t)a.B * a.M * 3, ns = (int64_t)a.B * a.S * 3;
    if (grad_mic && tid < nm) {
        const int k = (int)(tid % 3), m = (int)((tid / 3) % a.M), b = (int)(tid / (3 * a.M));
        const RoomConst rc = a.room[b];
        const int q0 = rc.item0, q1 = q0 + a.S * rc.ntiles;
        float acc = 0.f;
        for (int q = q0; q < q1; ++q) acc += a.part_mic[(int64_t)q * 3 * a.M + 3 * m + k];
        grad_mic[tid] = acc;
    }
    if (grad_src && tid < ns) {
        const int k = (int)(tid % 3), s = (int)((tid / 3) % a.S), b = (int)(tid / (3 * a.S));
        const RoomConst rc = a.room[b];
        const int q0 = rc.item0 + s * rc.ntiles, q1 = q0 + rc.ntiles;
        float acc = 0.f;
        for (int q = q0; q < q1; ++q) acc += a.part_src[3 * (int64_t)q + k];
        grad_src[tid] = acc;
    }
    if (grad_r && tid < a.B) {
        const RoomConst rc = a.room[tid];
        const int q0 = rc.item0, q1 = q0 + a.S * rc.ntiles;
        float acc = 0.f;
        for (int q = q0; q < q1; ++q) acc += a.part_r[q];
        grad_r[tid] = acc;
    }
}

template <int KT>
cudaError_t launch_bwd_t(const LaunchArgs& a, int margin_i, const float* pos_hi, const float* pos_lo, const float* g,
                         const float* grad_rir, const float* grad_early, float* grad_vs, cudaStream_t st)
{
    constexpr int NT = 256;
    const int smem = bwd_smem(a.tile, a.K, margin_i, a.M, NT / 32).total;
    int per_sm = 0;
    cudaError_t e = kernel_residency((const void*)bwd_kernel<NT, KT>, NT, smem, &per_sm);
    if (e != cudaSuccess) return e;
    bwd_kernel<NT, KT><<<device_sm_count() * per_sm, NT, smem, st>>>(a, margin_i, pos_hi, pos_lo, g, grad_rir,
                                                                     grad_early, grad_vs);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                            const float* r, const float* grad_rir, const float* grad_early, float* grad_vs,
                            float* grad_mic, float* grad_src, float* grad_r, cudaStream_t st)
{
    (void)r;
    if (a.M > 64) return cudaErrorInvalidValue;
    // Host-side bound on any room's per-mic delay spread around the binning key.
    const int margin_i = a.margin_i;
    cudaError_t e;
    if (a.K == 40) e = launch_bwd_t<40>(a, margin_i, pos_hi, pos_lo, g, grad_rir, grad_early, grad_vs, st);
    else if (a.K == 63) e = launch_bwd_t<63>(a, margin_i, pos_hi, pos_lo, g, grad_rir, grad_early, grad_vs, st);
    else e = launch_bwd_t<0>(a, margin_i, pos_hi, pos_lo, g, grad_rir, grad_early, grad_vs, st);
    if (e != cudaSuccess) return e;
    const int64_t n = std::max<int64_t>({(int64_t)a.B * a.M * 3, (int64_t)a.B * a.S * 3, (int64_t)a.B});
    if (n > 0 && (grad_mic || grad_src || grad_r)) {
        bwd_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, grad_mic, grad_src, grad_r);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace fram
