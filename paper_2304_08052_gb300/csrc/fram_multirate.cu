// fram_multirate.cu -- the paper's own multi-rate output path (delay_mode 1; Sec. II-B and
// Eq. 7-9 as printed).
//
// Every arrival (direct path with g = 0, then the images) is an impulse r^g / D at
//   q = min(ceil(D / c0 * r_h fs), L_h - 1),   L_h = ceil(T60 r_h fs),
// on a grid at the high rate r_h fs (r_h = floor(1e6 / fs), about 1 MHz).  That impulse train is
// resampled to r_l fs (r_l = floor(sqrt(r_h))), high-passed at 80 Hz and resampled to fs.  The
// paper does not give the filters; this library uses a Kaiser (beta 5) windowed-sinc polyphase
// resampler of half length 10 max(up, down) with DC gain `up`, and a 2nd-order Butterworth
// high-pass (bilinear transform, cutoff pre-warped), run forward from a zero state.
//
// The ~1 MHz train is never built.  With the first ratio up/down (reduced r_l/r_h), the
// intermediate signal is y1[k] = sum_j A_j F(k down - q_j up): each impulse touches at most 21
// consecutive intermediate samples (|m| <= 10 down).
//   mr_table        the first filter F in polyphase rows: row p holds F(p - HL + i down),
//                   i = 0..31, so the 21 taps of one impulse are one row read by 32 lanes.
//   mr_stage_a      persistent warps over (room, source, tile, mic, sub-tile of 128 r_l
//                   intermediate samples); the images that can reach the sub-tile come from the
//                   32-sample key blocks; each lane evaluates one image's q (the grid decides an
//                   integer): in float-pair arithmetic when that is more than 4e-6 from a grid
//                   point, else in FP64 with the same operations in the same order as an FP64
//                   reference (no fused multiply-add), then each impulse is added with one lane
//                   per tap into the warp's shared buffer (and into the early buffer when q lies
//                   in the Eq. 9 window on the high-rate grid).  Tiles go to y1 in global memory.
//   mr_room_order, mr_hpf_warm, mr_hpf_down<RL>   the high-pass as two complex first-order
//                   sections in FP32, each pairing one zero at z = 1 with one pole (well
//                   conditioned where the direct form, with its poles near z = 1, loses ~1e-5 of
//                   the peak in FP32), fused with the second resampler (ratio 1/r_l, compile-time
//                   taps): one thread walks a piece of Pn output samples of one channel, runs the
//                   recursion and accumulates the 21 outputs each intermediate sample reaches, so
//                   the high-passed signal never goes back to memory.  A piece starts from the
//                   state the recursion reaches over the W samples before it (rho^W <= 1e-9 of
//                   the state it forgets), stored by a warm-up pass; units (piece, room rank,
//                   channel) are grouped so a warp's pieces have nearly equal lengths.
#include <cmath>
#include <utility>

#include "fram_internal.cuh"

namespace fram {
namespace {

constexpr int kMrThreads = 256;
constexpr int kMrNJ = 32;        // polyphase row length (>= 21 taps per impulse)
// Stage A sub-tile: kSubA output samples (kSubA r_l intermediate ones) per unit.  A warp's buffers
// take ~8 KB at r_l = 7 with the early RIR, so three 8-warp CTAs fit an SM (256 took ~15 KB and
// left one CTA, latency-bound at 8 warps; 64 scans too many images twice at the sub-tile edges);
// tiles are multiples of 256.
constexpr int kSubA = 128;

// ---- the second resampler (ratio 1/RL): compile-time Kaiser windowed sinc --------------------
constexpr double cx_pi = 3.14159265358979323846;

constexpr double cx_i0(double x)
{
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= (x / (2.0 * k)) * (x / (2.0 * k));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// sin(pi n / d) for integers, after an exact reduction of n modulo 2d (argument in [-pi, pi]).
constexpr double cx_sinpi_ratio(int n, int d)
{
    int r = n % (2 * d);
    if (r > d) r -= 2 * d;
    if (r < -d) r += 2 * d;
    const double x = cx_pi * (double)r / (double)d;
    double term = x, acc = x;
    for (int j = 1; j < 40; ++j) {
        term *= -x * x / ((2.0 * j) * (2.0 * j + 1.0));
        acc += term;
    }
    return acc;
}

constexpr double cx_sqrt(double v)
{
    if (v <= 0.0) return 0.0;
    double g = v > 1.0 ? v : 1.0;
    for (int i = 0; i < 200; ++i) g = 0.5 * (g + v / g);
    return g;
}

template <int RL>
struct FcTab {
    float v[20 * RL + 1];
};

template <int RL>
constexpr FcTab<RL> make_fc()
{
    constexpr int HL = 10 * RL;
    double w[2 * HL + 1] = {};
    double sum = 0.0;
    const double i0b = cx_i0(5.0);
    for (int m = -HL; m <= HL; ++m) {
        const double lp = (m == 0) ? 1.0 / RL : cx_sinpi_ratio(m, RL) / (cx_pi * (double)m);
        const double rr = (double)m / (double)HL;
        const double win = cx_i0(5.0 * cx_sqrt(1.0 - rr * rr)) / i0b;
        w[m + HL] = lp * win;
        sum += w[m + HL];
    }
    FcTab<RL> t{};
    for (int i = 0; i <= 2 * HL; ++i) t.v[i] = (float)(w[i] / sum);
    return t;
}

template <int RL>
inline constexpr FcTab<RL> kFc = make_fc<RL>();

// ---- the first resampler's table, built on the device in FP64 --------------------------------
__device__ double dev_i0(double x)
{
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= (x / (2.0 * k)) * (x / (2.0 * k));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// F(m), |m| <= HL = 10 max(up, down): lowpass with cutoff pi / max(up, down), Kaiser window,
// scaled to sum to `up`; stored as tab[p * 32 + i] = F(p - HL + i down) (zero past the end).
// One CTA per row p: each CTA forms the normalising sum itself (a few FP64 Bessel series per
// thread) and writes its 32 entries, so the rows are built side by side.
__global__ void __launch_bounds__(256) mr_table(LaunchArgs a)
{
    __shared__ double part[256];
    const int up = a.up, down = a.down, HL = a.HLA;
    const int mx = up > down ? up : down;
    const double i0b = dev_i0(5.0);
    double local = 0.0;
    for (int m = -HL + (int)threadIdx.x; m <= HL; m += blockDim.x) {
        const double lp = (m == 0) ? 1.0 / mx : sinpi((double)m / mx) / (3.14159265358979323846 * m);
        const double rr = (double)m / HL;
        local += lp * dev_i0(5.0 * sqrt(fmax(0.0, 1.0 - rr * rr))) / i0b;
    }
    part[threadIdx.x] = local;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    const double scale = (double)up / part[0];
    for (int e = blockIdx.x * kMrNJ + threadIdx.x; e < (blockIdx.x + 1) * kMrNJ; e += blockDim.x) {
        const int p = e / kMrNJ, i = e % kMrNJ;
        const int m = p - HL + i * down;
        float v = 0.0f;
        if (m <= HL) {
            const double lp = (m == 0) ? 1.0 / mx : sinpi((double)m / mx) / (3.14159265358979323846 * m);
            const double rr = (double)m / HL;
            v = (float)(scale * lp * dev_i0(5.0 * sqrt(fmax(0.0, 1.0 - rr * rr))) / i0b);
        }
        a.mr_tab[e] = v;
    }
}

// ---- stage A ------------------------------------------------------------------------------
__device__ __forceinline__ int64_t ceil_div(int64_t n, int64_t d)   // d > 0
{
    return n >= 0 ? (n + d - 1) / d : -((-n) / d);
}

// ceil(n / d) for |n| < 2^24 and d > 0 without an integer division: n inv_d (inv_d = 1/d rounded,
// n exact in float) is within 2^-22 of n / d relative, less than one for every quotient below
// 2^21, so its ceiling is off by at most one, which an exact integer comparison each way fixes.
__device__ __forceinline__ int64_t ceil_div_small(int n, int d, float inv_d)
{
    int k = __float2int_ru(__fmul_rn((float)n, inv_d));
    if ((int64_t)(k - 1) * d >= n) --k;
    else if ((int64_t)k * d < n) ++k;
    return k;
}

// Intermediate-signal geometry of room b: L_h, L_m and the offset of channel (s, m).
struct MrChan {
    int64_t Lh, Lm, off;
};

__device__ __forceinline__ MrChan mr_chan(const LaunchArgs& a, const RoomConst& rc, int b, int s, int m)
{
    MrChan c;
    c.Lh = (int64_t)ceil(__dmul_rn((double)a.rt60[b], a.fh));
    c.Lm = ceil_div(c.Lh * a.up, a.down);
    // L_m <= r_l L_b + 2 when the device T60 matches the host layout; a channel holds r_l L_b + 5.
    const int64_t cap = (int64_t)a.rl * rc.len + 4;
    if (c.Lm > cap || c.Lh < 1) {
        atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
        c.Lm = c.Lh < 1 ? 0 : cap;
        if (c.Lh < 1) c.Lh = 1;
    }
    const int64_t chan = ((int64_t)b * a.S + s) * a.M + m;
    // rounded up to 4 floats (16 bytes): consecutive channels stay >= r_l L_b + 5 apart
    c.off = ((int64_t)a.rl * (rc.rir_off + ((int64_t)s * a.M + m) * rc.len) + 8 * chan + 3) & ~(int64_t)3;
    return c;
}

// Floats in each intermediate buffer (mr_y, mr_ye): the workspace layout's r_l * sum_b S M L_b
// plus 8 floats of slack per channel and 4 at the end; the debug build's guards check against it.
[[maybe_unused]] __device__ __forceinline__ int64_t mr_inter_floats(const LaunchArgs& a)
{
    return (int64_t)a.rl * a.rir_total + 8 * (int64_t)a.B * a.S * a.M + 4;
}

// Per-warp shared memory (floats): the tile buffer (TA + 64), the early buffer when wanted, and
// 32 staged impulses (A; buffer index of tap 0; filter row and Eq. 9 flag).
__host__ __device__ inline int mr_warp_floats(int TA, bool early) { return (early ? 2 : 1) * (TA + 64) + 3 * 32; }

// Adds a staged impulse: lane j adds A F(m0 + j down) to buffer index bi0 + j.
__device__ __forceinline__ void mr_add_staged(const float* __restrict__ tab, float* buf, float* bufe, int bi0, int row,
                                              float A, int TA, int lane)
{
    const int m0 = row >> 1;
    const float f = tab[m0 * kMrNJ + lane];
    const int bi = bi0 + lane;
    if (bi >= 0 && bi < TA + 64 && f != 0.0f) {
        buf[bi] = __fmaf_rn(A, f, buf[bi]);
        if (bufe && (row & 1)) bufe[bi] = __fmaf_rn(A, f, bufe[bi]);
    }
}

// Adds the impulse (q, A) to the buffers: lane j takes the intermediate sample kmin + j.
__device__ __forceinline__ void mr_add(const float* __restrict__ tab, float* buf, float* bufe, int64_t q, float A,
                                       bool in_early, int64_t K0, int TA, int up, int down, int HL, int lane)
{
    const int64_t c = q * up;
    const int64_t kmin = ceil_div(c - HL, down);
    const int m0 = (int)(kmin * down - c + HL);                  // in [0, down)
    const float f = tab[m0 * kMrNJ + lane];
    const int64_t bi = kmin + lane - K0 + 32;                    // buffer index
    if (bi >= 0 && bi < TA + 64 && f != 0.0f) {
        buf[bi] = __fmaf_rn(A, f, buf[bi]);
        if (bufe && in_early) bufe[bi] = __fmaf_rn(A, f, bufe[bi]);
    }
}

// q = ceil(D r_h fs / c0) from the float-pair image position, when the float-pair value of
// D r_h fs / c0 (error below 1e-7 samples) lies more than 4e-6 from an integer: then the FP64
// evaluation, within 1e-9 of the exact value, has the same ceiling.  Returns false otherwise
// (about one image in 10^5), and the caller decides in FP64.
__device__ __forceinline__ bool mr_delay_pair(float4 pa, float2 pb, float mx, float my, float mz, f2 q2, float rhf,
                                              int64_t Lh, float beyond, int64_t& q, float& D_out)
{
    f2 dx = two_sum(pa.x, -mx); dx.lo = __fadd_rn(dx.lo, pa.w);
    f2 dy = two_sum(pa.y, -my); dy.lo = __fadd_rn(dy.lo, pb.x);
    f2 dz = two_sum(pa.z, -mz); dz.lo = __fadd_rn(dz.lo, pb.y);
    f2 sx = two_prod(dx.hi, dx.hi); sx.lo = __fmaf_rn(__fmul_rn(2.0f, dx.hi), dx.lo, sx.lo);
    f2 sy = two_prod(dy.hi, dy.hi); sy.lo = __fmaf_rn(__fmul_rn(2.0f, dy.hi), dy.lo, sy.lo);
    f2 sz = two_prod(dz.hi, dz.hi); sz.lo = __fmaf_rn(__fmul_rn(2.0f, dz.hi), dz.lo, sz.lo);
    f2 ss = f2_add(f2_add(fast_two_sum(sx.hi, sx.lo), fast_two_sum(sy.hi, sy.lo)), fast_two_sum(sz.hi, sz.lo));
    const f2 D = f2_sqrt_fast(ss);
    const f2 v = f2_mul_f(f2_mul(D, q2), rhf);
    D_out = D.hi;
    if (v.hi > beyond) {                      // beyond = L_h + 2 rounded up: past the clamp either way
        q = Lh - 1;
        return true;
    }
    const float n = rintf(v.hi);
    const float fr = __fadd_rn(__fsub_rn(v.hi, n), v.lo);
    if (!(fabsf(fr) > 4.0e-6f)) return false;
    q = (int64_t)n + (fr > 0.0f ? 1 : 0);
    if (q > Lh - 1) q = Lh - 1;
    return true;
}

__global__ void __launch_bounds__(kMrThreads) mr_stage_a(LaunchArgs a, bool want_early)
{
    extern __shared__ __align__(16) float mr_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int T = a.tile, M = a.M, rl = a.rl, up = a.up, down = a.down, HL = a.HLA;
    const int TA = kSubA * rl, nsub = T / kSubA;
    float* tab = mr_smem;                                        // down x 32
    float* buf = mr_smem + down * kMrNJ + wid * mr_warp_floats(TA, want_early);
    float* bufe = want_early ? buf + TA + 64 : nullptr;
    float* rA = buf + (want_early ? 2 : 1) * (TA + 64);          // staged impulses: A,
    int* rbi = reinterpret_cast<int*>(rA + 32);                  // buffer index of tap 0,
    int* rrow = rbi + 32;                                        // 2 m0 + (q in the Eq. 9 window)
    for (int e = threadIdx.x; e < down * kMrNJ; e += blockDim.x) tab[e] = a.mr_tab[e];
    __syncthreads();
    const double c0 = a.c0, fh = a.fh;
    const float inv_down = 1.0f / (float)down;
    const int64_t n_units = (int64_t)a.hdr->n_items * M * nsub;
    int u = 0;
    if (lane == 0) u = atomicAdd(&a.hdr->queue, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    while ((int64_t)u < n_units) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&a.hdr->queue, 1);
        const int qi = u / (M * nsub);
        const int rem = u - qi * M * nsub;
        const int m = rem / nsub, st = rem - m * nsub;
        const ItemRec ir = a.irec[qi];
        const RoomConst rc = a.room[ir.b];
        const MrChan ch = mr_chan(a, rc, ir.b, ir.s, m);
        const int64_t K0 = (int64_t)ir.T0 * rl + (int64_t)st * TA;
        const int64_t tile_end = (int64_t)rc.ntiles * T * rl;
        const bool last = K0 + TA >= tile_end;
        const int64_t s_end = last ? ch.Lm : (K0 + TA < ch.Lm ? K0 + TA : ch.Lm);
        if (K0 < s_end &&
            FRAM_GUARD(a.hdr, K0 >= 0 && (ch.off & 3) == 0 && ch.off + s_end <= mr_inter_floats(a) &&
                                  ir.v0 >= 0 && (int64_t)ir.v0 + rc.n_vs <= a.n_vs_total)) {
            // TA + 64 is a multiple of 4 and the buffers start on 16 bytes: zero whole float4s
            for (int k = lane; k < (TA + 64) / 4; k += 32) {
                reinterpret_cast<float4*>(buf)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (bufe) reinterpret_cast<float4*>(bufe)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
            const DirectConst dc = a.direct[((int64_t)ir.b * a.S + ir.s) * M + m];
            {   // direct path (g = 0), uniform across the warp
                int64_t q = dc.q_h;
                if (q > ch.Lh - 1) q = ch.Lh - 1;
                if (dc.amp > 0.0f)
                    mr_add(tab, buf, bufe, q, dc.amp, q >= dc.early_lo_h && q <= dc.early_hi_h, K0, TA, up, down,
                           HL, lane);
                __syncwarp();
            }
            // Images whose taps can reach [K0 - 32, K0 + TA + 32): delay (at fs) within 11 r_l
            // intermediate samples and the array margin of the binning key; the last sub-tile
            // also takes every later key (impulses clamped to L_h - 1).
            const int* p32 = a.pos32 + ((int64_t)ir.b * a.S + ir.s) * ((int64_t)a.nb32 + 1);
            const int64_t tmin = (K0 - 64) / rl - a.margin_i - 2;
            const int64_t tmax = (K0 + TA + 64) / rl + a.margin_i + 2;
            const int bmin = (int)(tmin < 0 ? 0 : (tmin >> 5));
            const int bmax = (int)((tmax >> 5) + 1 < a.nb32 ? (tmax >> 5) + 1 : a.nb32);
            const int c_lo = p32[bmin];
            const int c_hi = last ? rc.n_vs : p32[bmax];
            const float* pm = a.mic + 3 * ((size_t)ir.b * M + m);
            const float mxf = pm[0], myf = pm[1], mzf = pm[2];
            const double mx = mxf, my = myf, mz = mzf;
            const float rhf = (float)a.rh;
            const float beyond = __ll2float_ru(ch.Lh + 2);
            for (int cb = c_lo; cb < c_hi; cb += 32) {
                const int p = cb + lane;
                bool valid = false;
                int64_t q = 0;
                float A = 0.0f;
                int bi0 = 0, row = 0;
                if (p < c_hi) {
                    const float4 pa = a.spa[ir.v0 + p];
                    const float2 pb = a.spb[ir.v0 + p];
                    float Df;
                    if (!mr_delay_pair(pa, pb, mxf, myf, mzf, a.q2, rhf, ch.Lh, beyond, q, Df)) {
                        // near a grid point: the reference's FP64 operations in its order
                        const double dx = __dsub_rn(__dadd_rn((double)pa.x, (double)pa.w), mx);
                        const double dy = __dsub_rn(__dadd_rn((double)pa.y, (double)pb.x), my);
                        const double dz = __dsub_rn(__dadd_rn((double)pa.z, (double)pb.y), mz);
                        const double D = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                              __dmul_rn(dz, dz)));
                        const double qh = ceil(__dmul_rn(__ddiv_rn(D, c0), fh));
                        q = (qh > (double)(ch.Lh - 1)) ? ch.Lh - 1 : (int64_t)qh;
                        Df = (float)D;
                    }
                    A = __fdividef(a.samp[ir.v0 + p], Df);       // ~2 ulp; no integer decision rests on A
                    const int64_t c = q * up;
                    const int64_t nn = c - HL;
                    const int64_t kmin = (nn > -(1 << 24) && nn < (1 << 24)) ? ceil_div_small((int)nn, down, inv_down)
                                                                             : ceil_div(nn, down);
                    valid = Df > 0.0f && A == A && fabsf(A) < 3.0e38f && kmin + 31 >= K0 - 32 && kmin < K0 + TA + 32;
                    bi0 = (int)(kmin - K0 + 32);
                    const int m0 = (int)(kmin * down - c + HL);
                    valid = valid && FRAM_GUARD(a.hdr, m0 >= 0 && m0 < down);      // the table row
                    row = 2 * m0 + ((q >= dc.early_lo_h && q <= dc.early_hi_h) ? 1 : 0);
                }
                const unsigned vb = __ballot_sync(0xffffffffu, valid);
                if (valid) {
                    const int slot = __popc(vb & ((1u << lane) - 1u));
                    rA[slot] = A;
                    rbi[slot] = bi0;
                    rrow[slot] = row;
                }
                __syncwarp();
                const int nv = __popc(vb);
                for (int j = 0; j < nv; ++j) {
                    mr_add_staged(tab, buf, bufe, rbi[j], rrow[j], rA[j], TA, lane);
                    __syncwarp();
                }
            }
            // K0 and the channel offset are multiples of 4 samples and buffer index 32 holds
            // sample K0, so whole float4s go out as 16-byte stores; then the tail of a channel.
            const int nk = (int)(s_end - K0), n4 = nk >> 2;
            float4* y4 = reinterpret_cast<float4*>(a.mr_y + ch.off + K0);
            float4* ye4 = bufe ? reinterpret_cast<float4*>(a.mr_ye + ch.off + K0) : nullptr;
            const float4* b4 = reinterpret_cast<const float4*>(buf + 32);
            const float4* be4 = bufe ? reinterpret_cast<const float4*>(bufe + 32) : nullptr;
            for (int v = lane; v < n4; v += 32) {
                y4[v] = b4[v];
                if (bufe) ye4[v] = be4[v];
            }
            if (lane < nk - 4 * n4) {
                const int k = 4 * n4 + lane;
                a.mr_y[ch.off + K0 + k] = buf[32 + k];
                if (bufe) a.mr_ye[ch.off + K0 + k] = bufe[32 + k];
            }
            __syncwarp();
        }
        u = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// ---- stages B and C: the high-pass and the second resampler ----------------------------------
// The 80 Hz Butterworth high-pass H(z) = b0 (1 - z^-1)^2 / ((1 - p z^-1)(1 - p* z^-1)) runs over
// each channel's L_m intermediate samples as a cascade of two complex first-order sections in FP32,
// each pairing one zero at z = 1 with one pole:
//   u[n] = p  u[n-1] + (x[n] - x[n-1]),   v[n] = p* v[n-1] + (u[n] - u[n-1]),   y[n] = b0 Re v[n].
// The poles lie close to z = 1 (|p| ~ 1 - 2.8e-3 at 112 kHz), where the direct form
// y[n] = b0 (x[n] - 2 x[n-1] + x[n-2]) - a1 y[n-1] - a2 y[n-2] amplifies every rounding by its DC
// gain ~ 1/|1 - p|^2 (~1e-5 of the peak in FP32).  A section with its zero at z = 1 has gain <= ~1.4
// at every frequency, and a rounding inside it grows only by sqrt(1 / (1 - |p|^2)) (~20-50 at the
// rates used): ~1e-6 of the peak with heavy low-frequency content.  12 FP32 operations per sample,
// two dependent fused multiply-adds on the critical path of each section.
struct HpfCoef {
    float pr, pi, b0;
};

// p = (1 + s_p) / (1 - s_p) for the analog pole s_p = k (-1 + j) / sqrt(2), k = tan(pi 80 / fsr)
// (the bilinear map with the cutoff pre-warped): Re p = (1 - k^2) / den, Im p = sqrt(2) k / den,
// b0 = 1 / den, den = 1 + sqrt(2) k + k^2 -- the same filter as b0 (1 - 2 z^-1 + z^-2) /
// (1 + a1 z^-1 + a2 z^-2) with a1 = -2 Re p and a2 = |p|^2, in FP64 without cancellation.
__device__ __forceinline__ HpfCoef hpf_coef(double fsr)
{
    const double k = tan(3.14159265358979323846 * 80.0 / fsr);
    const double r2k = sqrt(2.0) * k;
    const double den = 1.0 + r2k + k * k;
    HpfCoef c;
    c.pr = (float)((1.0 - k * k) / den);
    c.pi = (float)(r2k / den);
    c.b0 = (float)(1.0 / den);
    return c;
}

// Rooms whose rank needs the all-pairs count below; larger batches keep their own order.
constexpr int kOrderMax = 65536;

// Every RIR of room b has L_b output samples and ceil(L_b / Pn) pieces; L_b does not decrease
// with T60, so rooms are ranked by decreasing T60 (ties by index; a room the prologue rejected
// last).  counts[p] = the number of rooms with more than p pieces, so the rooms that have a piece p
// are ranks [0, counts[p]).  counts (pmax entries) must be zero on entry.
__global__ void __launch_bounds__(256) mr_room_order(LaunchArgs a, int Pn, int pmax, int* __restrict__ counts)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const RoomConst rb = a.room[b];
    const int Lb = rb.len >= 1 ? rb.len : 0;
    if (a.B <= kOrderMax) {
        const float tb = rb.len >= 1 ? a.rt60[b] : -1.0f;
        int rank = 0;
        for (int c = 0; c < a.B; ++c) {
            const float tc = __ldg(&a.room[c].len) >= 1 ? __ldg(&a.rt60[c]) : -1.0f;
            rank += (tc > tb) || (tc == tb && c < b);
        }
        a.mr_order[rank] = b;
        const int np = (Lb + Pn - 1) / Pn;
        for (int q = 0; q < np && q < pmax; ++q) atomicAdd(&counts[q], 1);
    } else if (b < pmax) {
        counts[b] = a.B;        // unsorted: every room is a candidate for every piece
    }
}

// The high-pass state of one channel: sections u, v and the last input.
struct HpfState {
    float ur, ui, vr, vi, x1;
};

// One sample through the two sections; returns y = b0 Re v.
__device__ __forceinline__ float hpf_step(const HpfCoef& c, HpfState& h, float x0)
{
    const float dx = __fsub_rn(x0, h.x1);
    h.x1 = x0;
    const float nr = __fmaf_rn(c.pr, h.ur, __fmaf_rn(-c.pi, h.ui, dx));       // u <- p u + dx
    const float ni = __fmaf_rn(c.pr, h.ui, __fmul_rn(c.pi, h.ur));
    const float dr = __fsub_rn(nr, h.ur), di = __fsub_rn(ni, h.ui);
    h.ur = nr;
    h.ui = ni;
    const float mr = __fmaf_rn(c.pr, h.vr, __fmaf_rn(c.pi, h.vi, dr));        // v <- p* v + du
    const float mi = __fmaf_rn(c.pr, h.vi, __fmaf_rn(-c.pi, h.vr, di));
    h.vr = mr;
    h.vi = mi;
    return __fmul_rn(c.b0, mr);
}

// A piece's start state, stored by the warm-up pass (one record per channel and piece).
struct PieceState {
    float ur, ui, vr, vi, x1, pad0, pad1, pad2;
};

// Unit t of the units (piece, room rank, channel) in that order, pieces from `first`: the rooms
// with a piece p are ranks [0, counts[p]) (mr_room_order), so a warp's 32 units are pieces of
// nearly equal length.  Returns the piece (-1: none) and sets the room, source, mic and channel
// kind; CH = channels per room.
__device__ __forceinline__ int mr_unit(const LaunchArgs& a, int64_t t, int first, int pmax, const int* counts, int CH,
                                       int& b, int& s, int& m, bool& is_early)
{
    int p = -1;
    for (int q = first; q < pmax; ++q) {
        const int64_t nq = (int64_t)counts[q] * CH;
        if (t < nq) { p = q; break; }
        t -= nq;
    }
    if (p < 0) return -1;
    const int SM = a.S * a.M;
    const int k = (int)(t / CH), j = (int)(t - (int64_t)k * CH);
    b = a.B <= kOrderMax ? a.mr_order[k] : k;
    is_early = j >= SM;
    const int jj = is_early ? j - SM : j;
    s = jj / a.M;
    m = jj - s * a.M;
    return p;
}

// ---- the warm-up pass: each piece's start state --------------------------------------------
constexpr int kSeqThreads = 128;
constexpr int kSeqChunk = 32;              // samples per staged chunk and unit (16 lanes x 2 per row)
constexpr int kSeqRow = kSeqChunk + 4;     // row stride (floats): 16-byte rows

// Asynchronous 8-byte global -> shared copy of n bytes (0, 4 or 8), the rest zero-filled.
__device__ __forceinline__ void cp_async8(float* dst, const float* src, int n)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// Chunk k0 of the warp's 32 units into the staging tile T (row q = unit q), as one group: half-warp
// h copies rows 2 i + h, lane (lane mod 16) samples k0 + 2 (lane mod 16) and the next; anyp: a
// valid pointer of the warp, the (unread) source of zero-byte copies.
__device__ __forceinline__ void seq_stage_in(float* T, float* const* ptr, const int* len, const float* anyp, int k0,
                                             int lane)
{
    const int c2 = 2 * (lane & 15), kk = k0 + c2;
#pragma unroll 8
    for (int i = 0; i < 16; ++i) {
        const int q = 2 * i + (lane >> 4);
        const int Lq = len[q];
        const int n = kk + 1 < Lq ? 8 : (kk < Lq ? 4 : 0);
        cp_async8(T + q * kSeqRow + c2, n ? ptr[q] + kk : anyp, n);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Piece p >= 1 starts at k_s = r_l (p Pn - kMrHalo); its start state is the state the recursion
// reaches from a zero state over the W samples before k_s (exact when k_s <= W: it starts at 0).
// Each unit reads those samples (staged in 32-sample chunks) and stores the state.
__global__ void __launch_bounds__(kSeqThreads) mr_hpf_warm(LaunchArgs a, bool with_early, int Pn, int W, int pmax,
                                                           const int* __restrict__ counts,
                                                           PieceState* __restrict__ state)
{
    __shared__ __align__(16) float tile[kSeqThreads / 32][2][32 * kSeqRow];
    __shared__ float* wptr[kSeqThreads / 32][32];
    __shared__ int wlen[kSeqThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int SM = a.S * a.M;
    const int CH = SM * (with_early ? 2 : 1);
    int b = 0, s = 0, m = 0;
    bool is_early = false;
    const int p = mr_unit(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, 1, pmax, counts, CH, b, s, m, is_early);
    int len = 0;
    float* x = nullptr;
    PieceState* rec = nullptr;
    if (p >= 1) {
        const RoomConst rc = a.room[b];
        if (rc.len >= 1) {
            const MrChan ch = mr_chan(a, rc, b, s, m);
            const int64_t ks = (int64_t)a.rl * ((int64_t)p * Pn - kMrHalo);
            if (ks > 0 && ks <= ch.Lm &&
                FRAM_GUARD(a.hdr, (ch.off & 3) == 0 && ch.off + ch.Lm <= mr_inter_floats(a))) {
                const int64_t gc = ((int64_t)b * a.S + s) * a.M + m + (is_early ? (int64_t)a.B * SM : 0);
                rec = state + gc * pmax + p;
                const int64_t b0 = ks > W ? ks - W : 0;           // both multiples of 4
                x = (is_early ? a.mr_ye : a.mr_y) + ch.off + b0;
                len = (int)(ks - b0);
            }
        }
    }
    float* const* ptr = wptr[wid];
    const int* lens = wlen[wid];
    wptr[wid][lane] = x;
    wlen[wid][lane] = len;
    int Lw = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, o));
    __syncwarp();
    if (Lw == 0) return;                     // the whole warp has no unit (uniform)
    const HpfCoef c = hpf_coef((double)a.rl * a.fs);
    HpfState h{0.f, 0.f, 0.f, 0.f, 0.f};
    const unsigned has = __ballot_sync(0xffffffffu, x != nullptr);
    const float* anyp = ptr[__ffs(has) - 1];
    seq_stage_in(tile[wid][0], ptr, lens, anyp, 0, lane);
    for (int k0 = 0, buf = 0; k0 < Lw; k0 += kSeqChunk, buf ^= 1) {
        // The next chunk flies while this one is filtered; its buffer was emptied by the previous chunk.
        if (k0 + kSeqChunk < Lw) {
            seq_stage_in(tile[wid][buf ^ 1], ptr, lens, anyp, k0 + kSeqChunk, lane);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncwarp();
        const float* row = tile[wid][buf] + lane * kSeqRow;
        // stop exactly at the unit's last sample
        const int n = len - k0 < kSeqChunk ? (len - k0 > 0 ? len - k0 : 0) : kSeqChunk;
        for (int i = 0; i < n; ++i) hpf_step(c, h, row[i]);
        __syncwarp();
    }
    if (rec) *rec = PieceState{h.ur, h.ui, h.vr, h.vi, h.x1, 0.f, 0.f, 0.f};
}

// ---- the high-pass fused with the second resampler (ratio 1/RL, compile-time taps) -----------
// Output n of a channel is y[n] = sum_k z[k] F_C(n RL - k), |n RL - k| <= HLC = 10 RL, z the
// high-passed intermediate signal (zero outside [0, L_m)).  One thread walks one piece: it runs the
// recursion from k_s = RL (n_lo - kMrHalo) in groups of RL samples (group m = samples m RL + j,
// j < RL) and keeps 21 accumulators, acc[t] for output m - 10 + t: sample j of group m adds
// z F_C((t - 10) RL - j) = z c[t RL - j] to every t it reaches (t >= 1 when j > 0), and after its
// first sample output m - 10 is complete.  Iterations take 4 groups = 4 RL samples of each of the
// warp's 32 pieces (k_s is a multiple of 4, so these are RL whole 16-byte vectors per piece), staged
// through shared memory by double-buffered asynchronous copies; every sample's register and
// coefficient are then compile-time.
// Two warps per block: a block keeps its slot until its slowest warp's pieces end, so small blocks
// waste less of the SM on pieces of unequal length (64 threads: 8.78 against 9.2 ms per
// batch_1024 step with 128; 32 took 9.1).
constexpr int kFuseThreads = 64;

struct FuseRow {
    const float* x;     // the channel's intermediate signal (sample 0)
    int ks, lm;         // first sample of the piece's walk (may be negative), L_m
};

// Asynchronous 16-byte global -> shared copy of n bytes (0..16), the rest zero-filled.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int n)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

template <int RL>
struct FuseLane {
    HpfCoef c;
    HpfState h;
    float acc[21];
    int rb;             // L_m - k_s: z is zero from this walk position on
    int n_lo, n_hi;     // the piece's outputs
    float* y;           // the channel's output (sample 0)

    template <int J, int T>
    __device__ __forceinline__ void add1(float z)
    {
        constexpr int i = T * RL - J;
        if constexpr (i >= 0) {
            constexpr float cf = kFc<RL>.v[i];
            acc[T] = __fmaf_rn(z, cf, acc[T]);
        }
    }
    template <int J, int... T>
    __device__ __forceinline__ void add(float z, std::integer_sequence<int, T...>)
    {
        (add1<J, T>(z), ...);
    }
    // walk position r (a multiple of RL plus J)
    template <int J>
    __device__ __forceinline__ void sample(float x, int r)
    {
        const float z0 = hpf_step(c, h, x);
        add<J>(r < rb ? z0 : 0.0f, std::make_integer_sequence<int, 21>{});
    }
    template <int J0, int... J>
    __device__ __forceinline__ void rest(const float* xv, int r, std::integer_sequence<int, J...>)
    {
        (sample<J + 1>(xv[J0 + J + 1], r + J + 1), ...);
    }
    // group GG of the iteration starting at walk position r0; g = the group's walk index
    template <int GG>
    __device__ __forceinline__ void group(const float* xv, int r0, int g)
    {
        constexpr int J0 = GG * RL;
        sample<0>(xv[J0], r0 + J0);
        const int n = n_lo + g - (kMrHalo + 10);
        if (g >= kMrHalo + 10 && n < n_hi) y[n] = acc[0];
        rest<J0>(xv, r0 + J0, std::make_integer_sequence<int, RL - 1>{});
#pragma unroll
        for (int t = 0; t < 20; ++t) acc[t] = acc[t + 1];
        acc[20] = 0.0f;
    }
};

template <int RL>
__global__ void __launch_bounds__(kFuseThreads) mr_hpf_down(LaunchArgs a, bool with_early, int Pn, int pmax,
                                                            const int* __restrict__ counts,
                                                            const PieceState* __restrict__ state,
                                                            float* __restrict__ rir, float* __restrict__ early)
{
    constexpr int CHK = 4 * RL;          // walk samples per iteration
    constexpr int RS = 8 * RL + 4;       // row stride (floats): two slots; RS / 4 odd, so the
                                         // 16-byte reads of 8 rows hit distinct banks
    __shared__ __align__(16) float ring[kFuseThreads / 32][32 * RS];
    __shared__ __align__(16) FuseRow rows[kFuseThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int SM = a.S * a.M;
    const int CH = SM * (with_early ? 2 : 1);
    int b = 0, s = 0, m = 0;
    bool is_early = false;
    const int p = mr_unit(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, 0, pmax, counts, CH, b, s, m, is_early);
    FuseLane<RL> L;
    L.c = hpf_coef((double)RL * a.fs);
    L.h = HpfState{0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 21; ++t) L.acc[t] = 0.0f;
    L.rb = 0;
    L.n_lo = 0;
    L.n_hi = 0;
    L.y = nullptr;
    FuseRow row{nullptr, 0, 0};
    int groups = 0;
    if (p >= 0) {
        const RoomConst rc = a.room[b];
        const int n_lo = p * Pn;
        if (rc.len >= 1 && n_lo < rc.len) {
            const MrChan ch = mr_chan(a, rc, b, s, m);
            if (FRAM_GUARD(a.hdr, (ch.off & 3) == 0 && ch.off + ch.Lm <= mr_inter_floats(a) && rc.rir_off >= 0 &&
                                      rc.rir_off + ((int64_t)s * a.M + m + 1) * rc.len <= a.rir_total)) {
                const int ks = RL * (n_lo - kMrHalo);
                L.n_lo = n_lo;
                L.n_hi = min(n_lo + Pn, rc.len);
                L.rb = (int)(ch.Lm - ks);
                L.y = (is_early ? early : rir) + rc.rir_off + ((int64_t)s * a.M + m) * rc.len;
                row = FuseRow{(is_early ? a.mr_ye : a.mr_y) + ch.off, ks, (int)ch.Lm};
                groups = L.n_hi - n_lo + kMrHalo + 10;
                if (p > 0 && ks > 0) {
                    const int64_t gc = ((int64_t)b * a.S + s) * a.M + m + (is_early ? (int64_t)a.B * SM : 0);
                    const PieceState st = state[gc * pmax + p];
                    L.h = HpfState{st.ur, st.ui, st.vr, st.vi, st.x1};
                }
            }
        }
    }
    rows[wid][lane] = row;
    int its = (groups + 3) / 4;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) its = max(its, __shfl_xor_sync(0xffffffffu, its, o));
    __syncwarp();
    if (its == 0) return;                    // the whole warp has no unit (uniform)
    const unsigned has = __ballot_sync(0xffffffffu, row.x != nullptr);
    const float* anyp = rows[wid][__ffs(has) - 1].x;
    // iteration `it` of every row into slot it & 1: vector v = i 32 + lane is vector e of row q
    auto stage = [&](int it) {
        float* slot = ring[wid] + (it & 1) * CHK;
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const int v = i * 32 + lane;
            const int q = v / RL, e = v - q * RL;
            const FuseRow rq = rows[wid][q];
            const int k = rq.ks + it * CHK + 4 * e;
            int nb = k < 0 ? 0 : 4 * (rq.lm - k);
            nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
            cp_async16(slot + q * RS + 4 * e, nb ? rq.x + k : anyp, nb);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    stage(0);
    for (int it = 0; it < its; ++it) {
        if (it + 1 < its) {
            stage(it + 1);       // its slot was emptied by iteration it - 1
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncwarp();
        const float4* src = reinterpret_cast<const float4*>(ring[wid] + lane * RS + (it & 1) * CHK);
        float xv[CHK];
#pragma unroll
        for (int e = 0; e < RL; ++e) {
            const float4 q = src[e];
            xv[4 * e] = q.x;
            xv[4 * e + 1] = q.y;
            xv[4 * e + 2] = q.z;
            xv[4 * e + 3] = q.w;
        }
        const int r0 = it * CHK;
        L.template group<0>(xv, r0, 4 * it);
        L.template group<1>(xv, r0, 4 * it + 1);
        L.template group<2>(xv, r0, 4 * it + 2);
        L.template group<3>(xv, r0, 4 * it + 3);
        __syncwarp();
    }
}

template <int RL>
cudaError_t launch_hpf_down(const LaunchArgs& a, int Pn, int pmax, const int* counts, const PieceState* pstate,
                            float* rir, float* early, cudaStream_t st)
{
    const int64_t nthr = (int64_t)a.B * a.S * a.M * (early ? 2 : 1) * pmax;
    if (nthr == 0) return cudaSuccess;
    const unsigned nblk = (unsigned)((nthr + kFuseThreads - 1) / kFuseThreads);
    mr_hpf_down<RL><<<nblk, kFuseThreads, 0, st>>>(a, early != nullptr, Pn, pmax, counts, pstate, rir, early);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_synthesize_mr(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, float* rir,
                                 float* early, cudaStream_t st)
{
    (void)pos_hi;
    (void)pos_lo;     // stage A reads the sorted copies the preparation made
    if (a.B == 0) return cudaSuccess;
    mr_table<<<a.down, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int TA = kSubA * a.rl;
    const int smem = (int)sizeof(float) * (a.down * kMrNJ + (kMrThreads / 32) * mr_warp_floats(TA, early != nullptr));
    int per_sm = 0;
    if ((e = kernel_residency((const void*)mr_stage_a, kMrThreads, smem, &per_sm)) != cudaSuccess) return e;
    mr_stage_a<<<device_sm_count() * per_sm, kMrThreads, smem, st>>>(a, early != nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // stages B and C: the high-pass fused with the second resampler, in pieces (warm-up states first)
    const MrPieces pc = mr_pieces(a.fs, a.max_len);
    int* counts = a.mr_counts;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * pc.pmax, st)) != cudaSuccess) return e;
    mr_room_order<<<(a.B + 255) / 256, 256, 0, st>>>(a, pc.Pn, pc.pmax, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    PieceState* pstate = reinterpret_cast<PieceState*>(a.mr_pstate);
    if (pc.pmax > 1) {
        const int64_t nthr = (int64_t)a.B * a.S * a.M * (early ? 2 : 1) * (pc.pmax - 1);
        const unsigned nblk = (unsigned)((nthr + kSeqThreads - 1) / kSeqThreads);
        mr_hpf_warm<<<nblk, kSeqThreads, 0, st>>>(a, early != nullptr, pc.Pn, pc.W, pc.pmax, counts, pstate);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    switch (a.rl) {
    case 2: return launch_hpf_down<2>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 3: return launch_hpf_down<3>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 4: return launch_hpf_down<4>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 5: return launch_hpf_down<5>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 6: return launch_hpf_down<6>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 7: return launch_hpf_down<7>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 8: return launch_hpf_down<8>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 9: return launch_hpf_down<9>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 10: return launch_hpf_down<10>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    case 11: return launch_hpf_down<11>(a, pc.Pn, pc.pmax, counts, pstate, rir, early, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fram
