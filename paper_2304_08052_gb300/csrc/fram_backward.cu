// fram_backward.cu -- adjoint of the windowed-sinc synthesis (gradients of a loss on the RIR
// with respect to source, mic and image positions and the reflection coefficient).
//
// Ownership instead of scattering: every image belongs to exactly one (room, source, tile)
// work item -- the tile its binning key (delay to the array centre) falls in -- and the
// direct path of a (room, source) belongs to the tile of the source's key.  A persistent warp
// takes an item and walks its images in passes of up to 128 (one image per lane, four chunks);
// for each mic it stages the upstream gradient
//   G[n] = dL/dh[n] + [n in Eq. 9 window] dL/dh_e[n]
// over the tile plus a halo of K + margin samples in its own shared memory, and each lane
// recomputes its image's arrival (float-pair delay, amplitude) and gathers the arrival's 2K taps
// (the support |n - t| < K, see the synthesis kernel for the re-based split t = base + delta):
//   S1 = sum G tap,   S2 = sum G dtap/dt,   tap = sigma (P + a C + b S) / (delta - o)
// with per-tap constants C = cos(pi o/K), S = sin(pi o/K), sigma = (-1)^o, and per-arrival
// P = sin(pi delta)/(2 pi), a = P cos(pi delta/K), b = P sin(pi delta/K) and their delta
// derivatives P', a', b', so that dtap/dt = (dnum - sigma tap) / e with e = sigma (delta - o).
// That quotient cancels on the tap nearest to t (|n - t| <= 1/2), which instead takes
// d/dt [sinc w] from a Taylor series of sinc'.  With A = r^g / D the chain rule gives
//   dL/dA = S1,  dL/dt = A S2,  dL/dD = A S2 fs/c0 - S1 A / D,  dD/dp = (p - mic)/D,
//   dL/dr = S1 A g / r,  dL/dg = S1 A ln r (summed over mics; for the gradient through the sampler).
// Image gradients are summed over mics in mic order by the owning lane; mic, source and r
// gradients are reduced per item in a fixed warp tree and then per room in item order, so the
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

// Compile-time copies: the unrolled tap loops read them as literal FMA operands.
template <int K>
inline constexpr TrigTab kTrig = make_trig_tab<K>();

constexpr float kShiftMin = 2.44140625e-4f;   // 2^-12: arrivals re-based as in the synthesis
constexpr float kTwoPiInv = 0.15915494309189535f;
constexpr int kBwdThreads = 128;
constexpr int kBwdChunks = 4;                   // images per lane and pass

// Per-arrival constants of the adjoint, unit amplitude.  d = delta of the re-based split,
// (P, a, b) and their delta derivatives (Pp, ap, bp), dnear = d/dt of the tap nearest to t,
// shifted = the arrival was re-based to n_c + 1.
struct ArrB {
    float d, P, a, b, Pp, ap, bp, dnear;
    bool shifted;
};

// cK, sK = cos, sin(pi / K): the rotation from the re-based delta to the original one.
__device__ __forceinline__ ArrB arrival_bwd(int& nc, float delta, float invK, bool exact_trig, float cK, float sK)
{
    ArrB r;
    if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
    r.shifted = delta > kShiftMin;
    if (r.shifted) {
        const float d1 = __fsub_rn(delta, 1.0f);
        delta = __fadd_rn(d1, 1.0f);                              // the delta the taps use
        r.d = d1;
        nc += 1;
    } else {
        r.d = delta;
    }
    // sin, cos (pi delta) at the delta the taps use (the re-based one negates both)
    const float sdl = sinpi_poly(delta), cdl = cospi_poly(delta);
    const float su = r.shifted ? -sdl : sdl, cu = r.shifted ? -cdl : cdl;
    const float piK = kPi * invK;
    float cy, sy, cn, sn;
    if (exact_trig) {
        sincospif(r.d * invK, &sy, &cy);
        sincospif(delta * invK, &sn, &cn);
    } else {
        cy = cospi_poly(r.d * invK); sy = sinpi_poly(r.d * invK);
        // re-based: delta = r.d + 1, so (cn, sn) is (cy, sy) rotated by pi / K
        cn = r.shifted ? __fmaf_rn(cy, cK, -sy * sK) : cy;
        sn = r.shifted ? __fmaf_rn(sy, cK, cy * sK) : sy;
    }
    r.P = su * kTwoPiInv;
    r.Pp = 0.5f * cu;
    r.a = r.P * cy;
    r.b = r.P * sy;
    r.ap = __fmaf_rn(r.Pp, cy, -r.P * piK * sy);
    r.bp = __fmaf_rn(r.Pp, sy, r.P * piK * cy);
    // Nearest tap: x = n - t = -delta (delta of the original split), tap = sinc(x) w(x), both
    // even, so dtap/dt = sinc'(delta) w(delta) + sinc(delta) w'(delta).
    const float sinc = sdl * kInvPi * rcp_approx(delta);      // |delta| >= kTinyDelta
    const float w = 0.5f * (1.0f + cn);
    const float wp = -0.5f * piK * sn;
    r.dnear = __fmaf_rn(dsinc_small(delta), w, sinc * wp);
    return r;
}

// S1 = sum_j G[j] tap_j, S2 = sum_j G[j] dtap_j/dt over the 2K slots j = o + K of one arrival;
// Gs points at G[base - K].  With r_j = 1/e_j the per-arrival constants factor out:
//   S1 = P U0 + a U1 + b U2,   S2 = P' U0 + a' U1 + b' U2 - (P V0 + a V1 + b V2),
//   U = sum G r (1, C, S),  V = sum G sigma r^2 (1, C, S),
// so a slot costs one reciprocal, two multiplies and six accumulations.  The two central slots
// (o = -1, 0), one of which holds the tap nearest to t, stay out of U and V and are added
// directly (the nearest one with its Taylor-series derivative).  Compile-time K: every per-slot
// constant is a literal operand.
//
// Slots go in pairs (J even, J + 1), the pair's values in the two halves of packed FP32
// registers: the constant-free products G r and G r^2 and the sums of U0 and V0 use
// mul/add.rn.f32x2 (two independent IEEE operations per instruction, each half rounded as the
// scalar operation would be), the products with the per-slot literals stay scalar.  Each
// accumulator keeps an even-slot and an odd-slot partial sum; V sums are taken without sigma,
// which is constant within each half (the slot parity fixes the sign of o) and enters when the
// halves are added.
struct TapAcc {
    float u0, u1, u2, v0, v1, v2;
};
// Packed partial sums: low half even slots, high half odd slots; u1/u2/v1/v2 as scalars per half.
struct TapAccP {
    f32x2 u0, v0;
    float u1e, u1o, u2e, u2o, v1e, v1o, v2e, v2o;
};

template <int KT, int J>
__device__ __forceinline__ void tap_half(const float* __restrict__ Gs, float d, float& u0, float& u1, float& u2,
                                         float& v0, float& v1, float& v2)
{
    constexpr int o = J - KT;
    constexpr float sg = (o & 1) ? -1.0f : 1.0f;
    constexpr float C = kTrig<KT>.c[J];
    constexpr float S = kTrig<KT>.s[J];
    constexpr float kp = -sg * (float)o;
    const float rc = rcp_approx(__fmaf_rn(sg, d, kp));
    const float y = __fmul_rn(Gs[J], rc);
    u0 = __fadd_rn(u0, y);
    u1 = __fmaf_rn(C, y, u1);
    u2 = __fmaf_rn(S, y, u2);
    const float z = __fmul_rn(y, rc);
    v0 = __fadd_rn(v0, z);
    v1 = __fmaf_rn(C, z, v1);
    v2 = __fmaf_rn(S, z, v2);
}

template <int KT, int J>
__device__ __forceinline__ void tap_pair(const float* __restrict__ Gs, float d, TapAccP& q)
{
    constexpr int o0 = J - KT, o1 = J + 1 - KT;
    constexpr bool c0 = o0 == 0 || o0 == -1, c1 = o1 == 0 || o1 == -1;
    if constexpr (!c0 && !c1) {
        constexpr float sg0 = (o0 & 1) ? -1.0f : 1.0f, sg1 = -sg0;
        constexpr float C0 = kTrig<KT>.c[J], C1 = kTrig<KT>.c[J + 1];
        constexpr float S0 = kTrig<KT>.s[J], S1 = kTrig<KT>.s[J + 1];
        const f32x2 rc = pack2(rcp_approx(__fmaf_rn(sg0, d, -sg0 * (float)o0)),
                               rcp_approx(__fmaf_rn(sg1, d, -sg1 * (float)o1)));
        const f32x2 y = mul2(pack2(Gs[J], Gs[J + 1]), rc);
        q.u0 = add2(q.u0, y);
        float y0, y1;
        unpack2(y, y0, y1);
        q.u1e = __fmaf_rn(C0, y0, q.u1e);
        q.u1o = __fmaf_rn(C1, y1, q.u1o);
        q.u2e = __fmaf_rn(S0, y0, q.u2e);
        q.u2o = __fmaf_rn(S1, y1, q.u2o);
        const f32x2 z = mul2(y, rc);
        q.v0 = add2(q.v0, z);
        float z0, z1;
        unpack2(z, z0, z1);
        q.v1e = __fmaf_rn(C0, z0, q.v1e);
        q.v1o = __fmaf_rn(C1, z1, q.v1o);
        q.v2e = __fmaf_rn(S0, z0, q.v2e);
        q.v2o = __fmaf_rn(S1, z1, q.v2o);
    } else if constexpr (!c0 || !c1) {
        // one central slot in the pair: the other one alone, into its own half
        float u0e, u0o, v0e, v0o;
        unpack2(q.u0, u0e, u0o);
        unpack2(q.v0, v0e, v0o);
        if constexpr (!c0) tap_half<KT, J>(Gs, d, u0e, q.u1e, q.u2e, v0e, q.v1e, q.v2e);
        else tap_half<KT, J + 1>(Gs, d, u0o, q.u1o, q.u2o, v0o, q.v1o, q.v2o);
        q.u0 = pack2(u0e, u0o);
        q.v0 = pack2(v0e, v0o);
    }
}

template <int KT, int... P>
__device__ __forceinline__ void tap_pairs(const float* __restrict__ Gs, float d, TapAccP& q,
                                          std::integer_sequence<int, P...>)
{
    (tap_pair<KT, 2 * P>(Gs, d, q), ...);
}

// One central slot o in {-1, 0}: value and derivative added directly.
__device__ __forceinline__ void central_slot(float G, int o, float C, float S, const ArrB& r, float& S1, float& S2)
{
    const float sg = (o & 1) ? -1.0f : 1.0f;
    const float e = __fmaf_rn(sg, r.d, -sg * (float)o);
    const float rc = rcp_approx(e);
    const float num = __fmaf_rn(C, r.a, __fmaf_rn(S, r.b, r.P));
    const float dnum = __fmaf_rn(C, r.ap, __fmaf_rn(S, r.bp, r.Pp));
    const float tap = num * rc;
    const bool near = (o == 0) != r.shifted;
    const float dtap = near ? r.dnear : (dnum - sg * tap) * rc;
    S1 = __fmaf_rn(G, tap, S1);
    S2 = __fmaf_rn(G, dtap, S2);
}

template <int KT>
__device__ __forceinline__ void gather_taps_ct(const float* __restrict__ Gs, const ArrB& r, float& S1, float& S2)
{
    TapAccP p{0ull, 0ull, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    tap_pairs<KT>(Gs, r.d, p, std::make_integer_sequence<int, KT>{});
    // sigma of the even slots (o = J - K with J even) and of the odd ones
    constexpr float sge = (KT & 1) ? -1.0f : 1.0f;
    float u0e, u0o, v0e, v0o;
    unpack2(p.u0, u0e, u0o);
    unpack2(p.v0, v0e, v0o);
    TapAcc q;
    q.u0 = u0e + u0o;
    q.u1 = p.u1e + p.u1o;
    q.u2 = p.u2e + p.u2o;
    q.v0 = sge * (v0e - v0o);
    q.v1 = sge * (p.v1e - p.v1o);
    q.v2 = sge * (p.v2e - p.v2o);
    S1 = __fmaf_rn(r.P, q.u0, __fmaf_rn(r.a, q.u1, r.b * q.u2));
    S2 = __fmaf_rn(r.Pp, q.u0, __fmaf_rn(r.ap, q.u1, r.bp * q.u2))
         - __fmaf_rn(r.P, q.v0, __fmaf_rn(r.a, q.v1, r.b * q.v2));
    constexpr float Cm = kTrig<KT>.c[KT - 1], Sm = kTrig<KT>.s[KT - 1];
    central_slot(Gs[KT - 1], -1, Cm, Sm, r, S1, S2);
    central_slot(Gs[KT], 0, 1.0f, 0.0f, r, S1, S2);
}

// Any K: the same taps, cos/sin(pi o/K) from a shared table.
__device__ __forceinline__ void gather_taps_rt(const float* __restrict__ Gs, int K, const ArrB& r,
                                               const float2* __restrict__ tab, float& S1, float& S2)
{
    float s1 = 0.f, s2 = 0.f;
    for (int j = 0; j < 2 * K; ++j) {
        const int o = j - K;
        const float sg = (o & 1) ? -1.0f : 1.0f;
        const float2 cs = tab[j];
        const float G = Gs[j];
        const float e = __fmaf_rn(sg, r.d, -sg * (float)o);
        const float rc = rcp_approx(e);
        const float num = __fmaf_rn(cs.x, r.a, __fmaf_rn(cs.y, r.b, r.P));
        const float dnum = __fmaf_rn(cs.x, r.ap, __fmaf_rn(cs.y, r.bp, r.Pp));
        s1 = __fmaf_rn(G * rc, num, s1);
        const bool near = (o == 0 && !r.shifted) || (o == -1 && r.shifted);
        const float dg = (dnum - sg * (num * rc)) * rc;
        s2 = __fmaf_rn(G, near ? r.dnear : dg, s2);
    }
    S1 = s1;
    S2 = s2;
}

// Per-warp shared memory (floats): two staging buffers of the upstream gradient (each covers a
// key span of up to smax samples plus a halo of K + margin + 2 on both sides) and the
// image-gradient accumulators of one pass ([chunk][xyz][lane], then [chunk][lane] of dL/dA A
// summed over mics when dL/dg is wanted).
__host__ __device__ inline int bwd_span(int T) { return T < 1024 ? T : 1024; }
__host__ __device__ inline int bwd_glen(int T, int K, int margin_i)
{
    // an image pass needs at most span + 2K + 2 margin + 6; a direct-only pass 2K + 4 margin + 8
    const int sp = bwd_span(T) > 2 * margin_i + 2 ? bwd_span(T) : 2 * margin_i + 2;
    return (sp + 2 * K + 2 * margin_i + 6 + 3 + 8) & ~3;       // + 8: the staging's shift and last vector
}
__host__ __device__ inline int bwd_warp_floats(int T, int K, int margin_i, bool with_g)
{
    return 2 * bwd_glen(T, K, margin_i) + kBwdChunks * (with_g ? 4 : 3) * 32;
}
__host__ __device__ inline int bwd_tab_floats(int K) { return (4 * K + 3) & ~3; }

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Image geometry for mic (mx, my, mz): delay split n_c + delta, distance D and the exact
// difference p - mic (as hi + lo), from the float-pair image position.
__device__ __forceinline__ void image_geom(float4 pa, float2 pb, float mx, float my, float mz, f2 q2, int& nc,
                                           float& delta, float& D, float& ux, float& uy, float& uz)
{
    f2 dx = two_sum(pa.x, -mx); dx.lo = __fadd_rn(dx.lo, pa.w);
    f2 dy = two_sum(pa.y, -my); dy.lo = __fadd_rn(dy.lo, pb.x);
    f2 dz = two_sum(pa.z, -mz); dz.lo = __fadd_rn(dz.lo, pb.y);
    f2 sx = two_prod(dx.hi, dx.hi); sx.lo = __fmaf_rn(__fmul_rn(2.0f, dx.hi), dx.lo, sx.lo);
    f2 sy = two_prod(dy.hi, dy.hi); sy.lo = __fmaf_rn(__fmul_rn(2.0f, dy.hi), dy.lo, sy.lo);
    f2 sz = two_prod(dz.hi, dz.hi); sz.lo = __fmaf_rn(__fmul_rn(2.0f, dz.hi), dz.lo, sz.lo);
    f2 ss = f2_add(f2_add(fast_two_sum(sx.hi, sx.lo), fast_two_sum(sy.hi, sy.lo)), fast_two_sum(sz.hi, sz.lo));
    f2 Dp = f2_sqrt_fast(ss);
    f2 t = f2_mul(Dp, q2);
    nc = __float2int_rn(t.hi);
    delta = __fadd_rn(__fsub_rn(t.hi, (float)nc), t.lo);
    D = Dp.hi;
    ux = dx.hi + dx.lo; uy = dy.hi + dy.lo; uz = dz.hi + dz.lo;
}

// (sorted g) for the adjoint, into the sorted-amplitude scratch.
__global__ void __launch_bounds__(256) g_gather(LaunchArgs a, const float* __restrict__ g)
{
    const int64_t seg = blockIdx.x;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    if (rc.ntiles < 1) return;
    const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
    for (int p = threadIdx.x; p < rc.n_vs; p += blockDim.x) {
        const int q = a.perm[v0 + p];
        if (FRAM_GUARD(a.hdr, q >= 0 && q < rc.n_vs && v0 + rc.n_vs <= a.n_vs_total)) a.samp[v0 + p] = g[v0 + q];
    }
}

// Asynchronous 4-byte global -> shared copy; a zero source size fills zeros and reads nothing.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One round of a pass: one arrival per lane (an image of chunk ch, or the direct path), with
// what the chain rule needs after the tap gather.
struct BwdRound {
    bool go, is_dir;
    int j0;                 // staged-gradient index of the arrival's slot 0
    float A, invD, ex, ey, ez, gg;
    ArrB r;
};

// One pass of an item: sorted positions [p0, p1) (at most 32 kBwdChunks images whose key blocks
// start less than bwd_span samples apart); the gradient is staged over [gb, gb + gl).
struct BwdPass {
    int p0, p1, gb, gl;
};

__device__ __forceinline__ BwdPass next_pass(const LaunchArgs& a, int64_t v0, int p0, int o_hi, int span, int K,
                                             int Mg, int lane)
{
    BwdPass P;
    P.p0 = p0;
    const int k0 = a.skey[v0 + p0];
    int p1 = min(p0 + 32 * kBwdChunks, o_hi);
    for (int c = 0; c < kBwdChunks; ++c) {
        const int p = p0 + 32 * c + lane;
        const bool stop = p < p1 && a.skey[v0 + p] >= k0 + span;
        const unsigned bal = __ballot_sync(0xffffffffu, stop);
        if (bal) {
            p1 = p0 + 32 * c + __ffs(bal) - 1;
            if (p1 - p0 > 32) p1 = p0 + ((p1 - p0) & ~31);   // whole chunks: no idle lanes
            break;
        }
    }
    P.p1 = p1;
    // skey is the first sample of a 32-sample key block: keys of block k1 reach k1 + 31, and
    // k1 - k0 <= span - 32 because both are block starts.
    const int k1 = a.skey[v0 + p1 - 1];
    P.gb = k0 - K - Mg - 2;
    P.gl = k1 - k0 + 32 + 2 * K + 2 * Mg + 6;
    return P;
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned), bypassing L1.
__device__ __forceinline__ void cp_async16(float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Stages G = dL/dh (+ Eq. 9 mask * dL/dh_e) of channel ch0 over [gb, gb + gl) into the buffer Gb
// and returns the shift sh: sample n sits at Gb[n - gb + sh], so the caller reads Gb + sh as "G
// from gb".  With only dL/dh given, the range is moved down to a 16-byte boundary of the row
// (sh = 0..3 floats) and copied as whole 16-byte vectors by asynchronous copies (committed as one
// group); a vector that straddles the channel's ends goes as four 4-byte copies, the samples
// outside [0, L_b) zero-filled.  Otherwise (an early-RIR gradient to mask and add) the values are
// formed synchronously, sh = 0.  The buffer holds gl + 6 floats at most.
__device__ __forceinline__ int stage_g(float* Gb, const float* grad_rir, const float* grad_early, int64_t ch0, int gb,
                                       int gl, int Lb, int elo, int ehi, int lane)
{
    if (grad_rir && !grad_early) {
        const float* row = grad_rir + ch0;
        const int sh = (int)((reinterpret_cast<uintptr_t>(row + gb) >> 2) & 3);
        const int g0 = gb - sh;                    // row + g0 is 16-byte aligned
        const int nvec = (gl + sh + 3) >> 2;
        for (int v = lane; v < nvec; v += 32) {
            const int n = g0 + 4 * v;
            if (n >= 0 && n + 3 < Lb) {
                cp_async16(Gb + 4 * v, row + n);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool ok = n + i >= 0 && n + i < Lb;
                    cp_async4(Gb + 4 * v + i, ok ? row + n + i : row, ok);
                }
            }
        }
        cp_async_commit();
        return sh;
    }
    for (int j = lane; j < gl; j += 32) {
        const int n = gb + j;
        float Gv = 0.f;
        if (n >= 0 && n < Lb) {
            if (grad_rir) Gv = grad_rir[ch0 + n];
            if (grad_early && n >= elo && n <= ehi) Gv += grad_early[ch0 + n];
        }
        Gb[j] = Gv;
    }
    return 0;
}

template <int KT>
__global__ void __launch_bounds__(kBwdThreads, 4) bwd_kernel(LaunchArgs a, const float* __restrict__ grad_rir,
                                                             const float* __restrict__ grad_early,
                                                             float* __restrict__ grad_vs, float* __restrict__ grad_g)
{
    extern __shared__ __align__(16) float bwd_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int T = a.tile, K = a.K, M = a.M, Mg = a.margin_i;
    const int span = bwd_span(T);
    const int glen = bwd_glen(T, K, Mg);
    const int tabf = (KT == 0) ? bwd_tab_floats(K) : 0;
    float2* tab = reinterpret_cast<float2*>(bwd_smem);
    const bool with_g = grad_g != nullptr;
    float* Gbuf = bwd_smem + tabf + wid * bwd_warp_floats(T, K, Mg, with_g);
    float* gv = Gbuf + 2 * glen;
    float* gq = gv + kBwdChunks * 96;      // dL/dA A per image (only with grad_g)
    if (KT == 0) {
        for (int j = threadIdx.x; j < 2 * K; j += blockDim.x) {
            float sn, cs;
            sincospif((float)(j - K) / (float)K, &sn, &cs);
            tab[j] = make_float2(cs, sn);
        }
        __syncthreads();
    }
    const float invK = 1.0f / (float)K;
    const bool exact_trig = K < 2;
    float sK, cK;
    sincospif(invK, &sK, &cK);
    const float qf = a.q;
    const int n_items = a.hdr->n_items;
    int qt = 0;
    if (lane == 0) qt = atomicAdd(&a.hdr->queue_bwd, 1);
    qt = __shfl_sync(0xffffffffu, qt, 0);
    while (qt < n_items) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&a.hdr->queue_bwd, 1);
        const int qi = a.order[qt];           // heaviest items first; partials stay per item
        const int2 it = a.items[qi];
        const int b = it.x, s = it.y >> 16, tau = it.y & 0xffff;
        const RoomConst rc = a.room[b];
        const int Lb = rc.len;
        const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
        const int* bo = a.bin_off + ((int64_t)b * a.S + s) * (a.max_tiles + 1);
        const int o_lo = bo[tau], o_hi = bo[tau + 1];
        const bool own_direct = a.src_tile[(int64_t)b * a.S + s] == tau;
        const int64_t chan0 = rc.rir_off + (int64_t)s * M * Lb;
        const DirectConst* dcs = a.direct + ((int64_t)b * a.S + s) * M;
        float rpart = 0.f, dsx = 0.f, dsy = 0.f, dsz = 0.f;
        float* pmic = a.part_mic + (int64_t)qi * 3 * M;
        if (o_hi <= o_lo && !own_direct) {     // nothing owned: zero partials, no staging
            for (int k = lane; k < 3 * M; k += 32) pmic[k] = 0.f;
        } else {
            // Passes over the images; then, if some mic's direct path fell outside every pass's
            // staged span, one pass around the direct path alone.
            const uint64_t dall = (M >= 64) ? ~0ull : ((1ull << M) - 1ull);
            uint64_t dmask = own_direct ? 0ull : dall;   // lane 0: mics whose direct path is added
            const int kd = (int)floorf(dcs[0].t_hi);
            const BwdPass Pdir{o_hi, o_hi, kd - K - 2 * Mg - 2, 2 * K + 4 * Mg + 8};
            bool direct_only = o_hi <= o_lo;
            BwdPass P = direct_only ? Pdir : next_pass(a, v0, o_lo, o_hi, span, K, Mg, lane);
            int stage = 0;
            __syncwarp();
            int sh_next = stage_g(Gbuf, grad_rir, grad_early, chan0, P.gb, P.gl, Lb, dcs[0].early_lo, dcs[0].early_hi,
                                  lane);
            for (bool first = true;; first = false) {
                const int nch = (P.p1 - P.p0 + 31) / 32;
                for (int k = 0; k < nch * 3; ++k) gv[k * 32 + lane] = 0.f;
                if (with_g)
                    for (int k = 0; k < nch; ++k) gq[k * 32 + lane] = 0.f;
                BwdPass Pn = P;
                bool more = false, next_direct_only = false;
                for (int m = 0; m < M; ++m, ++stage) {
                    float* Gs = Gbuf + (stage & 1) * glen + sh_next;
                    cp_async_wait_all();
                    __syncwarp();
                    // Prefetch the next stage: mic m + 1 of this pass, or mic 0 of the next pass.
                    int mn = m + 1;
                    if (m + 1 == M) {
                        mn = 0;
                        if (!direct_only && P.p1 < o_hi) {
                            Pn = next_pass(a, v0, P.p1, o_hi, span, K, Mg, lane);
                            more = true;
                        }
                    }
                    if (m + 1 < M || more)
                        sh_next = stage_g(Gbuf + ((stage + 1) & 1) * glen, grad_rir, grad_early,
                                          chan0 + (int64_t)mn * Lb, Pn.gb, Pn.gl, Lb, dcs[mn].early_lo,
                                          dcs[mn].early_hi, lane);
                    const float* pm = a.mic + 3 * ((size_t)b * M + m);
                    const float mx = pm[0], my = pm[1], mz = pm[2];
                    float mpx = 0.f, mpy = 0.f, mpz = 0.f;
                    // Chunks of images (one per lane), then one round for the direct path of
                    // (b, s, m) on lane 0, owned by one tile and added in the first pass whose
                    // staged span covers its taps.  One call site of the tap loop serves both.
                    const bool want_direct = lane == 0 && !((dmask >> m) & 1ull);
                    const int nround = nch + (__any_sync(0xffffffffu, want_direct) ? 1 : 0);
                    // Round ch: its arrival, ready for the tap gather (go), or nothing to gather.
                    auto setup = [&](int ch) {
                        BwdRound R;
                        R.go = false;
                        R.is_dir = ch == nch;
                        R.j0 = 0;
                        R.A = R.invD = R.ex = R.ey = R.ez = R.gg = 0.f;
                        if (ch >= nround) return R;
                        bool act;
                        int nc = 0;
                        float delta = 0.f;
                        if (!R.is_dir) {
                            const int slot = P.p0 + 32 * ch + lane;
                            act = slot < P.p1;
                            if (act) {
                                const float4 pa = a.spa[v0 + slot];
                                const float2 pb = a.spb[v0 + slot];
                                R.gg = a.samp[v0 + slot];
                                float D, ux, uy, uz;
                                image_geom(pa, pb, mx, my, mz, a.q2, nc, delta, D, ux, uy, uz);
                                R.invD = rcp_approx(D);
                                R.A = exp2f(R.gg * rc.log2r) * R.invD;
                                R.ex = ux * R.invD; R.ey = uy * R.invD; R.ez = uz * R.invD;
                                act = D > 0.0f;
                            }
                        } else {
                            act = want_direct;
                            if (act) {
                                const DirectConst dc = dcs[m];
                                nc = __float2int_rn(dc.t_hi);
                                delta = __fadd_rn(__fsub_rn(dc.t_hi, (float)nc), dc.t_lo);
                                R.A = dc.amp;
                                R.invD = dc.amp;
                                R.ex = dc.ex; R.ey = dc.ey; R.ez = dc.ez;
                            }
                        }
                        if (act && (nc + K < 0 || nc - K >= Lb)) {      // no tap inside the RIR
                            act = false;
                            if (R.is_dir) dmask |= 1ull << m;
                        }
                        if (act) {
                            const ArrB r = arrival_bwd(nc, delta, invK, exact_trig, cK, sK);
                            const int j0 = nc - K - P.gb;
                            if (j0 >= 0 && j0 + 2 * K <= P.gl) {
                                R.go = true;
                                R.j0 = j0;
                                R.r = r;
                            } else if (!R.is_dir || direct_only) {
                                atomicOr(&a.hdr->status, FRAM_DEV_CAPACITY);
                                if (R.is_dir) dmask |= 1ull << m;
                            }
                        }
                        return R;
                    };
                    // The chain rule of round ch from its tap sums.
                    auto finish = [&](const BwdRound& R, int ch, float S1, float S2) {
                        const float A = R.A;
                        const float dLdD = __fmaf_rn(A * S2, qf, -S1 * A * R.invD);
                        mpx = __fmaf_rn(-dLdD, R.ex, mpx);
                        mpy = __fmaf_rn(-dLdD, R.ey, mpy);
                        mpz = __fmaf_rn(-dLdD, R.ez, mpz);
                        if (!R.is_dir) {
                            float* g3 = gv + ch * 96 + lane;
                            g3[0] = __fmaf_rn(dLdD, R.ex, g3[0]);
                            g3[32] = __fmaf_rn(dLdD, R.ey, g3[32]);
                            g3[64] = __fmaf_rn(dLdD, R.ez, g3[64]);
                            rpart = __fmaf_rn(S1 * A * R.gg, rc.inv_r, rpart);
                            if (with_g) gq[ch * 32 + lane] = __fmaf_rn(S1, A, gq[ch * 32 + lane]);
                        } else {
                            dsx = __fmaf_rn(dLdD, R.ex, dsx);
                            dsy = __fmaf_rn(dLdD, R.ey, dsy);
                            dsz = __fmaf_rn(dLdD, R.ez, dsz);
                            dmask |= 1ull << m;
                        }
                    };
                    for (int ch = 0; ch < nround; ++ch) {
                        const BwdRound R = setup(ch);
                        if (R.go && FRAM_GUARD(a.hdr, R.j0 >= 0 &&
                                                          (int)(Gs - (Gbuf + (stage & 1) * glen)) + R.j0 + 2 * K < glen)) {
                            float S1, S2;
                            if constexpr (KT > 0) gather_taps_ct<KT>(Gs + R.j0, R.r, S1, S2);
                            else gather_taps_rt(Gs + R.j0, K, R.r, tab, S1, S2);
                            finish(R, ch, S1, S2);
                        }
                    }
                    mpx = warp_sum(mpx); mpy = warp_sum(mpy); mpz = warp_sum(mpz);
                    if (lane == 0) {
                        float* pw = pmic + 3 * m;
                        if (first) { pw[0] = mpx; pw[1] = mpy; pw[2] = mpz; }
                        else { pw[0] += mpx; pw[1] += mpy; pw[2] += mpz; }
                    }
                    if (m + 1 == M && !more && !direct_only) {
                        // All image passes done: a direct-only pass if a direct path is missing.
                        const uint64_t dm = __shfl_sync(0xffffffffu, dmask, 0);
                        if (dm != dall) {
                            Pn = Pdir;
                            more = true;
                            next_direct_only = true;
                            sh_next = stage_g(Gbuf + ((stage + 1) & 1) * glen, grad_rir, grad_early, chan0, Pn.gb,
                                              Pn.gl, Lb, dcs[0].early_lo, dcs[0].early_hi, lane);
                        }
                    }
                }
                __syncwarp();
                if (grad_vs || with_g) {
                    const float lnr = rc.log2r * 0.69314718055994531f;   // dA/dg = A ln r
                    for (int ch = 0; ch < nch; ++ch) {
                        const int slot = P.p0 + 32 * ch + lane;
                        const int64_t v = slot < P.p1 ? v0 + a.perm[v0 + slot] : -1;
                        if (slot < P.p1 && FRAM_GUARD(a.hdr, v >= v0 && v < v0 + rc.n_vs && v < a.n_vs_total)) {
                            const float* g3 = gv + ch * 96 + lane;
                            if (grad_vs) {
                                grad_vs[3 * v] = g3[0];
                                grad_vs[3 * v + 1] = g3[32];
                                grad_vs[3 * v + 2] = g3[64];
                            }
                            if (with_g) grad_g[v] = gq[ch * 32 + lane] * lnr;
                        }
                    }
                }
                __syncwarp();
                if (!more) break;
                P = Pn;
                direct_only = direct_only || next_direct_only;
            }
            cp_async_wait_all();
        }
        rpart = warp_sum(rpart);
        if (lane == 0) {
            a.part_r[qi] = rpart;
            a.part_src[3 * (int64_t)qi] = dsx;
            a.part_src[3 * (int64_t)qi + 1] = dsy;
            a.part_src[3 * (int64_t)qi + 2] = dsz;
        }
        qt = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

// The adjoint's work order: items by decreasing cost (owned images), so the last items a
// persistent warp takes are short ones.  One CTA: histogram of cost buckets, exclusive scan from
// the heaviest bucket down, scatter.  The order only decides which warp takes which item when;
// every item writes its own partials, reduced later in item order, so results do not depend on it.
constexpr int kOrderBuckets = 1024;

__global__ void __launch_bounds__(1024) bwd_order(LaunchArgs a)
{
    __shared__ int cnt[kOrderBuckets];
    __shared__ int warp_tot[32];
    const int n = a.hdr->n_items;
    for (int k = threadIdx.x; k < kOrderBuckets; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    auto bucket = [&](int qi) {
        const int2 it = a.items[qi];
        const int b = it.x, s = it.y >> 16, tau = it.y & 0xffff;
        const int* bo = a.bin_off + ((int64_t)b * a.S + s) * (a.max_tiles + 1);
        const int cost = bo[tau + 1] - bo[tau];
        return kOrderBuckets - 1 - min(cost >> 3, kOrderBuckets - 1);   // heavy -> low bucket
    };
    for (int qi = threadIdx.x; qi < n; qi += blockDim.x) atomicAdd(&cnt[bucket(qi)], 1);
    __syncthreads();
    // exclusive scan of cnt (one value per thread: blockDim == kOrderBuckets)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = cnt[threadIdx.x];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < 32; ++k) { const int t = warp_tot[k]; warp_tot[k] = run; run += t; }
    }
    __syncthreads();
    cnt[threadIdx.x] = warp_tot[w] + x - v;
    __syncthreads();
    for (int qi = threadIdx.x; qi < n; qi += blockDim.x) a.order[atomicAdd(&cnt[bucket(qi)], 1)] = qi;
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
cudaError_t launch_bwd_t(const LaunchArgs& a, const float* grad_rir, const float* grad_early, float* grad_vs,
                         float* grad_g, cudaStream_t st)
{
    const int smem = (int)sizeof(float) * ((KT == 0 ? bwd_tab_floats(a.K) : 0) +
                                           (kBwdThreads / 32) * bwd_warp_floats(a.tile, a.K, a.margin_i,
                                                                                grad_g != nullptr));
    int per_sm = 0;
    cudaError_t e = kernel_residency((const void*)bwd_kernel<KT>, kBwdThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    bwd_kernel<KT><<<device_sm_count() * per_sm, kBwdThreads, smem, st>>>(a, grad_rir, grad_early, grad_vs, grad_g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_backward(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                            const float* r, const float* grad_rir, const float* grad_early, float* grad_vs,
                            float* grad_mic, float* grad_src, float* grad_r, float* grad_g, cudaStream_t st)
{
    (void)r;
    (void)pos_hi;
    (void)pos_lo;   // the kernel reads the sorted copies the preparation made
    if (a.M > 64) return cudaErrorInvalidValue;   // direct-path bookkeeping is a 64-bit mask
    cudaError_t e;
    const int64_t segs = (int64_t)a.B * a.S;
    if (segs > 0) {
        g_gather<<<(unsigned)segs, 256, 0, st>>>(a, g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    bwd_order<<<1, kOrderBuckets, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.K == 40) e = launch_bwd_t<40>(a, grad_rir, grad_early, grad_vs, grad_g, st);
    else if (a.K == 63) e = launch_bwd_t<63>(a, grad_rir, grad_early, grad_vs, grad_g, st);
    else e = launch_bwd_t<0>(a, grad_rir, grad_early, grad_vs, grad_g, st);
    if (e != cudaSuccess) return e;
    const int64_t n = std::max<int64_t>({(int64_t)a.B * a.M * 3, (int64_t)a.B * a.S * 3, (int64_t)a.B});
    if (n > 0 && (grad_mic || grad_src || grad_r)) {
        bwd_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, grad_mic, grad_src, grad_r);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace fram
