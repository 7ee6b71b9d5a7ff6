// fram_internal.cuh -- shared device helpers and workspace layout of libfram (sm_103a).
//
// Contents:
//   * float-pair ("double-float") arithmetic built from error-free transformations
//     (Knuth's TwoSum, Dekker's FastTwoSum, FMA-based TwoProd).  GB300's FP64 units run at a
//     small fraction of its FP32 rate, so the few places that need more than 24 bits -- image
//     distances of up to c0*T60 ~ 400 m that must place a delay to ~1e-6 samples -- use pairs
//     of floats (about 44 bits) instead of doubles.  All operations use the _rn intrinsics so
//     the compiler cannot contract or reorder them.
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the image sampler.
//   * the workspace layout shared by the sampler, the synthesis and the adjoint.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fram.h"

namespace fram {

// --------------------------------------------------------------------------------------
// Float-pair arithmetic.  A value is hi + lo with |lo| <= ulp(hi)/2 after normalisation.
// --------------------------------------------------------------------------------------
struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ f2 fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ f2 two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ f2 f2_add_f(f2 a, float b)
{
    f2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ f2 f2_mul_f(f2 a, float b)
{
    f2 p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.hi, -a.lo}; }

// --------------------------------------------------------------------------------------
// Packed FP32 pairs (add/mul/fma.rn.f32x2): one instruction performs two independent IEEE
// operations, each half rounded exactly as the scalar operation would be.  A pair lives in one
// 64-bit register pair, low half first.
// --------------------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Hardware approximations (MUFU): relative error about one ulp.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt of a positive pair from an approximate float root: the pair residual a - y^2 is formed
// exactly and one Newton correction y + (a - y^2)/(2y) restores ~44-bit accuracy, so the seed
// and the correction's reciprocal only need float accuracy.
__device__ __forceinline__ f2 f2_sqrt_fast(f2 a)
{
    const float y = sqrt_approx(a.hi);
    const f2 yy = two_prod(y, y);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, yy.hi), yy.lo), a.lo);
    return fast_two_sum(y, __fmul_rn(r, __fmul_rn(0.5f, rcp_approx(y))));
}

// sin(pi x) and cos(pi x) for |x| <= 1/2 (arguments here are fractional delays delta and
// delta / K): Taylor series of sin and cos truncated after x^13 and x^14, whose remainders
// are below 7e-10 and 7e-11 on that interval; Horner evaluation in x^2.
__device__ __forceinline__ float sinpi_poly(float x)
{
    const float x2 = x * x;
    float p = 0.00046630280576761234f;
    p = __fmaf_rn(p, x2, -0.007370430945714348f);
    p = __fmaf_rn(p, x2, 0.08214588661112819f);
    p = __fmaf_rn(p, x2, -0.5992645293207919f);
    p = __fmaf_rn(p, x2, 2.550164039877345f);
    p = __fmaf_rn(p, x2, -5.167712780049969f);
    p = __fmaf_rn(p, x2, 3.141592653589793f);
    return p * x;
}

__device__ __forceinline__ float cospi_poly(float x)
{
    const float x2 = x * x;
    float p = -0.00010463810492484565f;
    p = __fmaf_rn(p, x2, 0.001929574309403922f);
    p = __fmaf_rn(p, x2, -0.02580689139001405f);
    p = __fmaf_rn(p, x2, 0.23533063035889312f);
    p = __fmaf_rn(p, x2, -1.3352627688545893f);
    p = __fmaf_rn(p, x2, 4.058712126416768f);
    p = __fmaf_rn(p, x2, -4.934802200544679f);
    return __fmaf_rn(p, x2, 1.0f);
}

// Host helper: split a double into a float pair.
__host__ __device__ inline f2 f2_from_double(double x)
{
    float hi = (float)x;
    float lo = (float)(x - (double)hi);
    return {hi, lo};
}

// --------------------------------------------------------------------------------------
// Philox4x32-10.  S-box: two 32x32 -> 64-bit products with the published multipliers;
// key schedule: Weyl increments (golden ratio and sqrt(3) - 1 in 0.32 fixed point).
// --------------------------------------------------------------------------------------
struct u4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u4 philox4x32_10(u4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
        const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
        c = u4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// Top 23 bits of a word, centred in their cell: exact float in (0, 1).
__device__ __forceinline__ float uniform_from_word(uint32_t w)
{
    return __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 1.0f / 8388608.0f);
}

// --------------------------------------------------------------------------------------
// Per-launch constants and workspace layout.
// --------------------------------------------------------------------------------------
constexpr int kMaxHalfLen = 128;
constexpr int kDefaultTile = 1024;
constexpr int kMaxTile = 4096;
constexpr int kSynthThreads = 256;

struct RoomConst {          // per room, written by the prologue
    float cx, cy, cz;       // array centre (float)
    float margin;           // max_m |mic_m - c| fs/c0 + 2 samples
    float log2r;            // log2 of the reflection coefficient r_b
    float inv_r;            // 1 / r_b
    int32_t len;            // L_b
    int32_t ntiles;         // ceil(L_b / tile)
    int32_t n_vs;           // images per source
    int32_t item0;          // first work item of the room
    int64_t rir_off;
    int64_t vs_off;
};

struct DirectConst {        // per (room, source, mic)
    float t_hi, t_lo;       // direct-path delay in samples as a float pair
    float amp;              // 1 / D_{0,m}
    float dist;             // D_{0,m}
    float ex, ey, ez;       // (src - mic) / D_{0,m}
    int32_t early_lo;       // Eq. 9 window, inclusive
    int32_t early_hi;
    int32_t q_h;            // multi-rate mode: ceil(D_{0,m} / c0 * r_h fs) (before the clamp)
    int32_t early_lo_h;     // multi-rate mode: Eq. 9 window on the high-rate grid, inclusive
    int32_t early_hi_h;
    int32_t pad_;
};

struct ItemRec {            // per work item (room, source, tile), written by the preparation
    int32_t b, s, T0, len;  // room, source, first sample of the tile, L_b
    int32_t c_lo, c_hi;     // sorted image positions whose key can reach the tile
    int32_t pad0, pad1;
    int64_t v0;             // first image row of (room, source)
    int64_t out0;           // first RIR sample of (room, source, mic 0)
};

struct Header {             // first 256 bytes of the workspace
    int32_t status;         // FRAM_DEV_* bits
    int32_t queue;          // persistent-kernel work counter
    int32_t queue_bwd;
    int32_t n_items;        // total work items (written by the prologue)
    int32_t pad_[60];
};

constexpr int kSampleRec = 256;   // bytes per (room, source) record of the sampler's constants

struct WsLayout {
    size_t header, room, direct, src_tile, item_off, items, order, bin_off, perm, key, skey, sconst;
    size_t spa, spb, pos32, samp, irec;
    size_t mr_y, mr_ye, mr_tab;           // multi-rate mode: intermediate signals, resampling table
    size_t mr_order;                      // multi-rate mode: rooms by decreasing RIR length
    size_t mr_counts, mr_pstate;          // multi-rate mode: rooms per high-pass piece, piece start states
    size_t part_mic, part_src, part_r, sb_part;
    size_t total;
    int tile;
    int max_tiles;          // ceil(max_len / tile)
    int nb32;               // 32-sample key blocks per (room, source), independent of the tile
    int64_t max_items;      // B * S * max_tiles
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Multi-rate mode rates: r_h = floor(1e6 / fs), r_l = floor(sqrt(r_h)); the first resampling
// ratio up/down = r_l/r_h reduced.
struct MrRates {
    int rh, rl, up, down;
};

inline MrRates mr_rates(double fs)
{
    MrRates r;
    r.rh = (int)floor(1.0e6 / fs);
    r.rl = (int)floor(sqrt((double)r.rh));
    int a = r.rh, b = r.rl;
    while (b) { const int t = a % b; a = b; b = t; }
    r.up = r.rl / a;
    r.down = r.rh / a;
    return r;
}

// Multi-rate mode: the high-pass and the second resampler run fused over pieces of Pn output
// samples.  The thread of piece p starts its recursion kMrHalo groups of r_l intermediate samples
// before the piece's first output, at k_s = r_l (p Pn - kMrHalo) (the resampler's window reaches
// 10 groups back; 12 keeps k_s a multiple of 4 for 16-byte copies), from the state the recursion
// reaches over the W samples before k_s (the pole radius rho of the 80 Hz high-pass at r_l fs gives
// rho^W <= 1e-9 of the state it forgets).  pmax pieces cover the longest RIR.  The recursion is
// latency bound per thread (two dependent fused multiply-adds per sample), so the pieces are short
// enough to give every SM enough independent channels (~16384 intermediate samples splits a
// 16 kHz batch's 0.1-0.7 s channels into 1-5 pieces) and long enough to keep the warm-up reads (W
// of every r_l Pn samples) modest; 8192 to 32768 measured within noise of each other on a
// 1024-room batch, 16384 best on 256 rooms.
constexpr int kMrHalo = 12;

struct MrPieces {
    int Pn, W, pmax;    // output samples per piece (a multiple of 4), warm-up length, pieces
};

inline MrPieces mr_pieces(double fs, int max_len)
{
    const MrRates r = mr_rates(fs);
    const double k = std::tan(3.14159265358979323846 * 80.0 / ((double)r.rl * fs));
    const double a2 = (1.0 - std::sqrt(2.0) * k + k * k) / (1.0 + std::sqrt(2.0) * k + k * k);
    const double rho = std::sqrt(a2);
    MrPieces pc;
    pc.W = ((int)std::ceil(std::log(1e-9) / std::log(rho)) + 63) & ~63;
    const int P = std::max(16384, 2 * pc.W);
    pc.Pn = ((P + r.rl - 1) / r.rl + 3) & ~3;
    pc.pmax = (int)(((int64_t)(max_len > 0 ? max_len : 1) + pc.Pn - 1) / pc.Pn);
    return pc;
}

inline WsLayout ws_layout(const fram_scene& sc, int tile, int delay_mode = 0, double fs = 16000.0)
{
    WsLayout w{};
    w.tile = tile;
    w.max_tiles = sc.max_len > 0 ? (sc.max_len + tile - 1) / tile : 1;
    w.max_items = (int64_t)sc.B * sc.S * w.max_tiles;
    w.nb32 = (sc.max_len > 0 ? (sc.max_len + 31) / 32 : 0) + 2 * kMaxTile / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    w.header = take(sizeof(Header));
    w.room = take(sizeof(RoomConst) * (size_t)sc.B);
    w.direct = take(sizeof(DirectConst) * (size_t)sc.B * sc.S * sc.M);
    w.src_tile = take(sizeof(int32_t) * (size_t)sc.B * sc.S);
    w.item_off = take(sizeof(int32_t) * ((size_t)sc.B + 1));
    w.items = take(sizeof(int32_t) * 2 * (size_t)w.max_items);
    w.order = take(sizeof(int32_t) * (size_t)w.max_items);
    w.bin_off = take(sizeof(int32_t) * (size_t)sc.B * sc.S * (w.max_tiles + 1));
    w.perm = take(sizeof(int32_t) * (size_t)sc.n_vs_total);
    w.key = take(sizeof(float) * (size_t)sc.n_vs_total);
    w.skey = take(sizeof(int32_t) * (size_t)sc.n_vs_total);
    w.spa = take(sizeof(float) * 4 * (size_t)sc.n_vs_total);
    w.spb = take(sizeof(float) * 2 * (size_t)sc.n_vs_total);
    w.pos32 = take(sizeof(int32_t) * (size_t)sc.B * sc.S * ((size_t)w.nb32 + 1));
    w.samp = take(sizeof(float) * (size_t)sc.n_vs_total);
    w.irec = take(sizeof(ItemRec) * (size_t)w.max_items);
    w.sconst = take((size_t)kSampleRec * sc.B * sc.S);
    if (delay_mode == 1) {
        // per channel (room, source, mic): r_l L_b + 8 intermediate samples, and the same for
        // the early RIR; the polyphase table is down x 32 floats.
        const MrRates mr = mr_rates(fs);
        const size_t inter = (size_t)mr.rl * (size_t)sc.rir_total + 8 * (size_t)sc.B * sc.S * sc.M + 4;
        w.mr_y = take(sizeof(float) * inter);
        w.mr_ye = take(sizeof(float) * inter);
        w.mr_tab = take(sizeof(float) * 32 * (size_t)mr.down);
        w.mr_order = take(sizeof(int32_t) * ((size_t)sc.B + 1));
        const MrPieces pc = mr_pieces(fs, sc.max_len);
        w.mr_counts = take(sizeof(int32_t) * ((size_t)pc.pmax + 1));
        w.mr_pstate = take(32 * (size_t)pc.pmax * 2 * (size_t)sc.B * sc.S * sc.M);
    }
    w.part_mic = take(sizeof(float) * 3 * (size_t)w.max_items * sc.M);
    w.part_src = take(sizeof(float) * 3 * (size_t)w.max_items);
    w.part_r = take(sizeof(float) * (size_t)w.max_items);
    w.sb_part = take(sizeof(double) * 5 * (size_t)sc.B * sc.S);
    w.total = off;
    return w;
}

// Device view of the scene + parameters for kernels (by value in kernel arguments).
struct LaunchArgs {
    double fs, c0;
    int32_t B, S, M;
    int32_t K;
    int32_t tile;
    int32_t max_tiles;
    int32_t nb32;           // last index of a (room, source) row of pos32
    float q;                // fs / c0 as a float
    f2 q2;                  // fs / c0 as a float pair
    int32_t early_pre, early_post;
    int32_t margin_i;       // ceil(array_radius fs/c0) + 3: halo of the adjoint's staged gradient
    int64_t n_vs_total;     // host sizes, used to bound every device index
    int64_t rir_total;
    uint32_t room_base;     // Philox room word of room 0 (the room's index in a larger batch)
    const float* dims;
    const float* rt60;
    const float* src;
    const float* mic;
    const int32_t* n_vs;
    const int64_t* vs_off;
    const int32_t* rir_len;
    const int64_t* rir_off;
    // workspace views
    Header* hdr;
    RoomConst* room;
    DirectConst* direct;
    int32_t* src_tile;
    int32_t* item_off;
    int2* items;
    int32_t* order;         // adjoint work order: item indices by decreasing cost
    int32_t* bin_off;
    int32_t* perm;          // per (room, source): image indices sorted by 32-sample key block
    float* key;             // per image: delay to the array centre in samples (binning key)
    int32_t* skey;          // per sorted position: first sample of the image's key block
    float4* spa;            // per sorted position: image position hi (x, y, z) and lo x
    float2* spb;            // per sorted position: image position lo (y, z)
    int32_t* pos32;         // per (room, source) and 32-sample block j: first sorted position
                            // whose key is >= 32 j (rows of nb32 + 1 entries)
    float* samp;            // per sorted position: r^g of the image (written per synthesis)
    ItemRec* irec;          // per work item
    char* sconst;           // per (room, source): the sampler's constants (kSampleRec bytes each)
    // multi-rate mode (delay_mode 1)
    int32_t mode;
    int32_t rh, rl, up, down, HLA;   // rates, first resampling ratio, its filter's half length
    double fh;                       // r_h fs
    double early_pre_ms, early_post_ms;
    float* mr_y;                     // intermediate signals at r_l fs, per channel
    float* mr_ye;                    // the same for the early RIR
    float* mr_tab;                   // first resampling filter, polyphase rows of 32
    int32_t* mr_order;               // rooms by decreasing RIR length (ties by index)
    int32_t* mr_counts;              // rooms with more than p high-pass pieces, per p
    void* mr_pstate;                 // high-pass piece start states
    int32_t max_len;                 // max_b L_b
    float* part_mic;
    float* part_src;
    float* part_r;
    double* sb_part;        // gradient through the sampler: per (room, source) partial sums
};

// Bounds guards of the debug build (compiled with -DFRAM_DEBUG_BOUNDS): a guarded access runs only
// if its index lies inside its buffer; otherwise FRAM_DEV_BOUNDS is set in the status word and the
// access is skipped (no trap).  In the release build every guard is the constant true, so it
// leaves no code.
#ifdef FRAM_DEBUG_BOUNDS
__device__ __forceinline__ bool fram_guard(Header* h, bool ok)
{
    if (!ok) atomicOr(&h->status, FRAM_DEV_BOUNDS);
    return ok;
}
#define FRAM_GUARD(hdr, cond) ::fram::fram_guard((hdr), (cond))
#else
#define FRAM_GUARD(hdr, cond) true
#endif

// Host-side launchers (defined in the .cu files; return cudaError_t of the launch).
cudaError_t launch_sample(const LaunchArgs& a, const fram_params& p, uint64_t seed, const uint64_t* d_seed,
                          float* pos_hi, float* pos_lo, float* g, float* r, uint32_t* words, cudaStream_t st);
cudaError_t launch_prepare(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* r,
                           cudaStream_t st);
cudaError_t launch_synthesize(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                              float* rir, float* early, cudaStream_t st);
cudaError_t launch_amp_gather(const LaunchArgs& a, const float* g, cudaStream_t st);
cudaError_t launch_sample_backward(const LaunchArgs& a, const fram_params& p, uint64_t seed, const uint64_t* d_seed,
                                   const float* grad_vs, const float* grad_g, const float* grad_r,
                                   const float* grad_src_dir, const float* grad_mic_dir, float* grad_src,
                                   float* grad_mic, float* grad_t60, float* grad_dims, double* part, cudaStream_t st);
cudaError_t launch_synthesize_mr(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, float* rir,
                                 float* early, cudaStream_t st);
cudaError_t launch_backward(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                            const float* r, const float* grad_rir, const float* grad_early, float* grad_vs,
                            float* grad_mic, float* grad_src, float* grad_r, float* grad_g, cudaStream_t st);

int device_sm_count();
int record_error(int code, const char* msg);   // sets fram_last_error's text, returns code

// Workspace bytes that a call with these parameters uses at the tile it actually launches with
// (p->tile, or the autotuned / default tile when p->tile is 0); fram_workspace_size instead
// sizes for every tile.  Checks the parameters and the scene like fram_workspace_size.
int workspace_bytes_at_launch_tile(const fram_scene* scene, const fram_params* p, size_t* bytes);

// Dynamic shared memory of one synthesis CTA for tile length T.
int synth_smem_total(int T);

// Raises the kernel's dynamic shared-memory limit to `smem` (once per device and size) and
// returns how many CTAs of `threads` threads fit on one SM.  Results are cached, so after the
// first call with a configuration no CUDA API call other than the launch itself is made --
// which keeps the entry points capturable in a CUDA graph.
cudaError_t kernel_residency(const void* func, int threads, int smem, int* per_sm);

}  // namespace fram
