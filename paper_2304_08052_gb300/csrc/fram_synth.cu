// fram_synth.cu -- prologue, delay binning and the forward synthesis kernel (FRAM-RIR
// Eq. 1 with fractional-delay Hann-windowed sincs at the output rate, Sec. III-D, Eq. 9).
//
// Pipeline of fram_synthesize (all on the caller's stream, no host synchronisation):
//   1. room_prologue   one thread per room and per (room, source, mic): RIR length, tile count,
//                      array centre, binning margin, log2 r, and the direct path of every
//                      (source, mic) pair in FP64 (delay split into a float pair, amplitude
//                      1/D, Eq. 9 window).
//   2. item_scan       one CTA: prefix sum of S * ntiles_b over the rooms (each room's first
//                      work item).
//   3. bin_images      one CTA per (room, source): each image's delay to the array centre
//                      (the binning key, in samples), a stable counting sort of the images by
//                      32-sample key block and the first sorted position of every block.
//                      Per-mic delays differ from the key by at most the array radius in
//                      samples ("margin").  sort_positions copies the positions into that
//                      order; item_ranges finds each work item's (room, source, tile) by binary
//                      search over the rooms' first items and writes the item table and the
//                      per-item records.
//   4. synth_kernel    persistent warps pull (room, source, tile, mic) units from a counter.
//                      Per unit the warp owns a private tile buffer in shared memory, computes
//                      the arrival (delay t = D fs/c0 from a float-pair distance, amplitude,
//                      sinc constants) of every image whose key lies within K + margin of the
//                      tile, and adds each arrival's 2K+1 taps with one lane per tap offset.
//
// Tap arithmetic.  With t = n_c + delta (n_c = nearest integer) and the tap at n = n_c + o,
// sin(pi (n - t)) = (-1)^o sin(-pi delta), so for |n - t| < K
//   A sinc(n - t) w(n - t) = (-1)^o [P + a cos(pi o/K) + b sin(pi o/K)] / (delta - o)
// with per-arrival constants P = A sin(pi delta) / (2 pi), a = P cos(pi delta/K),
// b = P sin(pi delta/K) (angle-difference form of the Hann term (1 + cos(pi (n - t)/K)) / 2).
// The o-dependent factors are per-lane constants, so a tap costs one FMA for the denominator,
// two for the numerator, one reciprocal and one FMA into the buffer.  No atomics touch the
// accumulators: a buffer belongs to one warp, whose lanes hit distinct samples in every step,
// and each sample sums its arrivals in the fixed sorted image order.
#include <cmath>

#include "fram_internal.cuh"

namespace fram {
namespace {

constexpr float kTwoPiInv = 0.15915494309189535f;   // 1 / (2 pi)
constexpr float kTinyDelta = 9.313225746154785e-10f; // 2^-30: keeps d != 0 at n = n_c

__global__ void room_prologue(LaunchArgs a, const float* __restrict__ r_in)
{
    const double fs = a.fs, c0 = a.c0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nbsm = (int64_t)a.B * a.S * a.M;
    if (tid < a.B) {
        const int b = (int)tid;
        RoomConst rc;
        double cx = 0, cy = 0, cz = 0;
        for (int m = 0; m < a.M; ++m) {
            const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
            cx += pm[0]; cy += pm[1]; cz += pm[2];
        }
        cx /= a.M; cy /= a.M; cz /= a.M;
        double rad = 0;
        for (int m = 0; m < a.M; ++m) {
            const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
            const double dx = pm[0] - cx, dy = pm[1] - cy, dz = pm[2] - cz;
            rad = fmax(rad, sqrt(dx * dx + dy * dy + dz * dz));
        }
        rc.cx = (float)cx; rc.cy = (float)cy; rc.cz = (float)cz;
        rc.margin = (float)(rad * fs / c0 + 2.0);
        const double r = r_in ? (double)r_in[b] : 0.5;
        const bool rok = (r > 0) && (r < 1) && isfinite(r);
        if (r_in && !rok) atomicOr(&a.hdr->status, FRAM_DEV_NONFINITE);
        rc.log2r = rok ? (float)log2(r) : 0.0f;
        rc.inv_r = rok ? (float)(1.0 / r) : 0.0f;
        rc.len = a.rir_len[b];
        rc.n_vs = a.n_vs[b];
        rc.item0 = 0;
        rc.rir_off = a.rir_off[b];
        rc.vs_off = a.vs_off[b];
        // Device arrays that disagree with the host sizes would index past the buffers: such
        // a room gets no work and the geometry bit is raised.
        bool bad = false;
        if (rc.len < 1 || rc.rir_off < 0 || rc.rir_off + (int64_t)a.S * a.M * rc.len > a.rir_total) {
            rc.len = 0;
            bad = true;
        }
        rc.ntiles = rc.len > 0 ? (rc.len + a.tile - 1) / a.tile : 0;
        if (rc.ntiles > a.max_tiles) { rc.ntiles = 0; rc.len = 0; bad = true; }
        if (rc.n_vs < 0 || rc.vs_off < 0 || rc.vs_off + (int64_t)a.S * rc.n_vs > a.n_vs_total) {
            rc.n_vs = 0;
            bad = true;
        }
        if (bad) atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
        a.room[b] = rc;
        a.item_off[b] = a.S * rc.ntiles;   // counts; item_scan turns them into offsets
        const double q = fs / c0;
        for (int s = 0; s < a.S; ++s) {
            const float* ps = a.src + 3 * ((size_t)b * a.S + s);
            const double dx = ps[0] - (double)rc.cx, dy = ps[1] - (double)rc.cy, dz = ps[2] - (double)rc.cz;
            const double key0 = sqrt(dx * dx + dy * dy + dz * dz) * q;
            int t = (int)floor(key0 / a.tile);
            t = t < 0 ? 0 : (t > rc.ntiles - 1 ? rc.ntiles - 1 : t);
            a.src_tile[(size_t)b * a.S + s] = t;
        }
    }
    if (tid < nbsm) {
        const int m = (int)(tid % a.M);
        const int s = (int)((tid / a.M) % a.S);
        const int b = (int)(tid / ((int64_t)a.M * a.S));
        const float* ps = a.src + 3 * ((size_t)b * a.S + s);
        const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
        const double dx = (double)ps[0] - pm[0], dy = (double)ps[1] - pm[1], dz = (double)ps[2] - pm[2];
        const double D = sqrt(dx * dx + dy * dy + dz * dz);
        DirectConst dc;
        const double t = D * fs / c0;
        const f2 tp = f2_from_double(t);
        dc.t_hi = tp.hi; dc.t_lo = tp.lo;
        dc.amp = (float)(1.0 / D);
        dc.dist = (float)D;
        dc.ex = (float)(dx / D); dc.ey = (float)(dy / D); dc.ez = (float)(dz / D);
        const double n0 = ceil(t);
        dc.early_lo = (int)(n0 - a.early_pre);
        dc.early_hi = (int)(n0 + a.early_post);
        dc.q_h = dc.early_lo_h = dc.early_hi_h = 0;
        if (a.mode == 1) {
            // The high-rate grid decides integers: evaluated in the oracle's order, with
            // separately rounded products and sums (no fused multiply-add).
            const double Dr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            const double qh = ceil(__dmul_rn(__ddiv_rn(Dr, c0), a.fh));
            dc.q_h = (int)fmin(qh, 2.0e9);
            dc.early_lo_h = (int)fmax(qh - ceil(__ddiv_rn(__dmul_rn(a.early_pre_ms, a.fh), 1000.0)), -2.0e9);
            dc.early_hi_h = (int)fmin(qh + ceil(__ddiv_rn(__dmul_rn(a.early_post_ms, a.fh), 1000.0)), 2.0e9);
        }
        dc.pad_ = 0;
        if (!(D > 0) || !isfinite(D)) atomicOr(&a.hdr->status, FRAM_DEV_BAD_GEOMETRY);
        a.direct[tid] = dc;
    }
}

// Single CTA: item_off[b] = sum_{b' < b} S ntiles_b', item table, total in the header.
__global__ void __launch_bounds__(1024) item_scan(LaunchArgs a)
{
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < a.B; base += blockDim.x) {
        const int b = base + threadIdx.x;
        const int v = b < a.B ? a.item_off[b] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        const int excl = carry + (wid > 0 ? warp_sum[wid - 1] : 0) + x - v;
        if (b < a.B) {
            a.item_off[b] = excl;
            a.room[b].item0 = excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.item_off[a.B] = carry;
        a.hdr->n_items = carry;
    }
}

// One warp per (room, source): binning keys and a stable counting sort of the images by 32-sample
// key block (ties by image index).  The result: perm (image indices in sorted order), skey (the
// first sample of each sorted image's block), p32 (the first sorted position of every block) and
// bin_off (the first sorted position of every tile; the last tile also owns every image keyed
// beyond the RIR).  Any delay range of a source's images is then one contiguous run.
__device__ __forceinline__ int block_of_key(float key, int nb)
{
    if (!(key < 3.0e9f)) return nb - 1;               // NaN or beyond any RIR: last block
    const int j = (int)floorf(key) >> 5;
    return j < 0 ? 0 : (j > nb - 1 ? nb - 1 : j);
}

// One CTA of W warps per (room, source).  Warp w owns the contiguous index range
// [w chunk, (w + 1) chunk) of the images and its own histogram row hist[w][0..NB); the exclusive
// offsets are taken in (block, warp) order, so every warp's scatter lands exactly where a single
// pass in index order would put it (the sort stays stable).  Shared memory: (W + 1) x (NB + 1)
// ints (the last row holds the block prefix) and 33 ints of scan scratch.
__host__ __device__ inline int bin_smem_ints(int W, int NB) { return (W + 1) * (NB + 1) + 33; }

__global__ void __launch_bounds__(256) bin_images(LaunchArgs a, const float* __restrict__ pos_hi)
{
    extern __shared__ int bin_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int64_t seg = blockIdx.x;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    const int T = a.tile, NB = a.nb32;
    const int n = rc.n_vs, nt = rc.ntiles;
    const int64_t v0 = rc.vs_off + (int64_t)s * n;
    int* bo = a.bin_off + seg * (a.max_tiles + 1);
    int* p32 = a.pos32 + seg * ((int64_t)NB + 1);
    if (nt < 1) {   // a room the prologue rejected: no work items reference its bins
        if (threadIdx.x == 0) bo[0] = 0;
        return;
    }
    int* hist = bin_smem + w * (NB + 1);
    int* pre = bin_smem + W * (NB + 1);
    int* scan = pre + (NB + 1);
    for (int k = threadIdx.x; k < W * (NB + 1); k += blockDim.x) bin_smem[k] = 0;
    __syncthreads();
    const int chunk = ((n + W - 1) / W + 31) & ~31;
    const int i0 = w * chunk, i1 = min(i0 + chunk, n);
    bool bad = false;
    for (int i = i0 + lane; i < i1; i += 32) {
        const float* p = pos_hi + 3 * (v0 + i);
        const float dx = p[0] - rc.cx, dy = p[1] - rc.cy, dz = p[2] - rc.cz;
        const float key = sqrtf(dx * dx + dy * dy + dz * dz) * a.q;
        a.key[v0 + i] = key;
        bad = bad || !(key == key) || isinf(key);
        atomicAdd(&hist[block_of_key(key, NB)], 1);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&a.hdr->status, FRAM_DEV_NONFINITE);
    __syncthreads();
    // Column totals over warps, exclusive prefix over blocks (each thread a contiguous range).
    const int per = (NB + blockDim.x - 1) / blockDim.x;
    const int j0 = threadIdx.x * per, j1 = min(j0 + per, NB);
    int local = 0;
    for (int j = j0; j < j1; ++j)
        for (int u = 0; u < W; ++u) local += bin_smem[u * (NB + 1) + j];
    int x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scan[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int u = 0; u < W; ++u) { const int t = scan[u]; scan[u] = run; run += t; }
    }
    __syncthreads();
    int run = scan[w] + x - local;           // exclusive prefix of this thread's first block
    for (int j = j0; j < j1; ++j) {
        pre[j] = run;
        p32[j] = run;
        for (int u = 0; u < W; ++u) {        // warp u's first position in block j
            const int c = bin_smem[u * (NB + 1) + j];
            bin_smem[u * (NB + 1) + j] = run;
            run += c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) p32[NB] = n;
    const int bpt = T >> 5;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) bo[t] = pre[t * bpt];
    if (threadIdx.x == 0) bo[nt] = n;
    // Stable scatter by block, warp w over its own range in index order.
    for (int base = i0; base < i1; base += 32) {
        const int i = base + lane;
        const bool act = i < i1;
        const int j = act ? block_of_key(a.key[v0 + i], NB) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int basepos = (lane == leader && act) ? hist[j] : 0;
        basepos = __shfl_sync(0xffffffffu, basepos, leader);
        __syncwarp();
        if (lane == leader && act) hist[j] = basepos + __popc(peers);
        __syncwarp();
        if (act && FRAM_GUARD(a.hdr, j >= 0 && j < NB && basepos + rank >= 0 && basepos + rank < n &&
                              v0 + n <= a.n_vs_total)) {
            a.perm[v0 + basepos + rank] = i;
            a.skey[v0 + basepos + rank] = j << 5;
        }
    }
}

// Image positions in sorted order (one CTA per (room, source), coalesced over sorted positions).
__global__ void __launch_bounds__(256) sort_positions(LaunchArgs a, const float* __restrict__ pos_hi,
                                                      const float* __restrict__ pos_lo)
{
    const int64_t seg = blockIdx.x;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    if (rc.ntiles < 1) return;      // a room the prologue rejected has no sorted order
    const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
    for (int p = threadIdx.x; p < rc.n_vs; p += blockDim.x) {
        const int q = a.perm[v0 + p];
        if (!FRAM_GUARD(a.hdr, q >= 0 && q < rc.n_vs && v0 + rc.n_vs <= a.n_vs_total)) continue;
        const int64_t i = v0 + q;
        const float* ph = pos_hi + 3 * i;
        float lx = 0.0f, ly = 0.0f, lz = 0.0f;
        if (pos_lo) { const float* pl = pos_lo + 3 * i; lx = pl[0]; ly = pl[1]; lz = pl[2]; }
        a.spa[v0 + p] = make_float4(ph[0], ph[1], ph[2], lx);
        a.spb[v0 + p] = make_float2(ly, lz);
    }
}

// Image arrival for mic (mx, my, mz): delay as integer n_c + delta and distance, from the
// float-pair image position.  The difference p - mic is formed exactly (TwoSum) before
// squaring, so no digit of the 400 m-scale coordinates is lost.
__device__ __forceinline__ void image_delay(float phx, float phy, float phz, float plx, float ply, float plz,
                                            float mx, float my, float mz, f2 q2, int& nc, float& delta, float& dist)
{
    f2 dx = two_sum(phx, -mx); dx.lo = __fadd_rn(dx.lo, plx);
    f2 dy = two_sum(phy, -my); dy.lo = __fadd_rn(dy.lo, ply);
    f2 dz = two_sum(phz, -mz); dz.lo = __fadd_rn(dz.lo, plz);
    f2 sx = two_prod(dx.hi, dx.hi); sx.lo = __fmaf_rn(__fmul_rn(2.0f, dx.hi), dx.lo, sx.lo);
    f2 sy = two_prod(dy.hi, dy.hi); sy.lo = __fmaf_rn(__fmul_rn(2.0f, dy.hi), dy.lo, sy.lo);
    f2 sz = two_prod(dz.hi, dz.hi); sz.lo = __fmaf_rn(__fmul_rn(2.0f, dz.hi), dz.lo, sz.lo);
    f2 ss = f2_add(f2_add(fast_two_sum(sx.hi, sx.lo), fast_two_sum(sy.hi, sy.lo)), fast_two_sum(sz.hi, sz.lo));
    f2 D = f2_sqrt_fast(ss);
    f2 t = f2_mul(D, q2);
    nc = __float2int_rn(t.hi);
    delta = __fadd_rn(__fsub_rn(t.hi, (float)nc), t.lo);
    dist = D.hi;
}

// Work-item records for the synthesis: room, source, tile, and the run of sorted images whose
// binning key lies within K + margin of the tile (from the 32-sample block table).
// Item qi belongs to the room b with item_off[b] <= qi < item_off[b + 1] (binary search; rooms
// without items have empty ranges), as source s and tile tau of its S x ntiles items.  The item
// table (room, source << 16 | tile) is written here, in parallel, for the adjoint (a serial fill
// in item_scan's single CTA took ~0.1 ms per large_4096 step).
__global__ void item_ranges(LaunchArgs a, int64_t max_items)
{
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= max_items || qi >= a.hdr->n_items) return;
    int lo = 0, hi = a.B;                  // item_off[lo] <= qi < item_off[hi] = n_items
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.item_off[mid] <= qi) lo = mid;
        else hi = mid;
    }
    const int b = lo;
    const RoomConst rc = a.room[b];
    const int r = (int)(qi - a.item_off[b]);
    if (!FRAM_GUARD(a.hdr, rc.ntiles >= 1 && r >= 0 && r < a.S * rc.ntiles)) return;
    const int s = r / rc.ntiles, tau = r - s * rc.ntiles;
    a.items[qi] = make_int2(b, (s << 16) | tau);
    ItemRec ir;
    ir.b = b;
    ir.s = s;
    ir.T0 = tau * a.tile;
    ir.len = rc.len;
    const int* p32 = a.pos32 + ((int64_t)b * a.S + s) * ((int64_t)a.nb32 + 1);
    const int kmin = max(ir.T0 - a.K - a.margin_i, 0);
    const int kmax = ir.T0 + a.tile - 1 + a.K + a.margin_i;
    ir.c_lo = p32[kmin >> 5];
    ir.c_hi = p32[min((kmax >> 5) + 1, a.nb32)];
    ir.pad0 = ir.pad1 = 0;
    ir.v0 = rc.vs_off + (int64_t)s * rc.n_vs;
    ir.out0 = rc.rir_off + (int64_t)s * a.M * rc.len;
    a.irec[qi] = ir;
}

// r^g of every image, in sorted order (one CTA per (room, source)).
__global__ void __launch_bounds__(256) amp_gather(LaunchArgs a, const float* __restrict__ g)
{
    const int64_t seg = blockIdx.x;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    if (rc.ntiles < 1) return;      // a room the prologue rejected has no sorted order
    const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
    for (int p = threadIdx.x; p < rc.n_vs; p += blockDim.x) {
        const int q = a.perm[v0 + p];
        if (FRAM_GUARD(a.hdr, q >= 0 && q < rc.n_vs && v0 + rc.n_vs <= a.n_vs_total))
            a.samp[v0 + p] = exp2f(g[v0 + q] * rc.log2r);
    }
}

// Arrival record (delta, P, a, b) of the tap identity for t = n_c + delta (|delta| <= 1/2),
// with P = A sin(pi delta) / (2 pi), a = P cos(pi delta / K), b = P sin(pi delta / K).  The taps
// with |n - t| < K are n_c - K + 1 .. n_c + K when delta > 0 and n_c - K .. n_c + K - 1 when
// delta < 0; an arrival with delta > 2^-12 is re-based to n_c + 1, delta - 1, so that every
// arrival's taps are base + o, o in [-K, K - 1].  The re-based delta rounds to a multiple of
// 2^-24 and every constant is computed from that rounded value, so the record describes one
// consistent delay (moved by < 3e-8 samples).  For 0 <= delta <= 2^-12 the dropped tap at
// n_c + K has the window weight sin^2(pi delta / 2K) < 1e-12.  The identity holds for any split
// of t; sin(pi (delta - 1)) = -sin(pi delta) keeps the polynomial arguments within [-1/2, 1/2].
constexpr float kShiftMin = 2.44140625e-4f;   // 2^-12

__device__ __forceinline__ float4 arrival_record(int& nc, float delta, float A, float invK, bool exact_trig)
{
    float sp;
    if (delta > kShiftMin) {
        const float d1 = __fsub_rn(delta, 1.0f);
        sp = -sinpi_poly(__fadd_rn(d1, 1.0f));
        delta = d1;
        nc += 1;
    } else {
        if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
        sp = sinpi_poly(delta);
    }
    const float P = A * sp * kTwoPiInv;
    const float y = delta * invK;
    float cy, sy;
    if (exact_trig) {               // K = 1: |delta / K| may exceed 1/2
        sincospif(y, &sy, &cy);
    } else {
        cy = cospi_poly(y);
        sy = sinpi_poly(y);
    }
    return make_float4(delta, P, P * cy, P * sy);
}

// Per-lane constants of the tap slots j = lane + 32 k (k < NR rounds), tap offset o = j - K:
// C = cos(pi o / K), S = sin(pi o / K), sg = (-1)^o, kp = -sg o, so that the tap at base + o is
// (P + a C + b S) / fma(sg, delta, kp).  Slots j >= 2K get kp = +inf: their reciprocal is 0 and
// their read-modify-write leaves the buffer unchanged.  Rounds go in pairs (k, k + 1) through
// packed FP32 (fma.rn.f32x2: two independent IEEE fused multiply-adds, each half rounded exactly
// as __fmaf_rn), so the constants of a pair sit in one 64-bit register pair; an odd last round
// stays scalar.
template <int NR>
struct TapLanes {
    static constexpr int NP = NR / 2 > 0 ? NR / 2 : 1;    // (one unused pair when NR = 1)
    f32x2 C[NP], S[NP], sg[NP], kp[NP];                   // rounds (2i, 2i + 1)
    float Cl, Sl, sgl, kpl;                                // round NR - 1 when NR is odd
};

template <int NR>
__device__ __forceinline__ void init_tap_lanes(TapLanes<NR>& L, int lane, int K)
{
    const float invK = 1.0f / (float)K;
    float C[NR], S[NR], sg[NR], kp[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int j = lane + 32 * k;
        const int o = j - K;
        float sn, cs;
        sincospif((float)o * invK, &sn, &cs);
        const bool ok = j < 2 * K;
        C[k] = ok ? cs : 0.0f;
        S[k] = ok ? sn : 0.0f;
        sg[k] = ok ? ((o & 1) ? -1.0f : 1.0f) : 0.0f;
        kp[k] = ok ? -sg[k] * (float)o : __int_as_float(0x7f800000);
    }
#pragma unroll
    for (int i = 0; i < NR / 2; ++i) {
        L.C[i] = pack2(C[2 * i], C[2 * i + 1]);
        L.S[i] = pack2(S[2 * i], S[2 * i + 1]);
        L.sg[i] = pack2(sg[2 * i], sg[2 * i + 1]);
        L.kp[i] = pack2(kp[2 * i], kp[2 * i + 1]);
    }
    L.Cl = C[NR - 1];
    L.Sl = S[NR - 1];
    L.sgl = sg[NR - 1];
    L.kpl = kp[NR - 1];
}

// An arrival record with each field duplicated into both halves of a packed pair.
struct Rec2 {
    f32x2 x, y, z, w;
};
__device__ __forceinline__ Rec2 splat_rec(float4 r)
{
    return Rec2{pack2(r.x, r.x), pack2(r.y, r.y), pack2(r.z, r.z), pack2(r.w, r.w)};
}

// The constants of round k (k a compile-time index after unrolling).
template <int NR>
__device__ __forceinline__ void lane_consts(const TapLanes<NR>& L, int k, float& C, float& S, float& sg, float& kp)
{
    if (k < 2 * (NR / 2)) {
        float c0, c1, s0, s1, g0, g1, p0, p1;
        unpack2(L.C[k >> 1], c0, c1);
        unpack2(L.S[k >> 1], s0, s1);
        unpack2(L.sg[k >> 1], g0, g1);
        unpack2(L.kp[k >> 1], p0, p1);
        const bool hi = k & 1;
        C = hi ? c1 : c0;
        S = hi ? s1 : s0;
        sg = hi ? g1 : g0;
        kp = hi ? p1 : p0;
    } else {
        C = L.Cl;
        S = L.Sl;
        sg = L.sgl;
        kp = L.kpl;
    }
}

// Adds one arrival's taps to the warp's tile buffer.  `rb` is the byte offset, from the start of
// the dynamic shared memory, of the buffer word that tap slot 0 of lane 0 updates; lane4 = 4 lane.
// add_arrival_inner: every round lies inside the buffer (the caller checked).
// add_arrival_edge: rounds that start outside (-32, T) are skipped -- they hold no sample of the
// tile -- so every index stays inside the buffer; s0 is the tile offset of slot 0.
template <int NR>
__device__ __forceinline__ void add_arrival_inner(char* __restrict__ smem, const TapLanes<NR>& L, float4 r, int rb,
                                                  int lane4)
{
    float* dst = reinterpret_cast<float*>(smem + (rb + lane4));
    const Rec2 r2 = splat_rec(r);
#pragma unroll
    for (int i = 0; i < NR / 2; ++i) {
        float e0, e1;
        unpack2(fma2(L.sg[i], r2.x, L.kp[i]), e0, e1);
        const f32x2 num = fma2(L.C[i], r2.z, fma2(L.S[i], r2.w, r2.y));
        float a0, a1;
        unpack2(fma2(num, pack2(rcp_approx(e0), rcp_approx(e1)), pack2(dst[64 * i], dst[64 * i + 32])), a0, a1);
        dst[64 * i] = a0;
        dst[64 * i + 32] = a1;
    }
    if constexpr ((NR & 1) != 0) {
        const float e = __fmaf_rn(L.sgl, r.x, L.kpl);
        const float num = __fmaf_rn(L.Cl, r.z, __fmaf_rn(L.Sl, r.w, r.y));
        dst[32 * (NR - 1)] = __fmaf_rn(num, rcp_approx(e), dst[32 * (NR - 1)]);
    }
}

template <int NR>
__device__ __forceinline__ void add_arrival_edge(char* __restrict__ smem, const TapLanes<NR>& L, float4 r, int rb,
                                                 int lane4, int s0, int T)
{
    float* dst = reinterpret_cast<float*>(smem + (rb + lane4));
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (s0 + 32 * k > -32 && s0 + 32 * k < T) {
            float C, S, sg, kp;
            lane_consts<NR>(L, k, C, S, sg, kp);
            const float e = __fmaf_rn(sg, r.x, kp);
            const float num = __fmaf_rn(C, r.z, __fmaf_rn(S, r.w, r.y));
            dst[32 * k] = __fmaf_rn(num, rcp_approx(e), dst[32 * k]);
        }
    }
}

// Per-warp shared memory (floats): the tile buffer (T + 68: sample T0 + k sits at index h + k,
// h = 32 + the output's word offset mod 4, so the store runs in aligned float4s and at least 32
// samples of halo remain on each side), 32 arrival records (float4) and their buffer offsets,
// each with one spare entry so the next record can be prefetched without a bound check.
__host__ __device__ inline int synth_warp_floats(int T) { return (T + 68) + 4 * 33 + 36; }

// Work unit = (room, source, tile, mic), one warp each, pulled from a counter (the next unit is
// requested when the current one starts).  Per unit: zero the tile buffer; add the direct path;
// walk the run of sorted images that can reach the tile 32 at a time -- each lane computes one
// image's arrival for this mic (the next 32 images' data is fetched meanwhile), the warp compacts
// the ones that reach the tile (those whose taps all fall inside the buffer first) and adds them
// one after another, each lane owning one tap slot; then store the tile (and the Eq. 9 early
// RIR).  The accumulation order of every sample is fixed by the sorted image order and the
// compaction, and no two lanes write one sample in the same step.
template <int NR>
__global__ void __launch_bounds__(kSynthThreads, 3) synth_kernel(LaunchArgs a, float* __restrict__ rir,
                                                                  float* __restrict__ early)
{
    extern __shared__ __align__(16) float synth_smem[];
    char* smem = reinterpret_cast<char*>(synth_smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lane4 = 4 * lane;
    const int T = a.tile, K = a.K, M = a.M;
    float* buf = synth_smem + wid * synth_warp_floats(T);
    const int buf_b = 4 * wid * synth_warp_floats(T);     // byte offset of buf
    float4* rec = reinterpret_cast<float4*>(buf + T + 68);
    int* rrb = reinterpret_cast<int*>(rec + 33);
    TapLanes<NR> L;
    init_tap_lanes<NR>(L, lane, K);
    const float invK = 1.0f / (float)K;
    const bool exact_trig = K < 2;
    const int64_t n_units = (int64_t)a.hdr->n_items * M;
    const int reach_lo = 1 - 2 * K;        // rel range of arrivals with a tap in the tile
    const int inner_hi = T - 32 * (NR - 1); // rel < inner_hi and rel > -32: every round inside
    int u = 0;
    if (lane == 0) u = atomicAdd(&a.hdr->queue, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    while ((int64_t)u < n_units) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&a.hdr->queue, 1);
        const int qi = u / M, m = u - qi * M;
        const ItemRec ir = a.irec[qi];
        const int T0 = ir.T0, Lb = ir.len;
        const float* pm = a.mic + 3 * ((size_t)ir.b * M + m);
        const float mx = pm[0], my = pm[1], mz = pm[2];
        const DirectConst dc = a.direct[((int64_t)ir.b * a.S + ir.s) * M + m];
        const int64_t v0 = ir.v0;
        if (!FRAM_GUARD(a.hdr, ir.out0 >= 0 && ir.out0 + (int64_t)(m + 1) * Lb <= a.rir_total && T0 >= 0 && T0 < Lb &&
                                   v0 >= 0 && v0 + ir.c_hi <= a.n_vs_total)) {
            u = __shfl_sync(0xffffffffu, nxt, 0);
            continue;
        }
        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 pb = make_float2(0.f, 0.f);
        float am = 0.0f;
        if (ir.c_lo + lane < ir.c_hi) {
            pa = a.spa[v0 + ir.c_lo + lane];
            pb = a.spb[v0 + ir.c_lo + lane];
            am = a.samp[v0 + ir.c_lo + lane];
        }
        float* dst = rir + ir.out0 + (int64_t)m * Lb + T0;       // sample T0 of this RIR
        const int al = (int)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3);
        const int h = 32 + al;
        const int hb = buf_b + 4 * h;                             // byte offset of sample T0

        float4* b4 = reinterpret_cast<float4*>(buf);
        for (int k = lane; k < (T + 68) / 4; k += 32) b4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        {   // direct path (uniform across the warp)
            int nc = __float2int_rn(dc.t_hi);
            const float delta = __fadd_rn(__fsub_rn(dc.t_hi, (float)nc), dc.t_lo);
            if (dc.amp > 0.0f) {
                const float4 r = arrival_record(nc, delta, dc.amp, invK, exact_trig);
                const int rel = nc - K - T0;
                if (rel >= reach_lo && rel < T) add_arrival_edge<NR>(smem, L, r, hb + 4 * rel, lane4, rel, T);
            }
            __syncwarp();
        }
        for (int c = ir.c_lo; c < ir.c_hi; c += 32) {
            bool valid = false, inner = false;
            float4 rr = make_float4(0.f, 0.f, 0.f, 0.f);
            int rel = 0;
            if (c + lane < ir.c_hi) {
                int nc;
                float delta, D;
                image_delay(pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, mx, my, mz, a.q2, nc, delta, D);
                const float A = am * rcp_approx(D);
                if (D > 0.0f && A == A && fabsf(A) < 3.0e38f) {
                    rr = arrival_record(nc, delta, A, invK, exact_trig);
                    rel = nc - K - T0;
                    valid = rel >= reach_lo && rel < T;
                    // inside the buffer for every round; a subset of valid (for K < 16 the
                    // offsets -31 .. -2K reach no sample of the tile and have no record)
                    inner = valid && rel > -32 && rel < inner_hi;
                }
            }
            if (c + 32 + lane < ir.c_hi) {      // next 32 images, in flight during the taps below
                pa = a.spa[v0 + c + 32 + lane];
                pb = a.spb[v0 + c + 32 + lane];
                am = a.samp[v0 + c + 32 + lane];
            }
            const unsigned lt = (1u << lane) - 1u;
            const unsigned vi = __ballot_sync(0xffffffffu, inner);
            const unsigned ve = __ballot_sync(0xffffffffu, valid && !inner);
            const int ni = __popc(vi), nv = ni + __popc(ve);
            if (valid) {
                const int slot = inner ? __popc(vi & lt) : ni + __popc(ve & lt);
                rec[slot] = rr;
                rrb[slot] = inner ? hb + 4 * rel : rel;
            }
            __syncwarp();
            // The records are read-only here: the next one is loaded before the current taps.  The
            // buffer offsets come from one load per batch (lane q holds slot q's) and a shuffle.
            const int rbq = rrb[lane];
            float4 rn = rec[0];
            for (int q = 0; q < ni; ++q) {
                const float4 r = rn;
                const int rb = __shfl_sync(0xffffffffu, rbq, q);
                rn = rec[q + 1];
                if (FRAM_GUARD(a.hdr, rb >= buf_b && rb - buf_b + 4 * (32 * NR - 1) < 4 * (T + 68)))
                    add_arrival_inner<NR>(smem, L, r, rb, lane4);
                __syncwarp();
            }
            for (int q = ni; q < nv; ++q) {
                const int rl = __shfl_sync(0xffffffffu, rbq, q);
                // every round add_arrival_edge runs starts inside (-32, T) of the tile
                if (FRAM_GUARD(a.hdr, h - 32 >= 0 && h + T + 31 < T + 68))
                    add_arrival_edge<NR>(smem, L, rec[q], hb + 4 * rl, lane4, rl, T);
                __syncwarp();
            }
        }
        // ---- store the tile (and the Eq. 9 early RIR): buffer index h + k holds sample T0 + k,
        // and (h + k) % 4 == 0 exactly where dst + k is 16-byte aligned ----
        const int nT = min(T, Lb - T0);
        float* dste = early ? early + ir.out0 + (int64_t)m * Lb + T0 : nullptr;
        const int k0 = (4 - al) & 3;                       // first aligned k
        const int nvec = nT > k0 ? (nT - k0) >> 2 : 0;
        for (int v = lane; v < nvec; v += 32) {
            const int k = k0 + 4 * v;
            const float4 x = *reinterpret_cast<const float4*>(buf + h + k);
            *reinterpret_cast<float4*>(dst + k) = x;
        }
        if (lane < k0 && lane < nT) dst[lane] = buf[h + lane];
        {
            const int kt = k0 + 4 * nvec + lane;
            if (lane < 3 && kt < nT) dst[kt] = buf[h + kt];
        }
        if (dste) {
            for (int k = lane; k < nT; k += 32) {
                const int n = T0 + k;
                dste[k] = (n >= dc.early_lo && n <= dc.early_hi) ? buf[h + k] : 0.0f;
            }
        }
        __syncwarp();
        u = __shfl_sync(0xffffffffu, nxt, 0);
    }
}

}  // namespace



int synth_smem_total(int T) { return (int)sizeof(float) * (kSynthThreads / 32) * synth_warp_floats(T); }

cudaError_t launch_prepare(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* r,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.hdr, 0, sizeof(Header), st);
    if (e != cudaSuccess) return e;
    const int64_t n = std::max<int64_t>((int64_t)a.B, (int64_t)a.B * a.S * a.M);
    if (n > 0) {
        room_prologue<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, r);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    item_scan<<<1, 1024, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t segs = (int64_t)a.B * a.S;
    if (segs > 0) {
        // warps per (room, source): 8, fewer when the histogram rows would not fit in 200 KiB
        int W = 8;
        while (W > 1 && (size_t)bin_smem_ints(W, a.nb32) * sizeof(int) > (size_t)200 * 1024) --W;
        const int sm = (int)(sizeof(int) * (size_t)bin_smem_ints(W, a.nb32));
        int per_sm = 0;
        if ((e = kernel_residency((const void*)bin_images, 32 * W, sm, &per_sm)) != cudaSuccess) return e;
        bin_images<<<(unsigned)segs, 32 * W, sm, st>>>(a, pos_hi);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sort_positions<<<(unsigned)segs, 256, 0, st>>>(a, pos_hi, pos_lo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int64_t max_items = segs * a.max_tiles;
        item_ranges<<<(unsigned)((max_items + 255) / 256), 256, 0, st>>>(a, max_items);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int NR>
static cudaError_t launch_synth_nr(const LaunchArgs& a, float* rir, float* early, cudaStream_t st)
{
    const int smem = synth_smem_total(a.tile);
    int per_sm = 0;
    cudaError_t e = kernel_residency((const void*)synth_kernel<NR>, kSynthThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = device_sm_count() * per_sm;
    synth_kernel<NR><<<grid, kSynthThreads, smem, st>>>(a, rir, early);
    return cudaGetLastError();
}

cudaError_t launch_amp_gather(const LaunchArgs& a, const float* g, cudaStream_t st)
{
    const int64_t segs = (int64_t)a.B * a.S;
    if (segs > 0) {
        amp_gather<<<(unsigned)segs, 256, 0, st>>>(a, g);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_synthesize(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                              float* rir, float* early, cudaStream_t st)
{
    (void)pos_hi;
    (void)pos_lo;   // the kernel reads the sorted copies the preparation made
    cudaError_t e = launch_amp_gather(a, g, st);
    if (e != cudaSuccess) return e;
    switch ((2 * a.K + 31) / 32) {
    case 1: return launch_synth_nr<1>(a, rir, early, st);
    case 2: return launch_synth_nr<2>(a, rir, early, st);
    case 3: return launch_synth_nr<3>(a, rir, early, st);
    case 4: return launch_synth_nr<4>(a, rir, early, st);
    case 5: return launch_synth_nr<5>(a, rir, early, st);
    case 6: return launch_synth_nr<6>(a, rir, early, st);
    case 7: return launch_synth_nr<7>(a, rir, early, st);
    case 8: return launch_synth_nr<8>(a, rir, early, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fram
