// fram_synth.cu -- prologue, delay binning and the forward synthesis kernel (FRAM-RIR
// Eq. 1 with fractional-delay Hann-windowed sincs at the output rate, Sec. III-D, Eq. 9).
//
// Pipeline of fram_synthesize (all on the caller's stream, no host synchronisation):
//   1. room_prologue   one thread per room and per (room, source, mic): RIR length, tile count,
//                      array centre, binning margin, log2 r, and the direct path of every
//                      (source, mic) pair in FP64 (delay split into a float pair, amplitude
//                      1/D, Eq. 9 window).
//   2. item_scan       one CTA: prefix sum of S * ntiles_b -> work-item table (room, source, tile).
//   3. bin_images      one warp per (room, source): each image's delay to the array centre
//                      (the binning key, in samples) and a stable counting sort of the images
//                      by output tile.  Per-mic delays differ from the key by at most the
//                      array radius in samples ("margin").
//   4. synth_kernel    persistent CTAs pull (room, source, tile) items from a counter.  Per item:
//                      stage the images whose key lies within K + margin of the tile; then for
//                      each mic: compute every arrival's delay t = D fs/c0 (float-pair distance),
//                      amplitude and sinc constants; counting-sort arrivals by integer delay
//                      (ties by staging index, so the order is deterministic); and let each warp
//                      own 32-sample rows, gathering the arrivals whose window covers the row.
//
// Tap arithmetic.  With t = n_c + delta (n_c = nearest integer), sin(pi (n - t)) =
// (-1)^(n - n_c) sin(-pi delta), so for |n - t| < K
//   A sinc(n - t) w(n - t) = (-1)^n [P + cos(pi n/K) a' + sin(pi n/K) b'] / (t - n)
// with per-arrival constants P = (-1)^n_c A sin(pi delta) / (2 pi), a' = P cos(pi t/K),
// b' = P sin(pi t/K) (angle-difference form of the Hann term (1 + cos(pi (n - t)/K)) / 2).
// Per tap: d = (n_c - n) + delta (exact float difference + one rounding), two FMAs for the
// numerator, one reciprocal shared by two arrivals (1/d1 = d2 / (d1 d2)), one FMA to
// accumulate.  No global atomics touch the accumulators: each output sample is owned by one
// lane and sums its arrivals in sorted order.
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
    __syncthreads();
    // Fill the item table: item -> (room, source << 16 | tile).
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        const int nt = a.room[b].ntiles;
        int q = a.item_off[b];
        for (int s = 0; s < a.S; ++s)
            for (int t = 0; t < nt; ++t) a.items[q++] = make_int2(b, (s << 16) | t);
    }
}

// One warp per (room, source): binning keys and a stable counting sort by tile.
__global__ void __launch_bounds__(128) bin_images(LaunchArgs a, const float* __restrict__ pos_hi)
{
    extern __shared__ int bin_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (seg >= (int64_t)a.B * a.S) return;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    int* hist = bin_smem + wib * (a.max_tiles + 1);
    const int n = rc.n_vs, nt = rc.ntiles;
    const int64_t v0 = rc.vs_off + (int64_t)s * n;
    const float invT = 1.0f / (float)a.tile;
    int* bo = a.bin_off + seg * (a.max_tiles + 1);
    if (nt < 1) {   // a room the prologue rejected: no work items reference its bins
        if (lane == 0) bo[0] = 0;
        return;
    }
    for (int t = lane; t <= nt; t += 32) hist[t] = 0;
    __syncwarp();
    bool bad = false;
    for (int i = lane; i < n; i += 32) {
        const float* p = pos_hi + 3 * (v0 + i);
        const float dx = p[0] - rc.cx, dy = p[1] - rc.cy, dz = p[2] - rc.cz;
        const float key = sqrtf(dx * dx + dy * dy + dz * dz) * a.q;
        a.key[v0 + i] = key;
        int t;
        if (!(key < 3.0e9f)) { t = nt - 1; bad = bad || !(key == key) || isinf(key); }
        else {
            t = (int)floorf(key * invT);
            t = t > nt - 1 ? nt - 1 : t;
        }
        atomicAdd(&hist[t], 1);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&a.hdr->status, FRAM_DEV_NONFINITE);
    __syncwarp();
    // Exclusive scan over nt bins (chunks of 32), write bin offsets, keep running fill.
    int carry = 0;
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        const int v = t < nt ? hist[t] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int excl = carry + x - v;
        if (t < nt) { bo[t] = excl; hist[t] = excl; }
        carry = __shfl_sync(0xffffffffu, carry + x, 31);
    }
    if (lane == 0) bo[nt] = carry;
    __syncwarp();
    // Stable scatter in index order, 32 images at a time.
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool act = i < n;
        int t = -1;
        if (act) {
            const float key = a.key[v0 + i];
            if (!(key < 3.0e9f)) t = nt - 1;
            else {
                t = (int)floorf(key * invT);
                t = t > nt - 1 ? nt - 1 : t;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, t);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int basepos = (lane == leader && act) ? hist[t] : 0;
        basepos = __shfl_sync(0xffffffffu, basepos, leader);
        __syncwarp();
        if (lane == leader && act) hist[t] = basepos + __popc(peers);
        __syncwarp();
        if (act) a.perm[v0 + basepos + rank] = i;
    }
}

// Shared-memory plan of synth_kernel (bytes, 16-byte aligned pieces).
//   stage  image indices staged for the tile
//   rec4/recb  arrival constants in arrival order (n_c - T0, delta, P, a') and b'
//   rkey   delay bin of each arrival (-1 = no tap in the tile)
//   sidx   arrival order after the counting sort
//   q0/q1/q2  sorted arrivals, two per 48-byte group: (n1, d1, n2, d2) (P1, a1, b1, P2) (a2, b2, -, -)
//   start/fill  bin starts (exclusive prefix) and scatter cursors
//   outt   the tile's output samples for the current mic
//   tabT   cos, sin(pi m / K) for the tile's samples m = T0 - K - 1 + k
struct SynthSmem {
    int stage, rec4, recb, rkey, sidx, q0, q1, q2, start, fill, outt, tabT, total;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SynthSmem synth_smem(int T, int K)
{
    SynthSmem s;
    const int NB = T + 2 * K + 2;
    const int NA = kImpCap + 1;        // arrivals per chunk (images + the direct path)
    const int NP = (NA + 2) / 2;       // sorted pairs
    int off = 0;
    s.stage = off; off = al16(off + 4 * kStageCap);
    s.rec4 = off; off = al16(off + 16 * NA);
    s.recb = off; off = al16(off + 4 * NA);
    s.rkey = off; off = al16(off + 4 * NA);
    s.sidx = off; off = al16(off + 4 * NA);
    s.q0 = off; off = al16(off + 16 * NP);
    s.q1 = off; off = al16(off + 16 * NP);
    s.q2 = off; off = al16(off + 16 * NP);
    s.start = off; off = al16(off + 4 * (NB + 1));
    s.fill = off; off = al16(off + 4 * (NB + 1));
    s.outt = off; off = al16(off + 4 * T);
    s.tabT = off; off = al16(off + 8 * NB);
    s.total = off;
    return s;
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

// Block-wide exclusive scan of cnt[0..nb) into out[0..nb] and out2[0..nb) (out[nb] = total).
template <int NT>
__device__ void block_exclusive_scan(const int* cnt, int* out, int* out2, int nb, int* warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (nb + NT - 1) / NT;
    const int lo = tid * per, hi = min(lo + per, nb);
    int sum = 0;
    for (int k = lo; k < hi; ++k) sum += cnt[k];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < NT / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    int run = (wid > 0 ? warp_tot[wid - 1] : 0) + x - sum;
    for (int k = lo; k < hi; ++k) {
        const int c = cnt[k];
        out[k] = run;
        out2[k] = run;
        run += c;
    }
    if (tid == NT - 1) out[nb] = warp_tot[NT / 32 - 1];
    __syncthreads();
}

// One arrival record, read from the pair-interleaved sorted arrays.
struct Arr {
    float nc, d, P, a, b;
};

__device__ __forceinline__ Arr load_single(const float4* q0, const float4* q1, const float4* q2, int p)
{
    const int q = p >> 1;
    const float4 A = q0[q], Bv = q1[q];
    if ((p & 1) == 0) return {A.x, A.y, Bv.x, Bv.y, Bv.z};
    const float4 C = q2[q];
    return {A.z, A.w, Bv.w, C.x, C.y};
}

// Taps of arrivals [lo, hi) (sorted order) for the lane's sample; masked = check |t - n| < K.
template <bool kMasked>
__device__ __forceinline__ float row_taps(const float4* __restrict__ q0, const float4* __restrict__ q1,
                                          const float4* __restrict__ q2, int lo, int hi, float nl, float cn, float sn,
                                          float Kf)
{
    float acc0 = 0.0f, acc1 = 0.0f;
    int p = lo;
    if (p >= hi) return 0.0f;  // empty range (also keeps p >> 1 from rounding below lo)
    if (p & 1) {               // leading odd element
        const Arr r = load_single(q0, q1, q2, p);
        const float d = __fadd_rn(__fsub_rn(r.nc, nl), r.d);
        float num = __fmaf_rn(cn, r.a, __fmaf_rn(sn, r.b, r.P));
        if (kMasked && !(fabsf(d) < Kf)) num = 0.0f;
        acc0 = __fmul_rn(num, rcp_approx(d));
        ++p;
    }
    const int qend = (hi - p) >> 1;   // full pairs from p (even)
    int q = p >> 1;
    const int qstop = q + qend;
    // Two pairs per iteration, two accumulators.
    for (; q + 1 < qstop; q += 2) {
        const float4 A0 = q0[q], B0 = q1[q], C0 = q2[q];
        const float4 A1 = q0[q + 1], B1 = q1[q + 1], C1 = q2[q + 1];
        {
            const float d1 = __fadd_rn(__fsub_rn(A0.x, nl), A0.y);
            const float d2 = __fadd_rn(__fsub_rn(A0.z, nl), A0.w);
            float n1 = __fmaf_rn(cn, B0.y, __fmaf_rn(sn, B0.z, B0.x));
            float n2 = __fmaf_rn(cn, C0.x, __fmaf_rn(sn, C0.y, B0.w));
            if (kMasked) {
                if (!(fabsf(d1) < Kf)) n1 = 0.0f;
                if (!(fabsf(d2) < Kf)) n2 = 0.0f;
            }
            const float rp = rcp_approx(__fmul_rn(d1, d2));
            const float t = __fmaf_rn(n1, d2, __fmul_rn(n2, d1));
            acc0 = __fmaf_rn(t, rp, acc0);
        }
        {
            const float d1 = __fadd_rn(__fsub_rn(A1.x, nl), A1.y);
            const float d2 = __fadd_rn(__fsub_rn(A1.z, nl), A1.w);
            float n1 = __fmaf_rn(cn, B1.y, __fmaf_rn(sn, B1.z, B1.x));
            float n2 = __fmaf_rn(cn, C1.x, __fmaf_rn(sn, C1.y, B1.w));
            if (kMasked) {
                if (!(fabsf(d1) < Kf)) n1 = 0.0f;
                if (!(fabsf(d2) < Kf)) n2 = 0.0f;
            }
            const float rp = rcp_approx(__fmul_rn(d1, d2));
            const float t = __fmaf_rn(n1, d2, __fmul_rn(n2, d1));
            acc1 = __fmaf_rn(t, rp, acc1);
        }
    }
    if (q < qstop) {
        const float4 A0 = q0[q], B0 = q1[q], C0 = q2[q];
        const float d1 = __fadd_rn(__fsub_rn(A0.x, nl), A0.y);
        const float d2 = __fadd_rn(__fsub_rn(A0.z, nl), A0.w);
        float n1 = __fmaf_rn(cn, B0.y, __fmaf_rn(sn, B0.z, B0.x));
        float n2 = __fmaf_rn(cn, C0.x, __fmaf_rn(sn, C0.y, B0.w));
        if (kMasked) {
            if (!(fabsf(d1) < Kf)) n1 = 0.0f;
            if (!(fabsf(d2) < Kf)) n2 = 0.0f;
        }
        const float rp = rcp_approx(__fmul_rn(d1, d2));
        const float t = __fmaf_rn(n1, d2, __fmul_rn(n2, d1));
        acc0 = __fmaf_rn(t, rp, acc0);
        ++q;
    }
    p = q << 1;
    if (p < hi) {              // trailing element
        const Arr r = load_single(q0, q1, q2, p);
        const float d = __fadd_rn(__fsub_rn(r.nc, nl), r.d);
        float num = __fmaf_rn(cn, r.a, __fmaf_rn(sn, r.b, r.P));
        if (kMasked && !(fabsf(d) < Kf)) num = 0.0f;
        acc1 = __fmaf_rn(num, rcp_approx(d), acc1);
    }
    return __fadd_rn(acc0, acc1);
}

template <int NT>
__global__ void __launch_bounds__(NT, 3) synth_kernel(LaunchArgs a, const float* __restrict__ pos_hi,
                                                       const float* __restrict__ pos_lo, const float* __restrict__ gref,
                                                       float* __restrict__ rir, float* __restrict__ early)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = a.tile, K = a.K;
    const int NB = T + 2 * K + 2;
    const SynthSmem L = synth_smem(T, K);
    int* stage = reinterpret_cast<int*>(smem + L.stage);
    float4* rec4 = reinterpret_cast<float4*>(smem + L.rec4);
    float* recb = reinterpret_cast<float*>(smem + L.recb);
    int* rkey = reinterpret_cast<int*>(smem + L.rkey);
    int* sidx = reinterpret_cast<int*>(smem + L.sidx);
    float4* q0 = reinterpret_cast<float4*>(smem + L.q0);
    float4* q1 = reinterpret_cast<float4*>(smem + L.q1);
    float4* q2 = reinterpret_cast<float4*>(smem + L.q2);
    int* start = reinterpret_cast<int*>(smem + L.start);
    int* fill = reinterpret_cast<int*>(smem + L.fill);
    float* outt = reinterpret_cast<float*>(smem + L.outt);
    float2* tabT = reinterpret_cast<float2*>(smem + L.tabT);
    __shared__ int s_item, s_count;
    __shared__ int warp_tot[NT / 32];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = NT / 32;
    const float invK = 1.0f / (float)K;
    const float Kf = (float)K;
    const int twoK = 2 * K;
    const int n_items = a.hdr->n_items;

    for (;;) {
        if (tid == 0) { s_item = atomicAdd(&a.hdr->queue, 1); s_count = 0; }
        __syncthreads();
        const int qi = s_item;
        if (qi >= n_items) break;
        const int2 it = a.items[qi];
        const int b = it.x, s = it.y >> 16, tau = it.y & 0xffff;
        const RoomConst rc = a.room[b];
        const int T0 = tau * T;
        const int Lb = rc.len;
        const int base = T0 - K - 1;           // sample index of delay bin 0
        const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
        const int* bo = a.bin_off + ((int64_t)b * a.S + s) * (a.max_tiles + 1);
        const float kmin = (float)(T0 - K) - rc.margin - 1.0f;
        const float kmax = (float)(T0 + T + K) + rc.margin + 1.0f;
        const int bin_lo = max(0, (int)floorf(kmin / (float)T));
        const int bin_hi = min(rc.ntiles - 1, (int)floorf(kmax / (float)T));
        const int c_lo = bo[bin_lo];
        const int c_hi = bo[bin_hi + 1];

        // Phase table for the tile's samples: cos, sin(pi m / K), m = base + k.
        for (int k = tid; k < NB; k += NT) {
            int m = (base + k) % twoK;
            m = m < 0 ? m + twoK : m;
            float sn_, cs_;
            sincospif((float)m * invK, &sn_, &cs_);
            tabT[k] = make_float2(cs_, sn_);
        }
        // ---- stage images whose key lies within reach of the tile (stable compaction) ----
        for (int cb = c_lo; cb < c_hi; cb += NT) {
            const int idx = cb + tid;
            int img = -1;
            if (idx < c_hi) {
                const int i = a.perm[v0 + idx];
                const float k = a.key[v0 + i];
                if (k >= kmin && k <= kmax) img = i;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, img >= 0);
            if (lane == 0) warp_tot[wid] = __popc(bal);
            __syncthreads();
            int before = s_count;
            for (int w = 0; w < wid; ++w) before += warp_tot[w];
            const int pos = before + __popc(bal & ((1u << lane) - 1u));
            if (img >= 0 && pos < kStageCap) stage[pos] = img;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < NW; ++w) tot += warp_tot[w];
                s_count += tot;
            }
            __syncthreads();
        }
        __syncthreads();
        int nstage = s_count;
        if (nstage > kStageCap) {
            if (tid == 0) atomicOr(&a.hdr->status, FRAM_DEV_CAPACITY);
            nstage = kStageCap;
        }
        const float log2r = rc.log2r;

        for (int m = 0; m < a.M; ++m) {
            const DirectConst dc = a.direct[((int64_t)b * a.S + s) * a.M + m];
            const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
            const float mx = pm[0], my = pm[1], mz = pm[2];
            for (int k = tid; k < T; k += NT) outt[k] = 0.0f;
            const int nchunks = nstage > 0 ? (nstage + kImpCap - 1) / kImpCap : 1;
            for (int ch = 0; ch < nchunks; ++ch) {
                const int c0 = ch * kImpCap;
                const int n_in = max(0, min(kImpCap, nstage - c0));
                // ---- arrival constants: slot 0 is the direct path (first chunk only) ----
                for (int j = tid; j <= n_in; j += NT) {
                    int nc = 0;
                    float delta = 0.f, A = 0.f;
                    bool ok;
                    if (j > 0) {
                        const int i = stage[c0 + j - 1];
                        const int64_t v = v0 + i;
                        const float* ph = pos_hi + 3 * v;
                        float plx = 0.f, ply = 0.f, plz = 0.f;
                        if (pos_lo) { plx = pos_lo[3 * v]; ply = pos_lo[3 * v + 1]; plz = pos_lo[3 * v + 2]; }
                        float D;
                        image_delay(ph[0], ph[1], ph[2], plx, ply, plz, mx, my, mz, a.q2, nc, delta, D);
                        A = exp2f(gref[v] * log2r) * rcp_approx(D);
                        ok = (D > 0.0f) && (A == A) && (fabsf(A) < 3.0e38f);
                    } else {
                        ok = (ch == 0);
                        nc = __float2int_rn(dc.t_hi);
                        delta = __fadd_rn(__fsub_rn(dc.t_hi, (float)nc), dc.t_lo);
                        A = dc.amp;
                    }
                    int key = -1;
                    if (ok) {
                        key = nc - base;
                        if (key < 0 || key >= NB) key = -1;
                    }
                    if (key >= 0) {
                        if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
                        const float P = ((nc & 1) ? -A : A) * sinpi_poly(delta) * kTwoPiInv;
                        const float y = delta * invK;
                        const float sk = sinpi_poly(y), ck = cospi_poly(y);
                        const float2 cs = tabT[key];
                        const float ca = cs.x * ck - cs.y * sk;   // cos(pi t / K)
                        const float sa = cs.y * ck + cs.x * sk;   // sin(pi t / K)
                        rec4[j] = make_float4((float)(nc - T0), delta, P, P * ca);
                        recb[j] = P * sa;
                    }
                    rkey[j] = key;
                }
                for (int k = tid; k <= NB; k += NT) fill[k] = 0;
                __syncthreads();
                // ---- counting sort by integer delay; ties keep arrival order ----
                for (int j = tid; j <= n_in; j += NT)
                    if (rkey[j] >= 0) atomicAdd(&fill[rkey[j]], 1);
                __syncthreads();
                block_exclusive_scan<NT>(fill, start, fill, NB, warp_tot);
                for (int j = tid; j <= n_in; j += NT) {
                    const int key = rkey[j];
                    if (key >= 0) sidx[atomicAdd(&fill[key], 1)] = j;
                }
                __syncthreads();
                for (int k = tid; k < NB; k += NT) {
                    const int lo = start[k], hi = start[k + 1];
                    for (int x = lo + 1; x < hi; ++x) {
                        const int id = sidx[x];
                        int y = x - 1;
                        while (y >= lo && sidx[y] > id) { sidx[y + 1] = sidx[y]; --y; }
                        sidx[y + 1] = id;
                    }
                }
                __syncthreads();
                const int total = start[NB];
                for (int p = tid; p < total; p += NT) {
                    const int j = sidx[p];
                    const float4 r = rec4[j];
                    const float bb = recb[j];
                    const int q = p >> 1;
                    float* f0 = reinterpret_cast<float*>(q0 + q);
                    float* f1 = reinterpret_cast<float*>(q1 + q);
                    float* f2p = reinterpret_cast<float*>(q2 + q);
                    if ((p & 1) == 0) { f0[0] = r.x; f0[1] = r.y; f1[0] = r.z; f1[1] = r.w; f1[2] = bb; }
                    else { f0[2] = r.x; f0[3] = r.y; f1[3] = r.z; f2p[0] = r.w; f2p[1] = bb; }
                }
                __syncthreads();
                // ---- taps: each warp owns rows of 32 consecutive samples ----
                for (int row = wid; row * 32 < T; row += NW) {
                    const int R0 = T0 + row * 32;
                    if (R0 >= Lb) break;
                    const int k0 = row * 32;
                    const int lo = start[k0 + 1];
                    const int ilo = start[min(k0 + 33, k0 + twoK + 1)];
                    const int ihi = start[k0 + twoK + 1];
                    const int hi = start[min(k0 + twoK + 33, NB)];
                    const float nl = (float)(k0 + lane);
                    const float2 cs = tabT[k0 + lane + K + 1];
                    float acc = row_taps<true>(q0, q1, q2, lo, ilo, nl, cs.x, cs.y, Kf);
                    acc = __fadd_rn(acc, row_taps<false>(q0, q1, q2, ilo, ihi, nl, cs.x, cs.y, Kf));
                    acc = __fadd_rn(acc, row_taps<true>(q0, q1, q2, max(ihi, ilo), hi, nl, cs.x, cs.y, Kf));
                    outt[k0 + lane] += ((R0 + lane) & 1) ? -acc : acc;
                }
                __syncthreads();
            }
            // ---- store the tile (and the Eq. 9 early RIR) ----
            float* dst = rir + rc.rir_off + ((int64_t)s * a.M + m) * Lb;
            float* dste = early ? early + rc.rir_off + ((int64_t)s * a.M + m) * Lb : nullptr;
            for (int k = tid; k < T; k += NT) {
                const int n = T0 + k;
                if (n < Lb) {
                    const float h = outt[k];
                    dst[n] = h;
                    if (dste) dste[n] = (n >= dc.early_lo && n <= dc.early_hi) ? h : 0.0f;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

int synth_smem_bytes(int T, int K) { return synth_smem(T, K).total; }

cudaError_t launch_prepare(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* r,
                           cudaStream_t st)
{
    (void)pos_lo;
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
        const size_t sm = sizeof(int) * 4 * (size_t)(a.max_tiles + 1);
        bin_images<<<(unsigned)((segs + 3) / 4), 128, sm, st>>>(a, pos_hi);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_synthesize(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                              float* rir, float* early, cudaStream_t st)
{
    const int smem = synth_smem(a.tile, a.K).total;
    int per_sm = 0;
    cudaError_t e = kernel_residency((const void*)synth_kernel<kSynthThreads>, kSynthThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = device_sm_count() * per_sm;
    synth_kernel<kSynthThreads><<<grid, kSynthThreads, smem, st>>>(a, pos_hi, pos_lo, g, rir, early);
    return cudaGetLastError();
}

}  // namespace fram
