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

// One warp per (room, source): binning keys, a stable counting sort of the images by tile, then
// a stable counting sort inside each tile by floor(key).  The result: perm (image indices) and
// skey (a monotone integer key per position), so any delay range of a source's images is one
// contiguous run, found by binary search.
__host__ __device__ inline int bin_warp_ints(int max_tiles, int T) { return (max_tiles + 1) + 2 * T; }

__device__ __forceinline__ int tile_of_key(float key, float invT, int nt)
{
    if (!(key < 3.0e9f)) return nt - 1;               // NaN or beyond any RIR: last tile
    const int t = (int)floorf(key * invT);
    return t > nt - 1 ? nt - 1 : t;
}

__global__ void __launch_bounds__(64) bin_images(LaunchArgs a, const float* __restrict__ pos_hi)
{
    extern __shared__ int bin_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (seg >= (int64_t)a.B * a.S) return;
    const int b = (int)(seg / a.S), s = (int)(seg % a.S);
    const RoomConst rc = a.room[b];
    const int T = a.tile;
    int* hist = bin_smem + wib * bin_warp_ints(a.max_tiles, T);
    int* fine = hist + (a.max_tiles + 1);
    const int n = rc.n_vs, nt = rc.ntiles;
    const int64_t v0 = rc.vs_off + (int64_t)s * n;
    const float invT = 1.0f / (float)T;
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
        bad = bad || !(key == key) || isinf(key);
        atomicAdd(&hist[tile_of_key(key, invT, nt)], 1);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&a.hdr->status, FRAM_DEV_NONFINITE);
    __syncwarp();
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
    // Pass 1: stable scatter by tile into ptmp (index order within a tile).
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const bool act = i < n;
        const int t = act ? tile_of_key(a.key[v0 + i], invT, nt) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, t);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int basepos = (lane == leader && act) ? hist[t] : 0;
        basepos = __shfl_sync(0xffffffffu, basepos, leader);
        __syncwarp();
        if (lane == leader && act) hist[t] = basepos + __popc(peers);
        __syncwarp();
        if (act) a.ptmp[v0 + basepos + rank] = i;
    }
    __syncwarp();
    // Pass 2: inside each tile, stable counting sort by floor(key) - tile start.  The last tile
    // also takes every key beyond the RIR, in a doubled bucket range clamped at its end.
    for (int t = 0; t < nt; ++t) {
        const int b0 = bo[t], b1 = bo[t + 1];
        if (b1 <= b0) continue;
        const int nb = (t == nt - 1) ? 2 * T : T;
        const int t0 = t * T;
        for (int f = lane; f < nb; f += 32) fine[f] = 0;
        __syncwarp();
        for (int p = b0 + lane; p < b1; p += 32) {
            const float key = a.key[v0 + a.ptmp[v0 + p]];
            int f = (key < 3.0e9f) ? (int)floorf(key) - t0 : nb - 1;
            f = f < 0 ? 0 : (f > nb - 1 ? nb - 1 : f);
            atomicAdd(&fine[f], 1);
        }
        __syncwarp();
        int run = b0;
        for (int base = 0; base < nb; base += 32) {
            const int f = base + lane;
            const int v = fine[f];
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            fine[f] = run + x - v;
            run = __shfl_sync(0xffffffffu, run + x, 31);
        }
        __syncwarp();
        for (int base = b0; base < b1; base += 32) {
            const int p = base + lane;
            const bool act = p < b1;
            int f = -1, i = 0;
            if (act) {
                i = a.ptmp[v0 + p];
                const float key = a.key[v0 + i];
                f = (key < 3.0e9f) ? (int)floorf(key) - t0 : nb - 1;
                f = f < 0 ? 0 : (f > nb - 1 ? nb - 1 : f);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, f);
            const int leader = __ffs(peers) - 1;
            const int rank = __popc(peers & ((1u << lane) - 1u));
            int basepos = (lane == leader && act) ? fine[f] : 0;
            basepos = __shfl_sync(0xffffffffu, basepos, leader);
            __syncwarp();
            if (lane == leader && act) fine[f] = basepos + __popc(peers);
            __syncwarp();
            if (act) {
                a.perm[v0 + basepos + rank] = i;
                a.skey[v0 + basepos + rank] = t0 + f;
            }
        }
        __syncwarp();
    }
}

// Shared-memory plan of synth_kernel (bytes, 16-byte aligned pieces).
//   sperm/skeys  the tile's candidate images (sorted by delay key) and their keys
//   rowb         per 32-sample row: first and one-past-last candidate in reach
//   q0/q1/q2     arrival records, two per 48-byte group: (n1, d1, n2, d2) (P1, a1, b1, P2) (a2, b2, -, -)
//   outt         the tile's samples for the current mic
//   tabT         cos, sin(pi m / K) for m = base + k, base = T0 - K - M - 1
struct SynthSmem {
    int sperm, skeys, rowb, q0, q1, q2, outt, tabT, total, nbk;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SynthSmem synth_smem(int T, int K, int M)
{
    SynthSmem s;
    s.nbk = T + 2 * K + 2 * M + 2;
    const int NP = kArrCap / 2 + 1;
    int off = 0;
    s.sperm = off; off = al16(off + 4 * kStageCap);
    s.skeys = off; off = al16(off + 4 * kStageCap);
    s.rowb = off; off = al16(off + 4 * (2 * (T / 32) + 2));
    s.q0 = off; off = al16(off + 16 * NP);
    s.q1 = off; off = al16(off + 16 * NP);
    s.q2 = off; off = al16(off + 16 * NP);
    s.outt = off; off = al16(off + 4 * T);
    s.tabT = off; off = al16(off + 8 * s.nbk);
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

// Arrival constants of the tap identity: P = (-1)^n_c A sin(pi delta)/(2 pi), a' = P cos(pi t/K),
// b' = P sin(pi t/K), from the phase table entry cs = (cos, sin)(pi n_c / K).
__device__ __forceinline__ float3 arrival_consts(int nc, float delta, float A, float2 cs, float invK)
{
    const float P = ((nc & 1) ? -A : A) * sinpi_poly(delta) * kTwoPiInv;
    const float y = delta * invK;
    const float sk = sinpi_poly(y), ck = cospi_poly(y);
    const float ca = cs.x * ck - cs.y * sk;
    const float sa = cs.y * ck + cs.x * sk;
    return make_float3(P, P * ca, P * sa);
}

__device__ __forceinline__ void put_record(float4* q0, float4* q1, float4* q2, int p, float nc_l, float delta,
                                           float3 c)
{
    const int q = p >> 1;
    float* f0 = reinterpret_cast<float*>(q0 + q);
    float* f1 = reinterpret_cast<float*>(q1 + q);
    float* f2p = reinterpret_cast<float*>(q2 + q);
    if ((p & 1) == 0) { f0[0] = nc_l; f0[1] = delta; f1[0] = c.x; f1[1] = c.y; f1[2] = c.z; }
    else { f0[2] = nc_l; f0[3] = delta; f1[3] = c.x; f2p[0] = c.y; f2p[1] = c.z; }
}

// Taps of the arrival pairs [q, qend) for the lane's sample.  Every arrival is masked with
// |t - n| < K, so a pair may include one arrival outside the row's reach (it contributes zero);
// a zero-weight record far from every sample completes an odd count.
__device__ __forceinline__ float pair_tap(const float4 A, const float4 B, const float4 C, float nl, float cn, float sn,
                                          float Kf, float acc)
{
    const float e1 = __fadd_rn(__fsub_rn(A.x, nl), A.y);
    const float e2 = __fadd_rn(__fsub_rn(A.z, nl), A.w);
    float n1 = __fmaf_rn(cn, B.y, __fmaf_rn(sn, B.z, B.x));
    float n2 = __fmaf_rn(cn, C.x, __fmaf_rn(sn, C.y, B.w));
    n1 = fabsf(e1) < Kf ? n1 : 0.0f;
    n2 = fabsf(e2) < Kf ? n2 : 0.0f;
    const float rp = rcp_approx(__fmul_rn(e1, e2));
    return __fmaf_rn(__fmaf_rn(n1, e2, __fmul_rn(n2, e1)), rp, acc);
}

__device__ __forceinline__ float row_taps(const float4* __restrict__ q0, const float4* __restrict__ q1,
                                          const float4* __restrict__ q2, int q, int qend, float nl, float cn, float sn,
                                          float Kf)
{
    float acc0 = 0.0f, acc1 = 0.0f;
    for (; q + 1 < qend; q += 2) {
        acc0 = pair_tap(q0[q], q1[q], q2[q], nl, cn, sn, Kf, acc0);
        acc1 = pair_tap(q0[q + 1], q1[q + 1], q2[q + 1], nl, cn, sn, Kf, acc1);
    }
    if (q < qend) acc0 = pair_tap(q0[q], q1[q], q2[q], nl, cn, sn, Kf, acc0);
    return __fadd_rn(acc0, acc1);
}

__device__ __forceinline__ int lower_bound_s(const int* a, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int upper_bound_s(const int* a, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int NT>
__global__ void __launch_bounds__(NT, 3) synth_kernel(LaunchArgs a, const float* __restrict__ pos_hi,
                                                       const float* __restrict__ pos_lo, const float* __restrict__ gref,
                                                       float* __restrict__ rir, float* __restrict__ early)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = a.tile, K = a.K, Mg = a.margin_i;
    const SynthSmem L = synth_smem(T, K, Mg);
    const int NBK = L.nbk;
    int* sperm = reinterpret_cast<int*>(smem + L.sperm);
    int* skeys = reinterpret_cast<int*>(smem + L.skeys);
    int* rowb = reinterpret_cast<int*>(smem + L.rowb);
    float4* q0 = reinterpret_cast<float4*>(smem + L.q0);
    float4* q1 = reinterpret_cast<float4*>(smem + L.q1);
    float4* q2 = reinterpret_cast<float4*>(smem + L.q2);
    float* outt = reinterpret_cast<float*>(smem + L.outt);
    float2* tabT = reinterpret_cast<float2*>(smem + L.tabT);
    __shared__ int s_item, s_lo, s_hi;
    __shared__ float s_dir[6];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = NT / 32;
    const float invK = 1.0f / (float)K;
    const float Kf = (float)K;
    const int twoK = 2 * K;
    const int nrows = T / 32;
    const int n_items = a.hdr->n_items;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.hdr->queue, 1);
        __syncthreads();
        const int qi = s_item;
        if (qi >= n_items) break;
        const int2 it = a.items[qi];
        const int b = it.x, s = it.y >> 16, tau = it.y & 0xffff;
        const RoomConst rc = a.room[b];
        const int T0 = tau * T;
        const int Lb = rc.len;
        const int base = T0 - K - Mg - 1;          // sample index of phase-table entry 0
        const int64_t v0 = rc.vs_off + (int64_t)s * rc.n_vs;
        const int* bo = a.bin_off + ((int64_t)b * a.S + s) * (a.max_tiles + 1);
        const int kmin = T0 - K - Mg, kmax = T0 + T + K + Mg;   // keys that can reach the tile
        const int bin_lo = min(max(0, kmin >= 0 ? kmin / T : 0), rc.ntiles - 1);
        const int bin_hi = min(rc.ntiles - 1, kmax / T);
        const int c_lo = bo[bin_lo];
        int ncand = bo[bin_hi + 1] - c_lo;
        if (ncand > kStageCap) {
            if (tid == 0) atomicOr(&a.hdr->status, FRAM_DEV_CAPACITY);
            ncand = kStageCap;
        }
        // ---- stage the candidate images (sorted by key) and the phase table ----
        for (int j = tid; j < ncand; j += NT) {
            sperm[j] = a.perm[v0 + c_lo + j];
            skeys[j] = a.skey[v0 + c_lo + j];
        }
        for (int k = tid; k < NBK; k += NT) {
            int m = (base + k) % twoK;
            m = m < 0 ? m + twoK : m;
            float sn_, cs_;
            sincospif((float)m * invK, &sn_, &cs_);
            tabT[k] = make_float2(cs_, sn_);
        }
        __syncthreads();
        // ---- the tile's range and each row's range, by binary search on the keys ----
        if (tid == 0) s_lo = lower_bound_s(skeys, ncand, kmin);
        if (tid == 1) s_hi = upper_bound_s(skeys, ncand, kmax);
        if (tid >= 2 && tid < 2 + 2 * nrows) {
            const int r = (tid - 2) >> 1;
            const int R0 = T0 + 32 * r;
            rowb[tid - 2] = (tid & 1) ? upper_bound_s(skeys, ncand, R0 + 31 + K + Mg)
                                      : lower_bound_s(skeys, ncand, R0 - K - Mg);
        }
        __syncthreads();
        const int slo = s_lo, nst = max(0, s_hi - s_lo);
        const float log2r = rc.log2r;

        for (int m = 0; m < a.M; ++m) {
            const DirectConst dc = a.direct[((int64_t)b * a.S + s) * a.M + m];
            const float* pm = a.mic + 3 * ((size_t)b * a.M + m);
            const float mx = pm[0], my = pm[1], mz = pm[2];
            for (int k = tid; k < T; k += NT) outt[k] = 0.0f;
            const int nchunks = nst > 0 ? (nst + kArrCap - 1) / kArrCap : 1;
            for (int ch = 0; ch < nchunks; ++ch) {
                const int c0 = ch * kArrCap;
                const int nin = max(0, min(kArrCap, nst - c0));
                // ---- arrival records at their sorted positions ----
                for (int p = tid; p < nin; p += NT) {
                    const int i = sperm[slo + c0 + p];
                    const int64_t v = v0 + i;
                    const float* ph = pos_hi + 3 * v;
                    float plx = 0.f, ply = 0.f, plz = 0.f;
                    if (pos_lo) { plx = pos_lo[3 * v]; ply = pos_lo[3 * v + 1]; plz = pos_lo[3 * v + 2]; }
                    int nc;
                    float delta, D;
                    image_delay(ph[0], ph[1], ph[2], plx, ply, plz, mx, my, mz, a.q2, nc, delta, D);
                    const float A = exp2f(gref[v] * log2r) * rcp_approx(D);
                    const int key = nc - base;
                    float3 c = make_float3(0.f, 0.f, 0.f);
                    float ncl = (float)(T + 4 * K + 64);              // out of reach: zero weight
                    if (key >= 0 && key < NBK && D > 0.0f && A == A && fabsf(A) < 3.0e38f) {
                        if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
                        c = arrival_consts(nc, delta, A, tabT[key], invK);
                        ncl = (float)(nc - T0);
                    }
                    put_record(q0, q1, q2, p, ncl, delta, c);
                }
                if (tid == 0) {
                    if (nin & 1) put_record(q0, q1, q2, nin, (float)(T + 4 * K + 64), 0.25f, make_float3(0.f, 0.f, 0.f));
                    // Direct path of (b, s, m): its constants for the rows within reach.
                    const int nc = __float2int_rn(dc.t_hi);
                    float delta = __fadd_rn(__fsub_rn(dc.t_hi, (float)nc), dc.t_lo);
                    if (fabsf(delta) < kTinyDelta) delta = kTinyDelta;
                    const int key = nc - base;
                    float3 c = make_float3(0.f, 0.f, 0.f);
                    if (ch == 0 && key >= 0 && key < NBK) c = arrival_consts(nc, delta, dc.amp, tabT[key], invK);
                    s_dir[0] = (float)(nc - T0); s_dir[1] = delta; s_dir[2] = c.x; s_dir[3] = c.y; s_dir[4] = c.z;
                }
                __syncthreads();
                // ---- taps: each warp owns rows of 32 consecutive samples ----
                const float dnc = s_dir[0], dd = s_dir[1], dP = s_dir[2], da = s_dir[3], db = s_dir[4];
                for (int row = wid; row < nrows; row += NW) {
                    const int R0 = T0 + row * 32;
                    if (R0 >= Lb) break;
                    const int k0 = row * 32;
                    const int lo = max(rowb[2 * row] - slo - c0, 0);
                    const int hi = min(rowb[2 * row + 1] - slo - c0, nin);
                    const float2 cs = tabT[k0 + lane + K + Mg + 1];
                    const float nl = (float)(k0 + lane);
                    float acc = lo < hi ? row_taps(q0, q1, q2, lo >> 1, (hi + 1) >> 1, nl, cs.x, cs.y, Kf) : 0.0f;
                    if (dP != 0.0f && dnc >= (float)(k0 - K - 1) && dnc <= (float)(k0 + 32 + K)) {
                        const float e = __fadd_rn(__fsub_rn(dnc, nl), dd);
                        const float num = __fmaf_rn(cs.x, da, __fmaf_rn(cs.y, db, dP));
                        if (fabsf(e) < Kf) acc = __fadd_rn(acc, __fmul_rn(num, rcp_approx(e)));
                    }
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
        }
        __syncthreads();
    }
}

}  // namespace



int synth_smem_total(int T, int K, int M) { return synth_smem(T, K, M).total; }

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
        const int sm = (int)(sizeof(int) * 2 * (size_t)bin_warp_ints(a.max_tiles, a.tile));
        int per_sm = 0;
        if ((e = kernel_residency((const void*)bin_images, 64, sm, &per_sm)) != cudaSuccess) return e;
        bin_images<<<(unsigned)((segs + 1) / 2), 64, sm, st>>>(a, pos_hi);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_synthesize(const LaunchArgs& a, const float* pos_hi, const float* pos_lo, const float* g,
                              float* rir, float* early, cudaStream_t st)
{
    const int smem = synth_smem(a.tile, a.K, a.margin_i).total;
    int per_sm = 0;
    cudaError_t e = kernel_residency((const void*)synth_kernel<kSynthThreads>, kSynthThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = device_sm_count() * per_sm;
    synth_kernel<kSynthThreads><<<grid, kSynthThreads, smem, st>>>(a, pos_hi, pos_lo, g, rir, early);
    return cudaGetLastError();
}

}  // namespace fram
