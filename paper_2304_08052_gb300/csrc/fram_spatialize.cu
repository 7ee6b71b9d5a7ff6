// fram_spatialize.cu -- spatialisation of the RIRs, the paper's use of them for training data
// (Sec. IV-A): every source signal convolved with its M-channel RIR, speakers scaled to a
// signal-to-interference ratio against speaker 0, point-source noise to a signal-to-noise ratio
// against the speech at mic 0, all summed into the microphone mixture; optionally per-speaker
// targets through a second RIR set (the early RIR of Eq. 9 for dereverberation targets).
//
// Convolution: uniformly partitioned overlap-save in the frequency domain.  With block Bk and
// FFT length P = 2 Bk (real), the RIR of length L splits into Q = ceil(L / Bk) partitions
// h_q = h[q Bk, (q+1) Bk) and the signal into J = ceil(N / Bk) windows
// x_j = x[(j-1) Bk, (j+1) Bk); output block j (samples [j Bk, (j+1) Bk)) is the second half of
// IFFT(sum_q X_{j-q} H_q) (the first half wraps around).  Real transforms of length P run as
// complex transforms of length NC = P/2 = Bk on even/odd pairs, with the usual split
// post-processing; the half spectrum is stored as NC complex bins with the Nyquist bin's real
// part packed into the imaginary part of bin 0, so the bin-wise product is elementwise.  Bins are
// stored conjugate-paired (slot p: bins p and NC - p), so the inverse's pre-step, which combines
// k with NC - k, runs in the registers of the thread that summed both.
//
// The complex transform is one CTA's Stockham autosort FFT in shared memory: radix-16 stages
// (one 16-point DFT per thread and column, computed as 4 x 4 in registers), then one radix-8, -4
// or -2 stage; each stage reads all its inputs into registers, synchronises and writes, so one
// NC-element buffer suffices.  A forward transform's first stage starts from the registers the
// inputs were loaded into; an inverse transform's last stage writes the kept half of the window
// straight to the output.
//
// Pipeline per chunk of rooms (by default about 4 GiB of spectra, so every launch fills the GPU):
//   sp_forward  spectra of every signal window and RIR partition (and target-RIR partition)
//   sp_image0   mic-0 image of every source, block by block, with each block's energy (for the
//               levels)
//   sp_gains    per room: energies (from the blocks) and speech cross terms at mic 0 -> gains
//               (FP64)
//   sp_mix      per (room, mic, block): IFFT(sum_s g_s sum_q X H) -> mixture (mic 0 summed from
//               the images instead); per (room, speaker, mic, block): IFFT(g_s sum_q X H') ->
//               targets
#include <algorithm>
#include <cmath>

#include "fram_internal.cuh"

namespace fram {
namespace {

constexpr int kMaxTerms = 8 * 16;      // sources x RIR partitions per output block

struct SpArgs {
    int B, S, M, ns;
    int64_t N;
    int Bk, J, Q;
    int room0, rooms;
    bool sep;                      // targets use a second RIR set
    int max_len;
    int64_t rir_total;
    const int32_t* rir_len;
    const int64_t* rir_off;
    const float* rir;
    const float* trir;
    const float* x;                // [B,S,N]
    const float* level;            // [B,S] dB
    float* mix;                    // [B,M,N]
    float* tg;                     // [B,ns,M,N] or null
    float* gains;                  // [B,S]
    const float2* tw_c;            // exp(-2 pi i k / NC), k < NC
    const float2* tw_r;            // exp(-2 pi i k / P),  k < NC
    float2* XS;                    // [rooms][S][J][NC]
    float2* HS;                    // [rooms][S][M][Q][NC]
    float2* HT;                    // [rooms][ns][M][Q][NC] (== HS when !sep)
    int* XF;                       // 1 where the spectrum is nonzero (same indexing, one int each)
    int* HF;
    int* HTF;                      // (== HF when !sep)
    float* img0;                   // [rooms][S][N]
    double* eparts;                // [rooms][S][J]: energy of each block of img0
    Header* hdr;
};

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// a * (-i) for the forward transform, a * (+i) for the inverse
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Complex add / subtract as one packed FP32 instruction each (add/sub.rn.f32x2: both halves
// rounded exactly as the scalar operations).
__device__ __forceinline__ float2 p_add(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 p_sub(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// 4-point DFT: six of its eight complex additions go through packed FP32; the two that add the
// +-i-rotated difference d stay scalar (a packed operation cannot apply the (+, -) signs).
template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3)
{
    const float2 t0 = p_add(v0, v2), t1 = p_sub(v0, v2), t2 = p_add(v1, v3), d = p_sub(v1, v3);
    const float2 t3 = c_rot<INV>(d);
    v0 = p_add(t0, t2);
    v2 = p_sub(t0, t2);
    v1 = c_add(t1, t3);
    v3 = c_sub(t1, t3);
}

// v * (c, +-s): multiply by the constant e^(-+i theta) given as (cos theta, sin theta).
template <bool INV>
__device__ __forceinline__ float2 c_mulk(float2 v, float c, float s)
{
    const float t = INV ? s : -s;
    return make_float2(__fmaf_rn(v.x, c, -v.y * t), __fmaf_rn(v.x, t, v.y * c));
}

// 16-point DFT as 4 x 4: DFT4 over n1 of v[4 n1 + n2], twiddle by w16^(n2 k1), DFT4 over n2; the
// result X[k1 + 4 k2] is left in v[4 k1 + k2] (the caller stores with that transposed index).
template <bool INV>
__device__ __forceinline__ void dft16_t(float2* v)
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    v[5] = c_mulk<INV>(v[5], c1, s1);          // (n2, k1) = (1, 1): w^1
    v[9] = c_mulk<INV>(v[9], h, h);            // (1, 2): w^2
    v[13] = c_mulk<INV>(v[13], s1, c1);        // (1, 3): w^3
    v[6] = c_mulk<INV>(v[6], h, h);            // (2, 1): w^2
    v[10] = c_rot<INV>(v[10]);                 // (2, 2): w^4
    v[14] = c_mulk<INV>(v[14], -h, h);         // (2, 3): w^6
    v[7] = c_mulk<INV>(v[7], s1, c1);          // (3, 1): w^3
    v[11] = c_mulk<INV>(v[11], -h, h);         // (3, 2): w^6
    v[15] = c_mulk<INV>(v[15], -c1, -s1);      // (3, 3): w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 2) {
        const float2 a = v[0];
        v[0] = c_add(a, v[1]);
        v[1] = c_sub(a, v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 16) {
        dft16_t<INV>(v);
    } else {
        static_assert(R == 8, "radix 2, 4, 8 or 16");
        // Even and odd halves, then X[k] = E[k] + w^k O[k], X[k+4] = E[k] - w^k O[k], w = e^(-+2 pi i/8).
        dft4<INV>(v[0], v[2], v[4], v[6]);
        dft4<INV>(v[1], v[3], v[5], v[7]);
        constexpr float h = 0.70710678118654752f;
        const float2 o1 = v[3], o2 = v[5], o3 = v[7];
        const float2 w1 = INV ? make_float2((o1.x - o1.y) * h, (o1.x + o1.y) * h)
                              : make_float2((o1.x + o1.y) * h, (o1.y - o1.x) * h);
        const float2 w2 = c_rot<INV>(o2);
        const float2 w3 = INV ? make_float2((-o3.x - o3.y) * h, (o3.x - o3.y) * h)
                              : make_float2((o3.y - o3.x) * h, (-o3.x - o3.y) * h);
        const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = c_add(e0, o0);
        v[4] = c_sub(e0, o0);
        v[1] = c_add(e1, w1);
        v[5] = c_sub(e1, w1);
        v[2] = c_add(e2, w2);
        v[6] = c_sub(e2, w2);
        v[3] = c_add(e3, w3);
        v[7] = c_sub(e3, w3);
    }
}

// Shared-memory layout of the NC-point buffer: element e lives at e ^ ((e >> 4) & 15), a
// permutation inside each 16-element (128-byte) row, so that the strided writes of the first
// two stages spread over all banks while unit-stride accesses stay conflict-free.
__device__ __forceinline__ int sw(int e) { return e ^ ((e >> 4) & 15); }

// exp(-2 pi i k / NC) as TA[k >> 7] * TB[k & 127] from two small tables in shared memory.  TB
// entry i sits at i + i / 16 (one pad entry per 16): the stages look TB up at strides 1 to 128
// entries across a half-warp, which the plain layout folds onto 2 to 8 addresses of one bank
// pair, and the padded one spreads over distinct bank pairs (or one broadcast address).
__device__ __forceinline__ int tb_pos(int i) { return i + (i >> 4); }
struct Twiddles {
    const float2* TA;
    const float2* TB;
    __device__ __forceinline__ float2 operator()(int k) const { return c_mul(TA[k >> 7], TB[tb_pos(k & 127)]); }
};

// Destination of an inverse transform's kept half: complex point n >= NC/2 of the window holds
// real samples 2 (n - NC/2) and 2 (n - NC/2) + 1 of output block j, written times `scale` to
// out[base + 2 (n - NC/2) + {0, 1}] while the index is below N; pair stores when out is 8-byte
// aligned.  put() returns the sum of squares of the samples it wrote.
struct BlockStore {
    float* out;
    int64_t N, base;
    float scale;
    bool v2;
    __device__ __forceinline__ float put(int n, float2 z, int NC) const
    {
        const int64_t u = base + 2 * (int64_t)(n - NC / 2);
        const float a = z.x * scale, b = z.y * scale;
        float e = 0.f;
        if (v2 && u + 1 < N) {
            *reinterpret_cast<float2*>(out + u) = make_float2(a, b);
            e = __fmaf_rn(b, b, a * a);
        } else {
            if (u < N) {
                out[u] = a;
                e = a * a;
            }
            if (u + 1 < N) {
                out[u + 1] = b;
                e = __fmaf_rn(b, b, e);
            }
        }
        return e;
    }
};

// One Stockham stage of radix R over the NC-point buffer, stride Ns (the length already done).
// Column j takes buf[j + r NC/R] (r < R), twiddles them by w^(r (j mod Ns) NC/(Ns R)), runs an
// R-point DFT and writes buf[(j - j mod Ns) R + j mod Ns + r Ns].  With `bs` (last stage only,
// Ns R = NC) the outputs n = j + r Ns >= NC/2 go to the output block instead, and the stage ends
// without a barrier.
// With `vin` (first stage only, one column per thread) the column's inputs come from the
// thread's registers instead of the buffer, and no barrier precedes the writes.
template <int NC, int NT, int R, bool INV, int Ns>
__device__ __forceinline__ float fft_stage(float2* buf, const Twiddles& tw, const BlockStore* bs = nullptr,
                                           const float2* vin = nullptr)
{
    constexpr int NJ = NC / R;
    static_assert(NJ % NT == 0, "threads must divide the columns");
    static_assert(NJ % 256 == 0, "column stride keeps the swizzle bits");
    constexpr int PER = NJ / NT;
    float2 v[PER][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int j = tid + p * NT;
        const int sj = sw(j);                  // sw(j + r NJ) = sw(j) + r NJ: NJ is a multiple of 256
        if (Ns == 1 && PER == 1 && vin) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = vin[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = buf[sj + r * NJ];
        }
        if constexpr (Ns > 1) {
            // w^r for r < R from two table entries (w and w^4 for radix 8), at most 2 products deep
            const int step = (j & (Ns - 1)) * (NC / (Ns * R));
            auto get = [&](int k) {
                float2 w = tw(k);
                if (INV) w.y = -w.y;
                return w;
            };
            if constexpr (R == 16) {
                // w^1, w^2, w^4, w^8 from the tables, the rest as one product of two of them
                const float2 w1 = get(step), w2 = get(2 * step), w4 = get(4 * step), w8 = get(8 * step);
                const float2 w3 = c_mul(w1, w2), w12 = c_mul(w8, w4);
                v[p][1] = c_mul(v[p][1], w1);
                v[p][2] = c_mul(v[p][2], w2);
                v[p][3] = c_mul(v[p][3], w3);
                v[p][4] = c_mul(v[p][4], w4);
                v[p][5] = c_mul(v[p][5], c_mul(w4, w1));
                v[p][6] = c_mul(v[p][6], c_mul(w4, w2));
                v[p][7] = c_mul(v[p][7], c_mul(w4, w3));
                v[p][8] = c_mul(v[p][8], w8);
                v[p][9] = c_mul(v[p][9], c_mul(w8, w1));
                v[p][10] = c_mul(v[p][10], c_mul(w8, w2));
                v[p][11] = c_mul(v[p][11], c_mul(w8, w3));
                v[p][12] = c_mul(v[p][12], w12);
                v[p][13] = c_mul(v[p][13], c_mul(w12, w1));
                v[p][14] = c_mul(v[p][14], c_mul(w12, w2));
                v[p][15] = c_mul(v[p][15], c_mul(w12, w3));
            } else {
                float2 w[R];
                w[1] = get(step);
                if constexpr (R >= 4) {
                    w[2] = c_mul(w[1], w[1]);
                    w[3] = c_mul(w[2], w[1]);
                }
                if constexpr (R == 8) {
                    w[4] = get(4 * step);
                    w[5] = c_mul(w[4], w[1]);
                    w[6] = c_mul(w[4], w[2]);
                    w[7] = c_mul(w[4], w[3]);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) v[p][r] = c_mul(v[p][r], w[r]);
            }
        }
        dft<R, INV>(v[p]);
    }
    // output r of the DFT sits in v[p][r], or in v[p][4 (r % 4) + r / 4] after the 4 x 4 DFT16
    if constexpr (Ns * R == NC) {
        if (bs) {
            float e = 0.f;                           // sum of squares of the samples stored
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int j = tid + p * NT;          // j < Ns: the output base is j itself
#pragma unroll
                for (int r = R / 2; r < R; ++r) e += bs->put(j + r * Ns, R == 16 ? v[p][4 * (r & 3) + (r >> 2)] : v[p][r], NC);
            }
            return e;
        }
    }
    if (!(Ns == 1 && PER == 1 && vin)) __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int j = tid + p * NT;
        const int jm = j & (Ns - 1);
        const int base = (j - jm) * R + jm;
        auto out = [&](int r) { return R == 16 ? v[p][4 * (r & 3) + (r >> 2)] : v[p][r]; };
        if constexpr (Ns % 256 == 0) {
            const int sb = sw(base);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[sb + r * Ns] = out(r);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[sw(base + r * Ns)] = out(r);
        }
    }
    __syncthreads();
    return 0.f;
}

// In-place complex FFT of NC points (a power of two >= 8) in shared memory; the buffer must be
// complete (synchronised) on entry and is complete on exit.  Forward: X[k] = sum x[n] w^(nk),
// w = e^(-2 pi i/NC); inverse: w = e^(+2 pi i/NC), unscaled.  With `bs` the last stage writes
// the upper half of the result to the output block instead (the buffer is then left incomplete)
// and returns the sum of squares of the samples this thread stored (0 without `bs`).
// With `vin` the first stage (radix 16, one column j = thread per thread: NC = 16 NT) takes its
// inputs x[j + r NT], r < 16, from the thread's registers; the buffer is then not read first.
template <int NC, int NT, bool INV, int Ns = 1>
__device__ __forceinline__ float cfft(float2* buf, const Twiddles& tw, const BlockStore* bs = nullptr,
                                     const float2* vin = nullptr)
{
    static_assert(Ns > 1 || NC == 16 * NT || NC < 256, "register inputs need one first-stage column per thread");
    if constexpr (Ns * 16 == NC) {
        return fft_stage<NC, NT, 16, INV, Ns>(buf, tw, bs, vin);
    } else if constexpr (Ns * 16 < NC) {
        fft_stage<NC, NT, 16, INV, Ns>(buf, tw, nullptr, vin);
        return cfft<NC, NT, INV, Ns * 16>(buf, tw, bs);
    } else if constexpr (Ns * 8 == NC) {
        return fft_stage<NC, NT, 8, INV, Ns>(buf, tw, bs);
    } else if constexpr (Ns * 4 == NC) {
        return fft_stage<NC, NT, 4, INV, Ns>(buf, tw, bs);
    } else {
        static_assert(Ns * 2 == NC, "power-of-two length");
        return fft_stage<NC, NT, 2, INV, Ns>(buf, tw, bs);
    }
}

__global__ void sp_twiddles(float2* tw_c, float2* tw_r, int NC)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NC) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)NC, &s, &c);
    tw_c[k] = make_float2((float)c, (float)s);
    sincospi(-(double)k / (double)NC, &s, &c);
    tw_r[k] = make_float2((float)c, (float)s);
}

// The two twiddle tables of the NC-point transform, copied from the global table into shared
// memory (valid after the caller's next __syncthreads).
template <int NC, int NT>
__device__ __forceinline__ Twiddles load_twiddles(const float2* __restrict__ tw_c)
{
    static_assert(NC >= 128 && NC / 128 <= 128, "two-level table covers 128 x 128 entries");
    __shared__ float2 ta[NC / 128], tb[128 + 8];
    for (int i = threadIdx.x; i < 128; i += NT) {
        tb[tb_pos(i)] = __ldg(&tw_c[i]);
        if (i < NC / 128) ta[i] = __ldg(&tw_c[i * 128]);
    }
    return Twiddles{ta, tb};
}

// Spectra: one CTA per signal window, RIR partition or target-RIR partition of the chunk.
// Residency at NC = 4096: five CTAs per SM (48 registers) for every transform kernel.  With the
// first stage fed from registers, six here spilled the 16 inputs (10.84 against 10.76 ms per
// batch_1024); before that six here beat five (12.82 ms), and four for all (64 registers) took
// 13.33, six for all 13.39.
template <int NC, int NT>
__global__ void __launch_bounds__(NT, NC == 4096 ? 5 : (NC == 8192 ? 2 : 1)) sp_forward(SpArgs A)
{
    extern __shared__ __align__(16) float2 sp_buf[];
    const int nsig = A.rooms * A.S * A.J;
    const int nrir = A.rooms * A.S * A.M * A.Q;
    int jid = blockIdx.x;
    const float* src;
    int64_t start, len;
    int lim;               // window samples taken from the source (the rest are zero)
    float2* dst;
    int* flag;
    if (jid < nsig) {
        const int cb = jid / (A.S * A.J), s = (jid / A.J) % A.S, j = jid % A.J;
        src = A.x + ((int64_t)(A.room0 + cb) * A.S + s) * A.N;
        start = (int64_t)(j - 1) * A.Bk;
        len = A.N;
        lim = 2 * A.Bk;
        dst = A.XS + (int64_t)jid * NC;
        flag = A.XF + jid;
    } else {
        jid -= nsig;
        const bool tgt = jid >= nrir;
        if (tgt) jid -= nrir;
        const int ss = tgt ? A.ns : A.S;
        const int cb = jid / (ss * A.M * A.Q), s = (jid / (A.M * A.Q)) % ss, m = (jid / A.Q) % A.M,
                  q = jid % A.Q;
        const int b = A.room0 + cb;
        const int L = A.rir_len[b];
        const int64_t off = A.rir_off[b] + ((int64_t)s * A.M + m) * L;
        if (L < 1 || L > A.max_len || off < 0 || off + L > A.rir_total) {   // layout disagrees with the host
            if (threadIdx.x == 0) atomicOr(&A.hdr->status, FRAM_DEV_BAD_GEOMETRY);
            len = 0;
        } else {
            len = L;
        }
        src = (tgt ? A.trir : A.rir) + (len ? off : 0);
        start = (int64_t)q * A.Bk;
        lim = A.Bk;
        dst = (tgt ? A.HT : A.HS) + (int64_t)jid * NC;
        flag = (tgt ? A.HTF : A.HF) + jid;
    }
    // Thread j's points j + r NT (r < 16) are exactly the first radix-16 stage's column j, so
    // they stay in registers.
    static_assert(NC == 16 * NT, "one first-stage column per thread");
    bool nonzero = false;
    float2 vin[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = threadIdx.x + r * NT;
        const int t0 = 2 * n, t1 = 2 * n + 1;
        const int64_t i0 = start + t0, i1 = start + t1;
        const float a = (t0 < lim && i0 >= 0 && i0 < len) ? src[i0] : 0.f;
        const float b = (t1 < lim && i1 >= 0 && i1 < len) ? src[i1] : 0.f;
        vin[r] = make_float2(a, b);
        nonzero = nonzero || a != 0.0f || b != 0.0f;
    }
    const Twiddles tw = load_twiddles<NC, NT>(A.tw_c);
    // An all-zero window (a silent stretch of a source, an RIR partition past its end) has a zero
    // spectrum: it is flagged and skipped by every sum that would read it.  (The barrier also
    // completes the twiddle tables.)
    const int nz = __syncthreads_or(nonzero ? 1 : 0);
    if (threadIdx.x == 0) *flag = nz;
    if (!nz) return;
    cfft<NC, NT, false>(sp_buf, tw, nullptr, vin);
    // Split: with Zc = conj(Z[NC-k]), E = (Z[k] + Zc)/2, O = -i (Z[k] - Zc)/2,
    // X[k] = E + w_P^k O and X[NC-k] = conj(E - w_P^k O).  Stored in the paired layout: slot
    // p < NC/2 holds (X[p], X[NC-p]), slot 0 (X[0] packed as (DC, Nyquist), X[NC/2]).
    float4* dst4 = reinterpret_cast<float4*>(dst);
    for (int k = threadIdx.x; k < NC / 2; k += NT) {
        const int kk = k == 0 ? NC / 2 : k;
        const float2 zk = sp_buf[sw(kk)], zc = c_conj(sp_buf[sw(NC - kk)]);
        const float2 E = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 D = c_sub(zk, zc);
        const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
        const float2 WO = c_mul(__ldg(&A.tw_r[kk]), O);
        const float2 Xk = c_add(E, WO);
        if (k == 0) {
            const float2 z = sp_buf[sw(0)];
            dst4[0] = make_float4(z.x + z.y, z.x - z.y, Xk.x, Xk.y);      // (DC, Nyquist), X[NC/2]
        } else {
            const float2 Xc = c_conj(c_sub(E, WO));
            dst4[k] = make_float4(Xk.x, Xk.y, Xc.x, Xc.y);
        }
    }
}

__device__ __forceinline__ float2 packed_mul(float2 a, float2 b, bool dc)
{
    return dc ? make_float2(a.x * b.x, a.y * b.y) : c_mul(a, b);
}

// One term g X H of an output block's spectral sum.
struct SpTerm {
    const float2* X;
    const float2* H;
    float g;
};

// sp_buf <- the packed spectrum Z of the real inverse transform of Y = sum_t g_t X_t H_t over nt
// terms (spectra in the paired layout: slot p holds bins p and NC - p, slot 0 bins 0 (DC and
// Nyquist packed) and NC/2).  Each thread owns slots p = tid + i NT, loaded as float4 with all of
// a term's loads in flight before the products; accumulators stay in registers, in term order
// (deterministic).  Both bins of a conjugate pair are then in one thread, so the pre-step of the
// half-length real inverse runs in registers: with Yc = conj(Y[NC-k]), E = (Y[k] + Yc)/2,
// O = (Y[k] - Yc)/2 conj(w_P^k), Z[k] = E + i O and Z[NC-k] = conj(E - i O); Z[0] from the
// packed DC and Nyquist.  The real sample t of the window is afterwards the unscaled inverse
// transform of Z at t/2 (.x even t, .y odd t), times 1/NC.
template <int NC, int NT>
__device__ __forceinline__ void spectral_sum(float2* sp_buf, const SpTerm* terms, int nt, const float2* __restrict__ tw_r)
{
    constexpr int KP = NC / (2 * NT);          // slots per thread
    constexpr int KH = KP >= 2 ? 2 : KP;       // slots per pass (four spilled at five CTAs per SM)
    static_assert(KP % KH == 0, "slots per pass must divide the slots per thread");
#pragma unroll 1
    for (int h0 = 0; h0 < KP; h0 += KH) {
        float4 acc[KH];
#pragma unroll
        for (int i = 0; i < KH; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int t = 0; t < nt; ++t) {
            const float4* X4 = reinterpret_cast<const float4*>(terms[t].X);
            const float4* H4 = reinterpret_cast<const float4*>(terms[t].H);
            const float g = terms[t].g;
            float4 xv[KH], hv[KH];
#pragma unroll
            for (int i = 0; i < KH; ++i) {
                const int p = threadIdx.x + (h0 + i) * NT;
                xv[i] = __ldg(&X4[p]);
                hv[i] = __ldg(&H4[p]);
            }
#pragma unroll
            for (int i = 0; i < KH; ++i) {
                const int p = threadIdx.x + (h0 + i) * NT;
                const float2 a = packed_mul(make_float2(xv[i].x, xv[i].y), make_float2(hv[i].x, hv[i].y), p == 0);
                const float2 b = c_mul(make_float2(xv[i].z, xv[i].w), make_float2(hv[i].z, hv[i].w));
                acc[i].x = __fmaf_rn(g, a.x, acc[i].x);
                acc[i].y = __fmaf_rn(g, a.y, acc[i].y);
                acc[i].z = __fmaf_rn(g, b.x, acc[i].z);
                acc[i].w = __fmaf_rn(g, b.y, acc[i].w);
            }
        }
#pragma unroll
        for (int i = 0; i < KH; ++i) {
            const int p = threadIdx.x + (h0 + i) * NT;
            // pair (k, NC - k): k = p, or NC/2 (self-paired) in slot 0, whose first bin is DC / Nyquist
            const int k = p == 0 ? NC / 2 : p;
            const float2 xk = p == 0 ? make_float2(acc[i].z, acc[i].w) : make_float2(acc[i].x, acc[i].y);
            const float2 xc = make_float2(acc[i].z, -acc[i].w);
            const float2 E = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y + xc.y));
            const float2 D = c_sub(xk, xc);
            const float2 O = c_mul(make_float2(0.5f * D.x, 0.5f * D.y), c_conj(__ldg(&tw_r[k])));
            sp_buf[sw(k)] = make_float2(E.x - O.y, E.y + O.x);                       // E + i O
            if (p == 0) sp_buf[sw(0)] = make_float2(0.5f * (acc[i].x + acc[i].y), 0.5f * (acc[i].x - acc[i].y));
            else sp_buf[sw(NC - k)] = make_float2(E.x + O.y, O.x - E.y);               // conj(E - i O)
        }
    }
}

// Writes zeros to output block j (every term of its sum was a zero spectrum).
template <int NC, int NT>
__device__ __forceinline__ void store_zero_block(float* out, int64_t N, int j)
{
    const int64_t base = (int64_t)j * NC;
    for (int u = threadIdx.x; u < NC; u += NT)
        if (base + u < N) out[base + u] = 0.0f;
}

// Term list of one output block, built by all threads at once: thread i < ncand tests candidate
// i (cand(i, term) loads its flags and gain and returns whether the term is nonzero), so the
// flag loads of all candidates are in flight together instead of one after another in a single
// thread; the nonzero terms are compacted in candidate order.  Returns the number of terms, in
// every thread; synchronises.
template <int NT, typename Cand>
__device__ __forceinline__ int build_terms(SpTerm* terms, int ncand, Cand cand)
{
    static_assert(NT >= kMaxTerms, "one candidate per thread");
    __shared__ int wcnt[NT / 32];
    SpTerm t{};
    const bool ok = (int)threadIdx.x < ncand && cand((int)threadIdx.x, t);
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int u = 0; u < NT / 32; ++u) {
        const int c = wcnt[u];
        base += u < w ? c : 0;
        total += c;
    }
    if (ok) terms[base + __popc(bal & ((1u << lane) - 1u))] = t;
    __syncthreads();
    return total;
}

// Mic-0 image of every (room, source), block by block.
template <int NC, int NT>
__global__ void __launch_bounds__(NT, NC == 4096 ? 5 : (NC == 8192 ? 2 : 1)) sp_image0(SpArgs A)
{
    extern __shared__ __align__(16) float2 sp_buf[];
    const int jid = blockIdx.x;
    const int cb = jid / (A.S * A.J), s = (jid / A.J) % A.S, j = jid % A.J;
    __shared__ SpTerm terms[kMaxTerms];
    const int64_t xi = ((int64_t)cb * A.S + s) * A.J, hi = (((int64_t)cb * A.S + s) * A.M) * A.Q;   // mic 0
    const Twiddles tw = load_twiddles<NC, NT>(A.tw_c);
    // nonzero terms only, in q order
    const int nt = build_terms<NT>(terms, min(A.Q, j + 1), [&](int q, SpTerm& t) {
        const bool nz = (A.XF[xi + j - q] != 0) & (A.HF[hi + q] != 0);
        t = SpTerm{A.XS + (xi + j - q) * NC, A.HS + (hi + q) * NC, 1.0f};
        return nz;
    });
    float* out = A.img0 + ((int64_t)cb * A.S + s) * A.N;
    double* ep = A.eparts + ((int64_t)cb * A.S + s) * A.J + j;
    if (nt == 0) {
        store_zero_block<NC, NT>(out, A.N, j);
        if (threadIdx.x == 0) *ep = 0.0;
        return;
    }
    spectral_sum<NC, NT>(sp_buf, terms, nt, A.tw_r);
    __syncthreads();
    const BlockStore bs{out, A.N, (int64_t)j * NC, 1.0f / NC, (reinterpret_cast<uintptr_t>(out) & 7) == 0};
    // the block's energy for the levels: each thread's FP32 sum of squares of the samples it
    // stored, added in FP64 across the warp (fixed tree) and across warps in warp order
    double e = cfft<NC, NT, true>(sp_buf, tw, &bs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    __shared__ double ew[NT / 32];
    if ((threadIdx.x & 31) == 0) ew[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += ew[w];
        *ep = t;
    }
}

constexpr int kGainThreads = 512;

// Sums over n < N of y_a[n] y_b[n] for nq <= NQ pairs (a[q], b[q]) at once, into out[q]
// (shared, written by thread 0).  Each thread takes samples n = tid + k kGainThreads in runs of
// 32, summed in FP32 per run and in FP64 across runs; the warps' FP64 sums are then added in warp
// order.  Every pair's loads of one sample are independent, so a pass keeps 2 NQ loads in flight
// per sample.
template <int NQ>
__device__ void pair_sums(const float* __restrict__ y, int64_t N, const int* a, const int* b, int nq, double* red,
                          double* out)
{
    const float* ya[NQ];
    const float* yb[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        ya[q] = y + (int64_t)a[q] * N;
        yb[q] = y + (int64_t)b[q] * N;
    }
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (int64_t n0 = threadIdx.x; n0 < N; n0 += 32 * (int64_t)kGainThreads) {
        const int cnt = (int)min((int64_t)32, (N - n0 + kGainThreads - 1) / kGainThreads);
        float part[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) part[q] = 0.f;
#pragma unroll 4
        for (int kk = 0; kk < cnt; ++kk) {
            const int64_t n = n0 + (int64_t)kk * kGainThreads;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < nq) {
                    const float u = __ldg(ya[q] + n);
                    const float v = __ldg(yb[q] + n);
                    part[q] = __fmaf_rn(u, v, part[q]);
                }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] += part[q];
    }
    constexpr int NW = kGainThreads / 32;
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q * NW + w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < nq; ++q) {
            double t = 0.0;
            for (int i = 0; i < NW; ++i) t += red[q * NW + i];
            out[q] = t;
        }
    __syncthreads();
}

// Per room: E_s = sum y_s0^2 from the block energies sp_image0 left (added in block order), the
// speech cross terms (pairs s < t < n_speech, four per pass over the images), then the gains
// (FP64, as the levels define them).
__global__ void __launch_bounds__(kGainThreads) sp_gains(SpArgs A)
{
    __shared__ double red[4 * (kGainThreads / 32)];
    __shared__ double E[8], Cx[8][8], tmp[4];
    const int cb = blockIdx.x;
    const float* y = A.img0 + (int64_t)cb * A.S * A.N;
    if (threadIdx.x < A.S) {
        const double* ep = A.eparts + ((int64_t)cb * A.S + threadIdx.x) * A.J;
        double t = 0.0;
        for (int j = 0; j < A.J; ++j) t += ep[j];
        E[threadIdx.x] = t;
    }
    __syncthreads();
    const int npairs = A.ns * (A.ns - 1) / 2;
    for (int p0 = 0; p0 < npairs; p0 += 4) {
        int a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {       // pair p0 + i in (s, t) order, s < t < n_speech
            int p = min(p0 + i, npairs - 1), s = 0;
            while (p >= A.ns - 1 - s) { p -= A.ns - 1 - s; ++s; }
            a[i] = s;
            b[i] = s + 1 + p;
        }
        pair_sums<4>(y, A.N, a, b, min(4, npairs - p0), red, tmp);
        if (threadIdx.x == 0)
            for (int i = 0; i < min(4, npairs - p0); ++i) Cx[a[i]][b[i]] = Cx[b[i]][a[i]] = tmp[i];
    }
    if (threadIdx.x == 0) {
        const int b = A.room0 + cb;
        double g[8];
        g[0] = 1.0;
        for (int s = 1; s < A.ns; ++s)
            g[s] = E[s] > 0.0 ? sqrt(E[0] / E[s] * pow(10.0, -(double)A.level[(int64_t)b * A.S + s] / 10.0)) : 0.0;
        double Ev = 0.0;
        for (int s = 0; s < A.ns; ++s)
            for (int t = 0; t < A.ns; ++t) Ev += g[s] * g[t] * (s == t ? E[s] : Cx[s][t]);
        for (int s = A.ns; s < A.S; ++s)
            g[s] = E[s] > 0.0 ? sqrt(Ev / E[s] * pow(10.0, -(double)A.level[(int64_t)b * A.S + s] / 10.0)) : 0.0;
        for (int s = 0; s < A.S; ++s) A.gains[(int64_t)b * A.S + s] = (float)g[s];
    }
}

// Mixture blocks (room, mic, block) and target blocks (room, speaker, mic, block).
template <int NC, int NT>
__global__ void __launch_bounds__(NT, NC == 4096 ? 5 : (NC == 8192 ? 2 : 1)) sp_mix(SpArgs A)
{
    extern __shared__ __align__(16) float2 sp_buf[];
    const int nmix = A.rooms * A.M * A.J;
    int jid = blockIdx.x;
    const bool tgt = jid >= nmix;
    int cb, s0, s1, m, j;
    if (!tgt) {
        cb = jid / (A.M * A.J); m = (jid / A.J) % A.M; j = jid % A.J;
        s0 = 0; s1 = A.S;
    } else {
        jid -= nmix;
        cb = jid / (A.ns * A.M * A.J); s0 = (jid / (A.M * A.J)) % A.ns; m = (jid / A.J) % A.M; j = jid % A.J;
        s1 = s0 + 1;
    }
    const int b = A.room0 + cb;
    if (!tgt && m == 0) {
        // Mixture at mic 0: sum_s g_s y_s0, the mic-0 images sp_image0 already transformed (the
        // inverse transform is linear), summed in the time domain in source order.
        float* out = A.mix + ((int64_t)b * A.M) * A.N;
        const float* img = A.img0 + (int64_t)cb * A.S * A.N;
        const int64_t base = (int64_t)j * NC;
        for (int u = threadIdx.x; u < NC; u += NT) {
            const int64_t n = base + u;
            if (n >= A.N) break;
            float acc = 0.0f;
            for (int s2 = 0; s2 < A.S; ++s2) acc = __fmaf_rn(A.gains[(int64_t)b * A.S + s2], img[(int64_t)s2 * A.N + n], acc);
            out[n] = acc;
        }
        return;
    }
    const float2* Hb = tgt ? A.HT : A.HS;
    const int hs = (tgt && A.sep) ? A.ns : A.S;
    __shared__ SpTerm terms[kMaxTerms];
    const int* Hf = tgt ? A.HTF : A.HF;
    const Twiddles tw = load_twiddles<NC, NT>(A.tw_c);
    // nonzero terms only, in (source, q) order: candidate i is source s0 + i / nq, partition i % nq
    const int nq = min(A.Q, j + 1);
    const int nt = build_terms<NT>(terms, (s1 - s0) * nq, [&](int i, SpTerm& t) {
        const int s = s0 + i / nq, q = i - (i / nq) * nq;
        const float g = A.gains[(int64_t)b * A.S + s];
        const int64_t xi = ((int64_t)cb * A.S + s) * A.J + (j - q);
        const int64_t hi = (((int64_t)cb * hs + s) * A.M + m) * A.Q + q;
        const bool nz = (g != 0.0f) & (A.XF[xi] != 0) & (Hf[hi] != 0);
        t = SpTerm{A.XS + xi * NC, Hb + hi * NC, g};
        return nz;
    });
    float* out = tgt ? A.tg + (((int64_t)b * A.ns + s0) * A.M + m) * A.N : A.mix + ((int64_t)b * A.M + m) * A.N;
    if (nt == 0) {
        store_zero_block<NC, NT>(out, A.N, j);
        return;
    }
    spectral_sum<NC, NT>(sp_buf, terms, nt, A.tw_r);
    __syncthreads();
    const BlockStore bs{out, A.N, (int64_t)j * NC, 1.0f / NC, (reinterpret_cast<uintptr_t>(out) & 7) == 0};
    cfft<NC, NT, true>(sp_buf, tw, &bs);
}

template <int NC, int NT>
cudaError_t launch_chunk(const SpArgs& A, cudaStream_t st)
{
    const int smem = NC * (int)sizeof(float2);
    int per_sm = 0;
    cudaError_t e;
    if ((e = kernel_residency((const void*)sp_forward<NC, NT>, NT, smem, &per_sm)) != cudaSuccess) return e;
    if ((e = kernel_residency((const void*)sp_image0<NC, NT>, NT, smem, &per_sm)) != cudaSuccess) return e;
    if ((e = kernel_residency((const void*)sp_mix<NC, NT>, NT, smem, &per_sm)) != cudaSuccess) return e;
    const int nfwd = A.rooms * (A.S * A.J + A.S * A.M * A.Q + (A.sep ? A.ns * A.M * A.Q : 0));
    sp_forward<NC, NT><<<nfwd, NT, smem, st>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sp_image0<NC, NT><<<A.rooms * A.S * A.J, NT, smem, st>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sp_gains<<<A.rooms, kGainThreads, 0, st>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nmix = A.rooms * A.J * A.M * (1 + (A.tg ? A.ns : 0));
    sp_mix<NC, NT><<<nmix, NT, smem, st>>>(A);
    return cudaGetLastError();
}

struct SpLayout {
    int Bk, J, Q, chunk;
    bool sep;
    size_t header, tw_c, tw_r, XS, HS, HT, XF, HF, HTF, img0, eparts, gains, total;
};

// Default block: 4096 (the smallest transform: more CTAs per SM hide the stage barriers better
// than fewer, larger transforms, even though each output block then sums more partitions),
// larger only when the sources x partitions exceed the term limit.
int auto_block(int S, int Lmax)
{
    for (int Bk = 4096; Bk < 16384; Bk *= 2)
        if ((int64_t)S * ((Lmax + Bk - 1) / Bk) <= kMaxTerms) return Bk;
    return 16384;
}

SpLayout sp_layout(const fram_scene& sc, const fram_spatial& sp, bool sep)
{
    SpLayout w{};
    const int Lmax = std::max(sc.max_len, 1);
    w.Bk = sp.block ? sp.block : auto_block(sc.S, Lmax);
    w.J = (int)((sp.n_samples + w.Bk - 1) / w.Bk);
    w.Q = (Lmax + w.Bk - 1) / w.Bk;
    w.sep = sep;
    const size_t spec = sizeof(float2) * (size_t)w.Bk;
    const size_t per_room = spec * ((size_t)sc.S * w.J + (size_t)sc.S * sc.M * w.Q +
                                    (sep ? (size_t)sp.n_speech * sc.M * w.Q : 0)) +
                            sizeof(float) * (size_t)sc.S * (size_t)sp.n_samples;
    int chunk = sp.chunk_rooms;
    if (chunk <= 0) {
        // Large chunks: each kernel needs thousands of CTAs to fill 152 SMs; the spectra then
        // stream through HBM rather than staying in L2, which costs less than idle SMs.
        const size_t target = (size_t)4 << 30;
        chunk = (int)std::max<size_t>(1, target / std::max<size_t>(per_room, 1));
        // equal chunks (e.g. 512 + 512 rooms rather than 690 + 334), so no launch runs half full
        const int nchunks = (std::max(sc.B, 1) + chunk - 1) / chunk;
        chunk = (std::max(sc.B, 1) + nchunks - 1) / nchunks;
    }
    w.chunk = std::max(1, std::min(chunk, std::max(sc.B, 1)));
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off += (n + 255) & ~(size_t)255;
        return o;
    };
    const size_t C = (size_t)w.chunk;
    w.header = take(sizeof(Header));
    w.tw_c = take(spec);
    w.tw_r = take(spec);
    w.XS = take(spec * C * sc.S * w.J);
    w.HS = take(spec * C * sc.S * sc.M * w.Q);
    w.HT = sep ? take(spec * C * sp.n_speech * sc.M * w.Q) : w.HS;
    w.XF = take(sizeof(int) * C * sc.S * w.J);
    w.HF = take(sizeof(int) * C * sc.S * sc.M * w.Q);
    w.HTF = sep ? take(sizeof(int) * C * sp.n_speech * sc.M * w.Q) : w.HF;
    w.img0 = take(sizeof(float) * C * sc.S * (size_t)sp.n_samples);
    w.eparts = take(sizeof(double) * C * sc.S * w.J);
    w.gains = take(sizeof(float) * (size_t)std::max(sc.B, 1) * sc.S);
    w.total = off;
    return w;
}

int sp_check(const fram_scene* sc, const fram_spatial* sp)
{
    if (!sc || !sp) return record_error(FRAM_EINVAL, "scene and spatial parameters must not be null");
    if (sc->B < 0 || sc->S < 1 || sc->M < 1) return record_error(FRAM_EINVAL, "need B >= 0, S >= 1, M >= 1");
    if (sc->S > 8) return record_error(FRAM_EINVAL, "spatialisation takes at most 8 sources per room");
    if (sc->B > 0 && sc->max_len < 1) return record_error(FRAM_EINVAL, "max_len must be >= 1");
    if (sp->n_samples < 1 || sp->n_samples > 0x7fffffffLL) return record_error(FRAM_EINVAL, "n_samples must be in [1, 2^31)");
    if (sp->n_speech < 1 || sp->n_speech > sc->S) return record_error(FRAM_EINVAL, "need 1 <= n_speech <= S");
    if (sp->block != 0 && sp->block != 4096 && sp->block != 8192 && sp->block != 16384)
        return record_error(FRAM_EINVAL, "block must be 0, 4096, 8192 or 16384");
    if (sp->chunk_rooms < 0) return record_error(FRAM_EINVAL, "chunk_rooms must be >= 0");
    {
        const int Lmax = std::max(sc->max_len, 1);
        const int Bk = sp->block ? sp->block : auto_block(sc->S, Lmax);
        if ((int64_t)sc->S * ((Lmax + Bk - 1) / Bk) > kMaxTerms)
            return record_error(FRAM_EINVAL, "S x RIR partitions exceeds 128 (raise block)");
    }
    return FRAM_OK;
}

}  // namespace
}  // namespace fram

using namespace fram;

extern "C" int fram_spatialize_workspace_size(const fram_scene* scene, const fram_spatial* sp, int32_t separate_targets,
                                              size_t* bytes)
{
    int rc = sp_check(scene, sp);
    if (rc != FRAM_OK) return rc;
    if (!bytes) return record_error(FRAM_EINVAL, "bytes is null");
    *bytes = sp_layout(*scene, *sp, separate_targets != 0).total;
    return FRAM_OK;
}

extern "C" int fram_spatialize(const fram_scene* scene, const fram_spatial* sp, const float* rir,
                               const float* target_rir, const float* signals, const float* level_db, float* mixture,
                               float* targets, float* gains, void* workspace, size_t workspace_bytes, void* stream)
{
    int rc = sp_check(scene, sp);
    if (rc != FRAM_OK) return rc;
    const bool sep = targets && target_rir && target_rir != rir;
    const SpLayout w = sp_layout(*scene, *sp, sep);
    if (!workspace) return record_error(FRAM_EWORKSPACE, "workspace is null");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return record_error(FRAM_EWORKSPACE, "workspace must be 256-byte aligned");
    if (workspace_bytes < w.total) return record_error(FRAM_EWORKSPACE, "workspace too small for fram_spatialize");
    if (scene->B == 0) return FRAM_OK;
    if (!scene->rir_len || !scene->rir_off) return record_error(FRAM_EINVAL, "scene rir_len / rir_off must not be null");
    if (!rir || !signals || !level_db || !mixture) return record_error(FRAM_EINVAL, "rir, signals, level_db and mixture must not be null");
    if (targets && !target_rir) return record_error(FRAM_EINVAL, "targets need target_rir (pass rir for reverberant targets)");
    char* base = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SpArgs A{};
    A.B = scene->B; A.S = scene->S; A.M = scene->M; A.ns = sp->n_speech;
    A.N = sp->n_samples;
    A.Bk = w.Bk; A.J = w.J; A.Q = w.Q;
    A.sep = sep;
    A.max_len = scene->max_len;
    A.rir_total = scene->rir_total;
    A.rir_len = scene->rir_len; A.rir_off = scene->rir_off;
    A.rir = rir; A.trir = targets ? target_rir : rir;
    A.x = signals; A.level = level_db; A.mix = mixture; A.tg = targets;
    A.gains = gains ? gains : reinterpret_cast<float*>(base + w.gains);
    A.tw_c = reinterpret_cast<const float2*>(base + w.tw_c);
    A.tw_r = reinterpret_cast<const float2*>(base + w.tw_r);
    A.XS = reinterpret_cast<float2*>(base + w.XS);
    A.HS = reinterpret_cast<float2*>(base + w.HS);
    A.HT = reinterpret_cast<float2*>(base + w.HT);
    A.img0 = reinterpret_cast<float*>(base + w.img0);
    A.eparts = reinterpret_cast<double*>(base + w.eparts);
    A.XF = reinterpret_cast<int*>(base + w.XF);
    A.HF = reinterpret_cast<int*>(base + w.HF);
    A.HTF = reinterpret_cast<int*>(base + w.HTF);
    A.hdr = reinterpret_cast<Header*>(base + w.header);
    cudaError_t e = cudaMemsetAsync(A.hdr, 0, sizeof(Header), st);
    if (e != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    sp_twiddles<<<(w.Bk + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2*>(base + w.tw_c),
                                                    reinterpret_cast<float2*>(base + w.tw_r), w.Bk);
    if ((e = cudaGetLastError()) != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    for (int r0 = 0; r0 < scene->B; r0 += w.chunk) {
        A.room0 = r0;
        A.rooms = std::min(w.chunk, scene->B - r0);
        if (w.Bk == 4096) e = launch_chunk<4096, 256>(A, st);
        else if (w.Bk == 8192) e = launch_chunk<8192, 512>(A, st);
        else e = launch_chunk<16384, 1024>(A, st);
        if (e != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    }
    return FRAM_OK;
}
