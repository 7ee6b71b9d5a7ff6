/*
 * fram.h -- C ABI of libfram: batched multi-channel room impulse response synthesis after
 * FRAM-RIR (Y. Luo, R. Gu, "Fast Random Approximation of Multi-channel Room Impulse
 * Response", arXiv 2304.08052), for NVIDIA GB300 (sm_103a).
 *
 * Problem statement (Sec. II-III): for every room (shoebox dimensions, T60), source and
 * microphone, the RIR is the sum of a direct path and I randomly placed virtual image sources.
 * Image i has a sampled distance D_i from the array centre (Eq. 3, 4), a uniformly sampled
 * direction (Sec. III-B) and a reflection count g_i (Eq. 5, 6); it reaches mic m after
 * D_{i,m} = |p_i - mic_m| metres with amplitude r^{g_i} / D_{i,m} (Eq. 1, 2).  Each arrival
 * is rendered at the output rate fs as a fractional-delay Hann-windowed sinc of half length
 * K centred on t = D_{i,m} fs / c0, and the early RIR (Eq. 9) keeps the samples within
 * [-pre, +post] ms of the direct path.
 *
 * Conventions for every entry point:
 *   - All array pointers are device pointers unless the comment says "host".  The caller
 *     owns every buffer; libfram never allocates device or pinned memory.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream) and returns without synchronising, so the calls can be captured in a CUDA
 *     graph.  Only fram_status() synchronises.
 *   - Errors detected on the host return a negative code and set a thread-local message
 *     (fram_last_error).  Errors detected on the device (invalid geometry, capacity
 *     overflow, non-finite input) set bits of a status word in the workspace, reported by
 *     fram_status().
 *   - Floating-point data are float32; geometry is in metres, time in seconds.
 *
 * Buffer layout (ragged, produced by fram_layout on the host):
 *   room b has L_b = ceil(T60_b * fs) samples per channel and S * n_vs[b] images;
 *   rir[rir_off[b] + (s*M + m)*L_b + n]   for n in [0, L_b)
 *   image (b, s, i) is row vs_off[b] + s*n_vs[b] + i of the image arrays.
 */
#ifndef FRAM_H
#define FRAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define FRAM_OK          0
#define FRAM_EINVAL     (-1)   /* bad argument or scene description                       */
#define FRAM_EWORKSPACE (-2)   /* workspace pointer null, misaligned or too small          */
#define FRAM_ECUDA      (-3)   /* a CUDA runtime call failed; fram_last_error has the text */
#define FRAM_EDEVICE    (-4)   /* the device status word reports an error (fram_status)    */

/* Device status word bits (fram_status). */
#define FRAM_DEV_BAD_GEOMETRY   0x1  /* c0*T60 <= D0, D0 == 0, T60 <= 0 or dims <= 0        */
#define FRAM_DEV_CAPACITY       0x2  /* a synthesis tile held more images than it can stage */
#define FRAM_DEV_NONFINITE      0x4  /* a non-finite position, g or r was read              */
#define FRAM_DEV_BOUNDS         0x8  /* debug builds only (FRAM_DEBUG_BOUNDS): an index fell  */
                                     /* outside its buffer; the access was skipped           */

/*
 * Method constants.  The paper fixes only their ranges: 0 <= alpha < beta <= 1 (Eq. 3),
 * tau > 0 (Eq. 6), and the [-6, 50] ms early window (Eq. 9).  fram_default_params fills
 * this project's defaults: alpha 0.25, beta 1, a -2, b 2, tau 0.25, c0 343 m/s, fs 16 kHz,
 * K 40, early window 6 / 50 ms, tile 0 (library default), delay_mode 0.
 */
typedef struct fram_params {
    double alpha;          /* Eq. 3: distance ratios are drawn on (alpha, beta]; alpha > 0 */
    double beta;           /*        (Eq. 4 divides by alpha)                              */
    double a;              /* Eq. 6: perturbation p_i ~ U(a, b)                            */
    double b;
    double tau;            /* Eq. 6: distance shrinkage factor, > 0                        */
    double c0;             /* speed of sound, m/s                                          */
    double fs;             /* output sample rate, Hz                                       */
    double early_pre_ms;   /* Eq. 9: early RIR keeps n - n0 in [-ceil(pre*fs/1000),        */
    double early_post_ms;  /*        +ceil(post*fs/1000)], n0 = ceil(D_{0,m} fs / c0)       */
    int32_t half_len;      /* K: taps at |n - t| < K, 2K+1 taps per arrival; 1..128        */
    int32_t tile;          /* synthesis tile length in samples (multiple of 256, 256..4096); */
                           /* 0 = the tile fram_autotune chose for this kind of workload,  */
                           /* else 1024; size workspaces with 0 to allow any tile          */
    int32_t delay_mode;    /* 0: continuous delay t = D fs/c0, windowed sinc at fs (default; */
                           /*    differentiable).                                            */
                           /* 1: the paper's multi-rate path (Sec. II-B, Eq. 7-9 as printed): */
                           /*    impulses at q = min(ceil(D r_h fs/c0), L_h - 1) on the r_h fs */
                           /*    grid (r_h = floor(1e6/fs), L_h = ceil(T60 r_h fs)), resampled */
                           /*    to r_l fs (r_l = floor(sqrt(r_h)), must be 2..11), 80 Hz      */
                           /*    high-pass, resampled to fs; the same output layout.  Filters */
                           /*    (not given in the paper): Kaiser (beta 5) windowed-sinc       */
                           /*    polyphase resamplers of half length 10 max(up, down), DC gain */
                           /*    up; 2nd-order Butterworth high-pass (bilinear, pre-warped).   */
                           /*    Forward only: fram_synthesize_backward returns FRAM_EINVAL.  */
                           /*    Needs r_l * max_len < 2^30 (FRAM_EINVAL otherwise).           */
    int32_t reserved;      /* must be 0                                                     */
} fram_params;

/*
 * Scene: B rooms, S sources and M microphones per room.  The host-side sizes must match
 * the device arrays (fram_layout produces them).
 */
typedef struct fram_scene {
    int32_t B, S, M;
    int32_t max_len;           /* max_b L_b                                        (host) */
    int64_t n_vs_total;        /* vs_off[B]: total image rows                      (host) */
    int64_t rir_total;         /* rir_off[B]: total RIR samples                    (host) */
    double array_radius;       /* max over rooms and mics of |mic_m - centre_b|, m (host); */
                               /* sizes the adjoint's halo; an arrival beyond it sets     */
                               /* FRAM_DEV_CAPACITY                                        */
    const float* dims;         /* [B,3]  room size Lx, Ly, Lz (Sec. III-A)                */
    const float* rt60;         /* [B]    T60 in seconds (Eq. 2, 4, 5, Sec. III-D)          */
    const float* src;          /* [B,S,3] source positions                                 */
    const float* mic;          /* [B,M,3] microphone positions                             */
    const int32_t* n_vs;       /* [B]    images per (room, source), I in Eq. 1             */
    const int64_t* vs_off;     /* [B+1]  image row offset of each room                     */
    const int32_t* rir_len;    /* [B]    L_b                                               */
    const int64_t* rir_off;    /* [B+1]  sample offset of each room                        */
    int64_t room_base;         /* index of room 0 in a larger batch (host; 0 for a whole    */
                               /* batch): room b draws its images with the Philox counter  */
                               /* room word room_base + b, so a shard of a batch drawn with */
                               /* the same seed gets exactly the images the whole batch     */
                               /* gives those rooms.  0 <= room_base, room_base + B <= 2^32 */
} fram_scene;

/* Library version (major*10000 + minor*100 + patch). */
int fram_version(void);

/* Thread-local text of the last host-side error ("" if none). */
const char* fram_last_error(void);

/* Fill *p with the defaults listed above. */
void fram_default_params(fram_params* p);

/*
 * Host only.  L_b = ceil(T60_b * fs) (Sec. III-D at the output rate) and the ragged offsets.
 * rt60 [B], n_vs [B] are host arrays; outputs rir_len [B], rir_off [B+1], vs_off [B+1] are
 * host arrays written by the call.  Returns FRAM_EINVAL for B < 0, S < 1, M < 1, fs <= 0,
 * T60 <= 0, n_vs < 0 or a length above 2^31 - 1.
 */
int fram_layout(int32_t B, int32_t S, int32_t M, double fs, const float* rt60, const int32_t* n_vs,
                int32_t* rir_len, int64_t* rir_off, int64_t* vs_off);

/*
 * Host only.  Bytes of device workspace that fram_sample, fram_synthesize and
 * fram_synthesize_backward need for this scene and these parameters (one buffer serves all
 * three).  The workspace must be 256-byte aligned.
 */
int fram_workspace_size(const fram_scene* scene, const fram_params* p, size_t* bytes);

/*
 * Virtual-image sampler (Sec. III-A to III-C).  For room b, source s and image i one
 * Philox4x32-10 call (Salmon et al., SC'11) with counter (i, s, room_base + b, 0) and key
 * (seed mod 2^32, seed div 2^32) gives four words w_k, mapped to u_k = ((w_k >> 9) + 0.5) 2^-23:
 *   x    = (alpha^3 + u0 (beta^3 - alpha^3))^(1/3)              inverse CDF of Eq. 3
 *   DR_i = 1 + alpha/(beta-alpha) (x/alpha - 1)(c0 T60/D0 - 1)  Eq. 4,  D_i = D0 DR_i
 *   theta = 2 pi u1, phi = pi (u2 - 1/2)                         Sec. III-B
 *   p_i  = c + D_i (cos phi cos theta, cos phi sin theta, sin phi), c = mean of the mics
 *   g_i  = clamp(1 + (D_i/(c0 T60))^2 (RR_max - 1) + (a + (b-a) u3) DR_i^tau, 1, RR_max)
 *                                                                Eq. 5, 6
 * with D0 = |src - c| and r from Eq. 2.
 * Outputs (device, caller-owned): vs_pos_hi, vs_pos_lo [N,3]: each coordinate as an
 * unevaluated float pair hi + lo (about 44 significant bits, so delays stay exact to well
 * below a microsample); vs_g [N]; r [B] (Eq. 2); words [N,4] (nullable: the raw Philox
 * words, for verification).
 * d_seed (nullable) is a device pointer to a uint64 seed read by the kernel instead of
 * `seed`, so a captured graph can be replayed with new draws.
 * Device status: FRAM_DEV_BAD_GEOMETRY if c0 T60 <= D0 or D0 == 0 (outputs for that room
 * are NaN).
 */
int fram_sample(const fram_scene* scene, const fram_params* p, uint64_t seed, const uint64_t* d_seed,
                float* vs_pos_hi, float* vs_pos_lo, float* vs_g, float* r, uint32_t* words,
                void* workspace, size_t workspace_bytes, void* stream);

/*
 * Synthesis (Eq. 1 with windowed-sinc arrivals, Sec. III-D; Eq. 9).  For every room b,
 * source s, mic m and n in [0, L_b):
 *   h[n] = sum over arrivals j with |n - t_j| < K of  A_j sinc(n - t_j) (1 + cos(pi (n - t_j)/K))/2
 * where the arrivals are the direct path (A = 1/D_{0,m}, t = D_{0,m} fs/c0) and every image
 * (A = r_b^{g_i} / D_{i,m}, t = D_{i,m} fs/c0, D_{i,m} = |p_i - mic_m|), sinc(x) = sin(pi x)/(pi x).
 * Taps outside [0, L_b) are dropped.  Sums are accumulated in float32 in an order fixed by the
 * inputs and the tile length (direct path first, then the images by delay to the array centre,
 * ties by image index), so results are bit-reproducible run to run; two tile lengths agree to
 * float32 rounding.
 * Inputs: image positions vs_pos_hi [N,3] and vs_pos_lo [N,3] (nullable = zero low parts,
 * i.e. plain float32 positions), reflection counts vs_g [N], coefficients r [B].
 * Outputs: rir [rir_total]; early [rir_total] (nullable) receives h_e of Eq. 9.  Both must be
 * 4-byte aligned (FRAM_EINVAL otherwise).
 */
int fram_synthesize(const fram_scene* scene, const fram_params* p,
                    const float* vs_pos_hi, const float* vs_pos_lo, const float* vs_g, const float* r,
                    float* rir, float* early, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Adjoint of fram_synthesize.  Given dL/dh (grad_rir, same layout as rir; nullable = 0) and
 * dL/dh_e (grad_early; nullable), computes by recomputing each arrival's taps:
 *   dL/dt_j = -A_j sum_n G[n] tap'(n - t_j),  dL/dA_j = sum_n G[n] tap(n - t_j),
 *   G = grad_rir + (Eq. 9 mask) * grad_early,
 * and chains them to positions and r:  dL/dD = dL/dt fs/c0 - dL/dA A/D,
 * dD_{i,m}/dp_i = (p_i - mic_m)/D_{i,m} = -dD_{i,m}/dmic_m, dA/dr = g A / r, dA/dg = A ln r.
 * Images are leaves here: the source gradient comes from the direct path only (see
 * fram_sample_backward for the path through the sampler).
 * Outputs (each nullable, overwritten): grad_vs [N,3], grad_mic [B,M,3], grad_src [B,S,3],
 * grad_r [B], grad_g [N] (dL/dg_i summed over mics).  Reductions run in a fixed order
 * (bit-reproducible).  Requires p->delay_mode == 0 (FRAM_EINVAL otherwise).
 */
int fram_synthesize_backward(const fram_scene* scene, const fram_params* p,
                             const float* vs_pos_hi, const float* vs_pos_lo, const float* vs_g,
                             const float* r, const float* grad_rir, const float* grad_early,
                             float* grad_vs, float* grad_mic, float* grad_src, float* grad_r,
                             float* grad_g, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Gradient through the sampler (reparameterised: with seed fixed, every image's Philox draws
 * u0..u3 are constants, so p_i, g_i and r are differentiable functions of the source, the mics,
 * T60 and the room size; Sec. III-A to III-C, Eq. 2-6 as fram_sample evaluates them).
 * With k_i = (x_i - alpha)/(beta - alpha), Eq. 4 reads D_i = D0 (1 - k_i) + k_i c0 T60, and
 *   p_i = c + D_i nu_i,      D0 = |src - c|,      c = mean of the mics,
 *   g_i: Eq. 6 (derivative 0 where the clamp holds g_i at 1; dg_i/dRR_max = 1 where it holds
 *   g_i at RR_max),  RR_max: Eq. 5,  r: Eq. 2 with R = V/S of the room.
 * Inputs (device): grad_vs [N,3] = dL/dp_i (required), grad_g [N] = dL/dg_i (nullable = 0),
 * grad_r [B] = dL/dr from the synthesis (nullable = 0), grad_src_in [B,S,3] and grad_mic_in
 * [B,M,3] = the direct gradients (nullable = 0), typically fram_synthesize_backward's grad_src
 * and grad_mic; they may alias grad_src / grad_mic (each element is read before it is written).
 * seed / d_seed must be those of the fram_sample call that drew the images.
 * Outputs (device, nullable, overwritten): grad_src [B,S,3], grad_mic [B,M,3] (totals: direct
 * plus sampler paths), grad_t60 [B], grad_dims [B,3].  Per (room, source) sums over images run
 * in FP32 per thread (strided images), then in FP64 across threads, in a fixed order
 * (bit-reproducible).  Device status FRAM_DEV_BAD_GEOMETRY as for fram_sample (that
 * (room, source) contributes no sampler path).  Uses the workspace (sized by
 * fram_workspace_size for this scene).
 */
int fram_sample_backward(const fram_scene* scene, const fram_params* p, uint64_t seed, const uint64_t* d_seed,
                         const float* grad_vs, const float* grad_g, const float* grad_r,
                         const float* grad_src_in, const float* grad_mic_in,
                         float* grad_src, float* grad_mic, float* grad_t60, float* grad_dims,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * The two stages of fram_synthesize / fram_synthesize_backward, for callers that reuse one
 * preparation (for instance a forward and a backward pass over the same images, or timing the
 * main kernel alone).  fram_prepare clears the status word and builds, in the workspace, the
 * per-room tables (RIR length, array centre, direct paths of Eq. 1 and the Eq. 9 windows),
 * the work-item list and each image's delay bin; it reads vs_pos_hi/lo and r only.
 * fram_synthesize_prepared and fram_synthesize_backward_prepared then run the main kernel;
 * they require the most recent fram_prepare on this workspace to have seen the same scene,
 * parameters, image positions and r (otherwise results are undefined, but every index stays
 * bounded by the host sizes).  Arguments mean what they mean for the one-shot calls.
 */
int fram_prepare(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_pos_lo,
                 const float* r, void* workspace, size_t workspace_bytes, void* stream);
int fram_synthesize_prepared(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                             const float* vs_pos_lo, const float* vs_g, const float* r, float* rir, float* early,
                             void* workspace, size_t workspace_bytes, void* stream);
int fram_synthesize_backward_prepared(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                                      const float* vs_pos_lo, const float* vs_g, const float* r,
                                      const float* grad_rir, const float* grad_early, float* grad_vs,
                                      float* grad_mic, float* grad_src, float* grad_r, float* grad_g,
                                      void* workspace, size_t workspace_bytes, void* stream);

/*
 * Tile-length autotuner for the synthesis kernel.  Runs fram_synthesize on the caller's own
 * inputs with each candidate tile length (256, 512, 1024, 2048 samples; those whose workspace
 * or shared memory does not fit are skipped), times them with CUDA events on `stream`, and
 * records the fastest for this kind of workload (device, K, fs, S, M, RIR-length octave, image
 * density).  Later calls with p->tile == 0 on a matching workload use it.  The tile length
 * sets how many images and arrivals each CTA stages and sorts, so it also picks the number of
 * impulses per CTA.  Writes the choice to *tile_out (nullable).  Overwrites `rir`.
 * Synchronises the stream: call it before capturing a CUDA graph.  The workspace must be sized
 * with p->tile == 0 (fram_workspace_size then covers every candidate).
 * Persistence (opt-in): if the environment variable FRAM_AUTOTUNE_CACHE names a file, each
 * choice is also written there (one JSON object per line, keyed by the GPU's name and SM count
 * and the workload group above; rewritten through a temporary file and a rename), and a later
 * process's first tile = 0 launch on that GPU model reads it, so it need not re-tune.  Errors
 * reading or writing the file are ignored (the in-memory choice still applies).
 */
int fram_autotune(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_pos_lo,
                  const float* vs_g, const float* r, float* rir, void* workspace, size_t workspace_bytes,
                  void* stream, int32_t* tile_out);

/*
 * Host only (but queries the current device).  The tile length a call with these parameters
 * launches with: p->tile if nonzero, else the tile fram_autotune chose for this kind of workload
 * (in this process, or from the FRAM_AUTOTUNE_CACHE file), else the library default 1024.
 */
int fram_tuned_tile(const fram_scene* scene, const fram_params* p, int32_t* tile);

/*
 * Synchronises `stream` and reads the device status word that the last call which used
 * this workspace wrote (FRAM_DEV_* bits) into *flags.  Returns FRAM_EDEVICE if any bit is
 * set, FRAM_ECUDA on a CUDA error, FRAM_OK otherwise.
 */
int fram_status(void* workspace, void* stream, int32_t* flags);

/*
 * fram_synthesize without a workspace argument, for callers that cannot allocate device
 * memory (a plugin whose host application owns all device memory, a real-time thread that
 * must not block on cudaMalloc/cudaFree, a fixed device-memory budget).  The paper has no
 * counterpart: this is a deployment convenience around the same synthesis.
 * Inputs, outputs and results are those of fram_synthesize.  The scratch is a static 16 MiB
 * device array that every GPU loading libfram reserves until the process exits; a scene whose
 * workspace at the tile length the call launches with (p->tile, or the tuned or default tile
 * when p->tile is 0) exceeds 16 MiB is rejected with FRAM_EWORKSPACE before any GPU work.
 * Contexts: each CUDA context (a device's primary context, a context created through the driver
 * API, a primary context re-created after cudaDeviceReset) has its own copy of the array.  A call
 * made while `stream` is not being captured looks up the copy of the current context with
 * cudaGetSymbolAddress; a call made during stream capture reuses the address an earlier
 * non-capturing call found in the same context, so the first call in a context must come before
 * any capture (FRAM_ECUDA otherwise).
 * All calls in a context share the one array: calls that overlap on the GPU (different streams
 * or threads without ordering) race and corrupt each other's results.  Device status bits of
 * these calls are not reported (fram_status needs the caller's workspace).  Allocates nothing.
 */
int fram_synthesize_noalloc(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                            const float* vs_pos_lo, const float* vs_g, const float* r, float* rir,
                            float* early, void* stream);

/*
 * Throughput probe for the roofline denominators of the synthesis and the adjoint (the paper has
 * no counterpart: it measures this GPU).  kind 0: scalar FP32 fused multiply-add; 1: packed FP32
 * fma.rn.f32x2 (two lane operations per instruction); 2: MUFU reciprocal rcp.approx.ftz.f32
 * (chained as x -> 1/x + b, the add on the FP32 pipe).
 * Launches 8 CTAs of 256 threads per SM, each thread running 8 independent chains of
 * iters x 64 operations, and synchronises the stream.  result (host, 4 doubles): kernel time in
 * ms (CUDA events on `stream`), SM clock cycles of the longest CTA (clock64), total lane
 * operations, SM count.  Lane operations per SM per clock = result[2] / (result[1] result[3]).
 * Uses a static device buffer of one cycle count per CTA; allocates nothing.  Returns
 * FRAM_EINVAL for a bad kind, iters < 1 or a null result.
 */
int fram_measure_alu(int32_t kind, int64_t iters, double* result, void* stream);

/*
 * Spatialisation: the paper's use of the RIRs for training data (Sec. IV-A).  For every room
 * b, source s < S, mic m and sample n < N:
 *   y_{s,m}[n] = sum_{k=0}^{min(L_b-1, n)} h_{s,m}[k] x_s[n-k]          (image of source s)
 *   E_s = sum_n y_{s,0}[n]^2                                              (energy at mic 0)
 *   g_0 = 1;  speakers 1 <= s < n_speech: g_s = sqrt(E_0/E_s 10^(-level_s/10))   (level = SIR, dB)
 *   speech at mic 0 v = sum_{s<n_speech} g_s y_{s,0}, E_v = sum_n v[n]^2;
 *   noise s >= n_speech: g_s = sqrt(E_v/E_s 10^(-level_s/10))                   (level = SNR, dB)
 *   (g_s = 0 for a silent image, E_s = 0)
 *   mixture_m[n] = sum_s g_s y_{s,m}[n];  targets_{s,m}[n] = g_s (h'_{s,m} * x_s)[n], s < n_speech,
 * with h' = target_rir (the early RIR of Eq. 9 for dereverberation targets, or rir itself).
 * The paper mixes two speakers (SIR in [-6, 6] dB, overlap >= 0.5) and one point-source noise
 * (SNR in [10, 20] dB); signals are given already placed on the mixture's timeline.
 * Computed by FFT overlap-save convolution in FP32 (error ~1e-6 of each channel's peak) with
 * FP64 energies; results are bit-reproducible run to run.
 * Inputs (device): rir / target_rir in fram_synthesize's ragged layout (scene->rir_len,
 * rir_off, max_len; dims, src and the image fields of the scene are not read); signals
 * [B,S,N]; level_db [B,S] (entry 0 of each room unused).  Outputs (device, caller-owned,
 * overwritten): mixture [B,M,N]; targets [B,n_speech,M,N] (nullable; needs target_rir);
 * gains [B,S] (nullable).  Host errors: FRAM_EINVAL (S > 8, n_speech outside [1, S], N < 1,
 * bad block), FRAM_EWORKSPACE.  Device status: FRAM_DEV_BAD_GEOMETRY if a room's rir_len /
 * rir_off disagree with max_len / rir_total (that RIR is read as zeros).
 * The workspace (256-byte aligned, fram_spatialize_workspace_size with separate_targets = 1
 * when targets come from a different RIR buffer) holds the spectra of one chunk of rooms.
 */
typedef struct {
    int64_t n_samples;         /* N: samples of every source signal and output channel       */
    int32_t n_speech;          /* sources [0, n_speech) are speakers, the rest noise           */
    int32_t block;             /* overlap-save block (= FFT length / 2): 0 = auto (4096, or   */
                               /* the least of 8192, 16384 with S x ceil(max_len / block) <=  */
                               /* 128), or one of 4096, 8192, 16384 meeting that limit         */
    int32_t chunk_rooms;       /* rooms per pipeline chunk: 0 = auto (spectra ~4 GiB)          */
    int32_t reserved;
} fram_spatial;

int fram_spatialize_workspace_size(const fram_scene* scene, const fram_spatial* sp, int32_t separate_targets,
                                   size_t* bytes);
int fram_spatialize(const fram_scene* scene, const fram_spatial* sp, const float* rir, const float* target_rir,
                    const float* signals, const float* level_db, float* mixture, float* targets, float* gains,
                    void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FRAM_H */
