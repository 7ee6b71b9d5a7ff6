// fram_api.cu -- host side of the C ABI declared in include/fram.h: argument checks, the
// ragged layout, workspace sizing and the launch sequence of each entry point.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fram_internal.cuh"

namespace fram {

// A named NVTX range around an entry point's host work and launches, so a timeline tool shows
// the sampler, the preparation, the synthesis and the adjoint as separate ranges (the NVTX
// calls do nothing unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

static int cuda_fail(cudaError_t e, const char* what)
{
    return fail(FRAM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

cudaError_t kernel_residency(const void* func, int threads, int smem, int* per_sm)
{
    struct Entry {
        const void* func;
        int dev, threads, smem, per_sm;
    };
    struct Limit {           // largest dynamic shared memory already allowed per kernel and device
        const void* func;
        int dev, smem;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    static std::vector<Limit> limits;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& c : cache)
        if (c.func == func && c.dev == dev && c.threads == threads && c.smem == smem) {
            *per_sm = c.per_sm;
            return cudaSuccess;
        }
    // The limit only ever grows, so an earlier, larger configuration stays launchable.
    Limit* lim = nullptr;
    for (Limit& l : limits)
        if (l.func == func && l.dev == dev) lim = &l;
    if (!lim || lim->smem < smem) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (lim) lim->smem = smem;
        else limits.push_back({func, dev, smem});
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem);
    if (e != cudaSuccess) return e;
    if (n < 1) n = 1;
    cache.push_back({func, dev, threads, smem, n});
    *per_sm = n;
    return cudaSuccess;
}

static int check_params(const fram_params* p)
{
    if (!p) return fail(FRAM_EINVAL, "params is null");
    if (!(p->alpha > 0.0) || !(p->beta > p->alpha) || !(p->beta <= 1.0))
        return fail(FRAM_EINVAL, "need 0 < alpha < beta <= 1 (Eq. 3, 4), got alpha=%g beta=%g", p->alpha, p->beta);
    if (!(p->tau > 0.0)) return fail(FRAM_EINVAL, "need tau > 0 (Eq. 6)");
    if (!(p->b >= p->a)) return fail(FRAM_EINVAL, "need a <= b (Eq. 6)");
    if (!(p->c0 > 0.0) || !(p->fs > 0.0)) return fail(FRAM_EINVAL, "need c0 > 0 and fs > 0");
    if (p->half_len < 1 || p->half_len > kMaxHalfLen) return fail(FRAM_EINVAL, "half_len must be in [1, %d]", kMaxHalfLen);
    if (!(p->early_pre_ms >= 0.0) || !(p->early_post_ms >= 0.0)) return fail(FRAM_EINVAL, "early window must be >= 0");
    if (p->tile != 0 && (p->tile < 256 || p->tile > 4096 || p->tile % 256 != 0))
        return fail(FRAM_EINVAL, "tile must be 0 or a multiple of 256 in [256, 4096]");
    if (p->delay_mode != 0 && p->delay_mode != 1) return fail(FRAM_EINVAL, "delay_mode must be 0 or 1");
    if (p->delay_mode == 1) {
        const int rh = (int)std::floor(1.0e6 / p->fs), rl = (int)std::floor(std::sqrt((double)rh));
        if (rl < 2 || rl > 11)
            return fail(FRAM_EINVAL, "delay_mode 1 needs r_l = floor(sqrt(floor(1e6/fs))) in [2, 11] (fs = %g)", p->fs);
    }
    return FRAM_OK;
}

// ---- tile length: explicit, or chosen by fram_autotune for this kind of workload ----------
// Workloads are grouped by device, K, fs, sources, mics, the RIR-length octave and the image
// density (images per output sample, half-octave bins); fram_autotune records the fastest tile
// per group and launches with tile = 0 use it (the library default until a group is tuned).
static const int kTileCandidates[] = {256, 512, 1024, 2048};

struct TuneKey {
    int dev, K, S, M, len_oct, dens_bin;
    double fs;
    bool operator==(const TuneKey& o) const
    {
        return dev == o.dev && K == o.K && S == o.S && M == o.M && len_oct == o.len_oct && dens_bin == o.dens_bin &&
               fs == o.fs;
    }
};

static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, int>> g_tune;

// ---- persistent tile cache (opt-in: the file named by FRAM_AUTOTUNE_CACHE) ------------------
// One line per tuned workload group, keyed by the GPU's name and SM count (so a cache copied to
// a different GPU model is not used) and the group of TuneKey:
//   {"gpu": "<name>", "sms": N, "K": K, "fs": fs, "S": S, "M": M, "len_oct": o, "dens_bin": d, "tile": T}
// Read once per device the first time a tile = 0 launch finds no in-memory choice; rewritten
// whole (to a temporary file, then renamed) by fram_autotune.
struct DevId {
    char name[256];
    int sms;
};

static bool dev_id(int dev, DevId* id)
{
    cudaDeviceProp prop;
    if (dev < 0 || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
    snprintf(id->name, sizeof id->name, "%s", prop.name);
    for (char* c = id->name; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    id->sms = prop.multiProcessorCount;
    return true;
}

struct CacheLine {
    DevId id;
    TuneKey k;
    int tile;
};

static std::vector<CacheLine> read_cache_file(const char* path)
{
    std::vector<CacheLine> out;
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        CacheLine c{};
        if (sscanf(line,
                   " {\"gpu\": \"%255[^\"]\", \"sms\": %d, \"K\": %d, \"fs\": %lf, \"S\": %d, \"M\": %d, "
                   "\"len_oct\": %d, \"dens_bin\": %d, \"tile\": %d}",
                   c.id.name, &c.id.sms, &c.k.K, &c.k.fs, &c.k.S, &c.k.M, &c.k.len_oct, &c.k.dens_bin, &c.tile) == 9 &&
            (c.tile == 256 || c.tile == 512 || c.tile == 1024 || c.tile == 2048))
            out.push_back(c);
    }
    fclose(f);
    return out;
}

static void write_cache_file(const char* path, const std::vector<CacheLine>& lines)
{
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;                       // the cache is an optimisation: failures are silent
    bool ok = true;
    for (const CacheLine& c : lines)
        ok = ok && fprintf(f,
                           "{\"gpu\": \"%s\", \"sms\": %d, \"K\": %d, \"fs\": %.17g, \"S\": %d, \"M\": %d, "
                           "\"len_oct\": %d, \"dens_bin\": %d, \"tile\": %d}\n",
                           c.id.name, c.id.sms, c.k.K, c.k.fs, c.k.S, c.k.M, c.k.len_oct, c.k.dens_bin, c.tile) > 0;
    ok = (fclose(f) == 0) && ok;
    if (ok) rename(tmp.c_str(), path);
    else remove(tmp.c_str());
}

static bool same_group(const CacheLine& c, const DevId& id, const TuneKey& k)
{
    return strcmp(c.id.name, id.name) == 0 && c.id.sms == id.sms && c.k.K == k.K && c.k.fs == k.fs &&
           c.k.S == k.S && c.k.M == k.M && c.k.len_oct == k.len_oct && c.k.dens_bin == k.dens_bin;
}

static std::vector<int> g_cache_loaded;   // devices whose cache lines are in g_tune (under g_tune_mu)

// Under g_tune_mu: merge the cache file's lines for device k.dev into g_tune, once per device.
static void load_cache_locked(int dev)
{
    const char* path = getenv("FRAM_AUTOTUNE_CACHE");
    if (!path || !*path || dev < 0) return;
    for (int d : g_cache_loaded)
        if (d == dev) return;
    g_cache_loaded.push_back(dev);
    DevId id;
    if (!dev_id(dev, &id)) return;
    for (const CacheLine& c : read_cache_file(path)) {
        if (strcmp(c.id.name, id.name) != 0 || c.id.sms != id.sms) continue;
        TuneKey k = c.k;
        k.dev = dev;
        bool found = false;
        for (const auto& e : g_tune) found = found || e.first == k;
        if (!found) g_tune.push_back({k, c.tile});
    }
}

static void store_cache(const TuneKey& k, int tile)
{
    const char* path = getenv("FRAM_AUTOTUNE_CACHE");
    DevId id;
    if (!path || !*path || !dev_id(k.dev, &id)) return;
    std::vector<CacheLine> lines = read_cache_file(path);
    bool found = false;
    for (CacheLine& c : lines)
        if (same_group(c, id, k)) { c.tile = tile; found = true; }
    if (!found) lines.push_back(CacheLine{id, k, tile});
    write_cache_file(path, lines);
}

static TuneKey tune_key(const fram_scene* sc, const fram_params* p)
{
    TuneKey k{};
    if (cudaGetDevice(&k.dev) != cudaSuccess) k.dev = -1;
    k.K = p->half_len;
    k.S = sc->S;
    k.M = sc->M;
    k.fs = p->fs;
    k.len_oct = sc->max_len > 0 ? (int)std::ceil(std::log2((double)sc->max_len)) : 0;
    const double samples = sc->M > 0 ? (double)sc->rir_total / sc->M : 0.0;
    const double dens = samples > 0 ? (double)sc->n_vs_total / samples : 0.0;
    k.dens_bin = dens > 0 ? (int)std::floor(2.0 * std::log2(dens)) : -1000;
    return k;
}

static int tile_for(const fram_scene* sc, const fram_params* p)
{
    if (p->tile) return p->tile;
    const TuneKey k = tune_key(sc, p);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune)
        if (e.first == k) return e.second;
    load_cache_locked(k.dev);
    for (const auto& e : g_tune)
        if (e.first == k) return e.second;
    return kDefaultTile;
}

static int tile_of(const fram_params* p) { return p->tile ? p->tile : kTileCandidates[0]; }

static int check_scene(const fram_scene* sc, bool need_arrays)
{
    if (!sc) return fail(FRAM_EINVAL, "scene is null");
    if (sc->B < 0 || sc->S < 1 || sc->M < 1) return fail(FRAM_EINVAL, "need B >= 0, S >= 1, M >= 1");
    if (sc->S >= 32768) return fail(FRAM_EINVAL, "S must be below 32768");
    if (sc->M > 64) return fail(FRAM_EINVAL, "M must be at most 64");
    if (sc->n_vs_total < 0 || sc->rir_total < 0 || sc->max_len < 0) return fail(FRAM_EINVAL, "negative totals");
    if (sc->B > 0 && sc->max_len < 1) return fail(FRAM_EINVAL, "max_len must be >= 1");
    if (!(sc->array_radius >= 0.0) || !std::isfinite(sc->array_radius)) return fail(FRAM_EINVAL, "array_radius must be finite and >= 0");
    if (sc->room_base < 0 || sc->room_base + (int64_t)sc->B > (int64_t(1) << 32))
        return fail(FRAM_EINVAL, "need 0 <= room_base and room_base + B <= 2^32 (the Philox room word)");
    if (need_arrays && sc->B > 0) {
        if (!sc->dims || !sc->rt60 || !sc->src || !sc->mic || !sc->n_vs || !sc->vs_off || !sc->rir_len || !sc->rir_off)
            return fail(FRAM_EINVAL, "scene device arrays must not be null");
    }
    return FRAM_OK;
}

// Multi-rate mode: the kernels index a channel's intermediate samples (r_l per output sample) in
// 32-bit integers, so r_l max_len must stay below 2^30 (an RIR of ~97 million samples at r_l = 11).
static int check_mr_len(const fram_scene* sc, const fram_params* p)
{
    if (p->delay_mode == 1 && (int64_t)mr_rates(p->fs).rl * sc->max_len >= ((int64_t)1 << 30))
        return fail(FRAM_EINVAL, "delay_mode 1 needs r_l * max_len < 2^30 (r_l = %d, max_len = %d)",
                    mr_rates(p->fs).rl, sc->max_len);
    return FRAM_OK;
}

static int check_ws(const fram_scene* sc, const fram_params* p, void* ws, size_t bytes, WsLayout* out)
{
    if (check_mr_len(sc, p) != FRAM_OK) return FRAM_EINVAL;
    const WsLayout w = ws_layout(*sc, tile_for(sc, p), p->delay_mode, p->fs);
    if (w.max_tiles > 0xffff) return fail(FRAM_EINVAL, "too many tiles per RIR (raise the tile length)");
    if (!ws) return fail(FRAM_EWORKSPACE, "workspace is null");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FRAM_EWORKSPACE, "workspace must be 256-byte aligned");
    if (bytes < w.total) return fail(FRAM_EWORKSPACE, "workspace too small: %zu < %zu bytes", bytes, w.total);
    *out = w;
    return FRAM_OK;
}

int workspace_bytes_at_launch_tile(const fram_scene* sc, const fram_params* p, size_t* bytes)
{
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(sc, false)) != FRAM_OK) return rc;
    if (!bytes) return fail(FRAM_EINVAL, "bytes is null");
    if ((rc = check_mr_len(sc, p)) != FRAM_OK) return rc;
    const WsLayout w = ws_layout(*sc, tile_for(sc, p), p->delay_mode, p->fs);
    if (w.max_tiles > 0xffff) return fail(FRAM_EINVAL, "too many tiles per RIR (raise the tile length)");
    *bytes = w.total;
    return FRAM_OK;
}

static LaunchArgs make_args(const fram_scene* sc, const fram_params* p, const WsLayout& w, void* ws)
{
    LaunchArgs a{};
    a.fs = p->fs;
    a.c0 = p->c0;
    a.B = sc->B; a.S = sc->S; a.M = sc->M;
    a.K = p->half_len;
    a.tile = w.tile;
    a.max_tiles = w.max_tiles;
    a.nb32 = w.nb32;
    const double q = p->fs / p->c0;
    a.q = (float)q;
    a.q2 = f2_from_double(q);
    a.early_pre = (int32_t)std::ceil(p->early_pre_ms * p->fs / 1000.0);
    a.early_post = (int32_t)std::ceil(p->early_post_ms * p->fs / 1000.0);
    a.margin_i = (int32_t)std::ceil(sc->array_radius * q) + 3;
    a.n_vs_total = sc->n_vs_total;
    a.rir_total = sc->rir_total;
    a.room_base = (uint32_t)sc->room_base;
    a.dims = sc->dims; a.rt60 = sc->rt60; a.src = sc->src; a.mic = sc->mic;
    a.n_vs = sc->n_vs; a.vs_off = sc->vs_off; a.rir_len = sc->rir_len; a.rir_off = sc->rir_off;
    unsigned char* base = static_cast<unsigned char*>(ws);
    a.hdr = reinterpret_cast<Header*>(base + w.header);
    a.room = reinterpret_cast<RoomConst*>(base + w.room);
    a.direct = reinterpret_cast<DirectConst*>(base + w.direct);
    a.src_tile = reinterpret_cast<int32_t*>(base + w.src_tile);
    a.item_off = reinterpret_cast<int32_t*>(base + w.item_off);
    a.items = reinterpret_cast<int2*>(base + w.items);
    a.order = reinterpret_cast<int32_t*>(base + w.order);
    a.bin_off = reinterpret_cast<int32_t*>(base + w.bin_off);
    a.perm = reinterpret_cast<int32_t*>(base + w.perm);
    a.key = reinterpret_cast<float*>(base + w.key);
    a.skey = reinterpret_cast<int32_t*>(base + w.skey);
    a.spa = reinterpret_cast<float4*>(base + w.spa);
    a.spb = reinterpret_cast<float2*>(base + w.spb);
    a.pos32 = reinterpret_cast<int32_t*>(base + w.pos32);
    a.samp = reinterpret_cast<float*>(base + w.samp);
    a.irec = reinterpret_cast<ItemRec*>(base + w.irec);
    a.part_mic = reinterpret_cast<float*>(base + w.part_mic);
    a.part_src = reinterpret_cast<float*>(base + w.part_src);
    a.part_r = reinterpret_cast<float*>(base + w.part_r);
    a.sb_part = reinterpret_cast<double*>(base + w.sb_part);
    a.sconst = reinterpret_cast<char*>(base + w.sconst);
    a.max_len = sc->max_len;
    a.mode = p->delay_mode;
    a.early_pre_ms = p->early_pre_ms;
    a.early_post_ms = p->early_post_ms;
    if (p->delay_mode == 1) {
        const MrRates mr = mr_rates(p->fs);
        a.rh = mr.rh; a.rl = mr.rl; a.up = mr.up; a.down = mr.down;
        a.HLA = 10 * (mr.up > mr.down ? mr.up : mr.down);
        a.fh = (double)mr.rh * p->fs;
        a.mr_y = reinterpret_cast<float*>(base + w.mr_y);
        a.mr_ye = reinterpret_cast<float*>(base + w.mr_ye);
        a.mr_tab = reinterpret_cast<float*>(base + w.mr_tab);
        a.mr_order = reinterpret_cast<int32_t*>(base + w.mr_order);
        a.mr_counts = reinterpret_cast<int32_t*>(base + w.mr_counts);
        a.mr_pstate = base + w.mr_pstate;
    }
    return a;
}

}  // namespace fram

using namespace fram;

extern "C" {

int fram_version(void) { return 10200; }

const char* fram_last_error(void) { return g_last_error.c_str(); }

void fram_default_params(fram_params* p)
{
    if (!p) return;
    p->alpha = 0.25;
    p->beta = 1.0;
    p->a = -2.0;
    p->b = 2.0;
    p->tau = 0.25;
    p->c0 = 343.0;
    p->fs = 16000.0;
    p->early_pre_ms = 6.0;
    p->early_post_ms = 50.0;
    p->half_len = 40;
    p->tile = 0;
    p->delay_mode = 0;
    p->reserved = 0;
}

int fram_layout(int32_t B, int32_t S, int32_t M, double fs, const float* rt60, const int32_t* n_vs,
                int32_t* rir_len, int64_t* rir_off, int64_t* vs_off)
{
    if (B < 0 || S < 1 || M < 1 || !(fs > 0.0)) return fail(FRAM_EINVAL, "need B >= 0, S >= 1, M >= 1, fs > 0");
    if (B > 0 && (!rt60 || !n_vs || !rir_len)) return fail(FRAM_EINVAL, "null host array");
    if (!rir_off || !vs_off) return fail(FRAM_EINVAL, "null host array");
    rir_off[0] = 0;
    vs_off[0] = 0;
    for (int32_t b = 0; b < B; ++b) {
        const double t60 = (double)rt60[b];
        if (!(t60 > 0.0) || !std::isfinite(t60)) return fail(FRAM_EINVAL, "room %d: T60 must be > 0", b);
        if (n_vs[b] < 0) return fail(FRAM_EINVAL, "room %d: negative image count", b);
        const double len = std::ceil(t60 * fs);
        if (len < 1.0 || len > 2147483647.0) return fail(FRAM_EINVAL, "room %d: RIR length out of range", b);
        rir_len[b] = (int32_t)len;
        rir_off[b + 1] = rir_off[b] + (int64_t)S * M * (int64_t)rir_len[b];
        vs_off[b + 1] = vs_off[b] + (int64_t)S * (int64_t)n_vs[b];
    }
    return FRAM_OK;
}

int fram_workspace_size(const fram_scene* scene, const fram_params* p, size_t* bytes)
{
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, false)) != FRAM_OK) return rc;
    if (!bytes) return fail(FRAM_EINVAL, "bytes is null");
    if ((rc = check_mr_len(scene, p)) != FRAM_OK) return rc;
    const WsLayout w = ws_layout(*scene, tile_of(p), p->delay_mode, p->fs);
    if (w.max_tiles > 0xffff) return fail(FRAM_EINVAL, "too many tiles per RIR (raise the tile length)");
    *bytes = w.total;
    return FRAM_OK;
}

int fram_sample(const fram_scene* scene, const fram_params* p, uint64_t seed, const uint64_t* d_seed,
                float* vs_pos_hi, float* vs_pos_lo, float* vs_g, float* r, uint32_t* words,
                void* workspace, size_t workspace_bytes, void* stream)
{
    NvtxRange nvtx("fram_sample");
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, true)) != FRAM_OK) return rc;
    WsLayout w;
    if ((rc = check_ws(scene, p, workspace, workspace_bytes, &w)) != FRAM_OK) return rc;
    if (scene->n_vs_total > 0 && (!vs_pos_hi || !vs_g)) return fail(FRAM_EINVAL, "vs_pos_hi and vs_g must not be null");
    const LaunchArgs a = make_args(scene, p, w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(a.hdr, 0, sizeof(Header), st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_sample: clearing the status word");
    e = launch_sample(a, *p, seed, d_seed, vs_pos_hi, vs_pos_lo, vs_g, r, words, st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_sample: launch");
    return FRAM_OK;
}

static int common_checks(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_g,
                         const float* r, void* ws, size_t ws_bytes, WsLayout* w)
{
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, true)) != FRAM_OK) return rc;
    if ((rc = check_ws(scene, p, ws, ws_bytes, w)) != FRAM_OK) return rc;
    if (scene->n_vs_total > 0 && (!vs_pos_hi || !vs_g)) return fail(FRAM_EINVAL, "vs_pos_hi and vs_g must not be null");
    if (scene->B > 0 && !r) return fail(FRAM_EINVAL, "r must not be null");
    return FRAM_OK;
}

int fram_prepare(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_pos_lo,
                 const float* r, void* workspace, size_t workspace_bytes, void* stream)
{
    NvtxRange nvtx("fram_prepare");
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, true)) != FRAM_OK) return rc;
    WsLayout w;
    if ((rc = check_ws(scene, p, workspace, workspace_bytes, &w)) != FRAM_OK) return rc;
    if (scene->n_vs_total > 0 && !vs_pos_hi) return fail(FRAM_EINVAL, "vs_pos_hi must not be null");
    if (scene->B > 0 && !r) return fail(FRAM_EINVAL, "r must not be null");
    const LaunchArgs a = make_args(scene, p, w, workspace);
    cudaError_t e = launch_prepare(a, vs_pos_hi, vs_pos_lo, r, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "fram_prepare");
    return FRAM_OK;
}

int fram_synthesize_prepared(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                             const float* vs_pos_lo, const float* vs_g, const float* r, float* rir, float* early,
                             void* workspace, size_t workspace_bytes, void* stream)
{
    NvtxRange nvtx("fram_synthesize_prepared");
    WsLayout w;
    int rc = common_checks(scene, p, vs_pos_hi, vs_g, r, workspace, workspace_bytes, &w);
    if (rc != FRAM_OK) return rc;
    if (scene->rir_total > 0 && !rir) return fail(FRAM_EINVAL, "rir must not be null");
    if ((reinterpret_cast<uintptr_t>(rir) | reinterpret_cast<uintptr_t>(early)) & 3)
        return fail(FRAM_EINVAL, "rir and early must be 4-byte aligned");
    if (scene->B == 0) return FRAM_OK;
    const LaunchArgs a = make_args(scene, p, w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(&a.hdr->queue, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_synthesize: resetting the work counter");
    if (p->delay_mode == 1) {
        e = launch_amp_gather(a, vs_g, st);     // r^g in sorted order
        if (e == cudaSuccess) e = launch_synthesize_mr(a, vs_pos_hi, vs_pos_lo, rir, early, st);
    } else {
        e = launch_synthesize(a, vs_pos_hi, vs_pos_lo, vs_g, rir, early, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fram_synthesize: launch");
    return FRAM_OK;
}

int fram_synthesize(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_pos_lo,
                    const float* vs_g, const float* r, float* rir, float* early, void* workspace,
                    size_t workspace_bytes, void* stream)
{
    WsLayout w;
    int rc = common_checks(scene, p, vs_pos_hi, vs_g, r, workspace, workspace_bytes, &w);
    if (rc != FRAM_OK) return rc;
    if (scene->rir_total > 0 && !rir) return fail(FRAM_EINVAL, "rir must not be null");
    if ((rc = fram_prepare(scene, p, vs_pos_hi, vs_pos_lo, r, workspace, workspace_bytes, stream)) != FRAM_OK)
        return rc;
    return fram_synthesize_prepared(scene, p, vs_pos_hi, vs_pos_lo, vs_g, r, rir, early, workspace, workspace_bytes,
                                    stream);
}

int fram_synthesize_backward_prepared(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                                      const float* vs_pos_lo, const float* vs_g, const float* r,
                                      const float* grad_rir, const float* grad_early, float* grad_vs, float* grad_mic,
                                      float* grad_src, float* grad_r, float* grad_g, void* workspace,
                                      size_t workspace_bytes, void* stream)
{
    NvtxRange nvtx("fram_synthesize_backward_prepared");
    WsLayout w;
    int rc = common_checks(scene, p, vs_pos_hi, vs_g, r, workspace, workspace_bytes, &w);
    if (rc != FRAM_OK) return rc;
    if (p->delay_mode != 0)
        return fail(FRAM_EINVAL, "the multi-rate path (delay_mode 1) quantises delays and has no adjoint; use delay_mode 0");
    if (scene->B == 0) return FRAM_OK;
    const LaunchArgs a = make_args(scene, p, w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(&a.hdr->queue_bwd, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_synthesize_backward: resetting the work counter");
    e = launch_backward(a, vs_pos_hi, vs_pos_lo, vs_g, r, grad_rir, grad_early, grad_vs, grad_mic, grad_src, grad_r,
                        grad_g, st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_synthesize_backward: launch");
    return FRAM_OK;
}

int fram_synthesize_backward(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                             const float* vs_pos_lo, const float* vs_g, const float* r, const float* grad_rir,
                             const float* grad_early, float* grad_vs, float* grad_mic, float* grad_src, float* grad_r,
                             float* grad_g, void* workspace, size_t workspace_bytes, void* stream)
{
    WsLayout w;
    int rc = common_checks(scene, p, vs_pos_hi, vs_g, r, workspace, workspace_bytes, &w);
    if (rc != FRAM_OK) return rc;
    if (p->delay_mode != 0)
        return fail(FRAM_EINVAL, "the multi-rate path (delay_mode 1) quantises delays and has no adjoint; use delay_mode 0");
    if ((rc = fram_prepare(scene, p, vs_pos_hi, vs_pos_lo, r, workspace, workspace_bytes, stream)) != FRAM_OK)
        return rc;
    return fram_synthesize_backward_prepared(scene, p, vs_pos_hi, vs_pos_lo, vs_g, r, grad_rir, grad_early, grad_vs,
                                             grad_mic, grad_src, grad_r, grad_g, workspace, workspace_bytes, stream);
}

int fram_sample_backward(const fram_scene* scene, const fram_params* p, uint64_t seed, const uint64_t* d_seed,
                         const float* grad_vs, const float* grad_g, const float* grad_r, const float* grad_src_in,
                         const float* grad_mic_in, float* grad_src, float* grad_mic, float* grad_t60, float* grad_dims,
                         void* workspace, size_t workspace_bytes, void* stream)
{
    NvtxRange nvtx("fram_sample_backward");
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, true)) != FRAM_OK) return rc;
    WsLayout w;
    if ((rc = check_ws(scene, p, workspace, workspace_bytes, &w)) != FRAM_OK) return rc;
    if (scene->n_vs_total > 0 && !grad_vs) return fail(FRAM_EINVAL, "grad_vs must not be null");
    if (scene->B == 0) return FRAM_OK;
    const LaunchArgs a = make_args(scene, p, w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Only the status word: the tables a fram_prepare left in the workspace stay valid.
    cudaError_t e = cudaMemsetAsync(&a.hdr->status, 0, sizeof(a.hdr->status), st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_sample_backward: clearing the status word");
    e = launch_sample_backward(a, *p, seed, d_seed, grad_vs, grad_g, grad_r, grad_src_in, grad_mic_in, grad_src,
                               grad_mic, grad_t60, grad_dims, a.sb_part, st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_sample_backward: launch");
    return FRAM_OK;
}

int fram_autotune(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi, const float* vs_pos_lo,
                  const float* vs_g, const float* r, float* rir, void* workspace, size_t workspace_bytes, void* stream,
                  int32_t* tile_out)
{
    NvtxRange nvtx("fram_autotune");
    WsLayout w0;
    fram_params base = *p;
    base.tile = 0;
    int rc = common_checks(scene, &base, vs_pos_hi, vs_g, r, workspace, workspace_bytes, &w0);
    if (rc != FRAM_OK) return rc;
    if (scene->rir_total > 0 && !rir) return fail(FRAM_EINVAL, "rir must not be null");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "fram_autotune: event");
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "fram_autotune: event"); }
    int best = kDefaultTile;
    float best_ms = 3.0e38f;
    for (int T : kTileCandidates) {
        fram_params cand = *p;
        cand.tile = T;
        const WsLayout w = ws_layout(*scene, T, p->delay_mode, p->fs);
        if (w.max_tiles > 0xffff || w.total > workspace_bytes) continue;
        if (synth_smem_total(T) > 227 * 1024) continue;
        rc = fram_synthesize(scene, &cand, vs_pos_hi, vs_pos_lo, vs_g, r, rir, nullptr, workspace, workspace_bytes,
                             stream);
        if (rc != FRAM_OK) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && rc == FRAM_OK; ++rep)
            rc = fram_synthesize(scene, &cand, vs_pos_hi, vs_pos_lo, vs_g, r, rir, nullptr, workspace,
                                 workspace_bytes, stream);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "fram_autotune: timing"); break; }
        if (rc != FRAM_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = T; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FRAM_OK) return rc;
    const TuneKey k = tune_key(scene, p);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        bool found = false;
        for (auto& ent : g_tune)
            if (ent.first == k) { ent.second = best; found = true; }
        if (!found) g_tune.push_back({k, best});
        store_cache(k, best);
    }
    if (tile_out) *tile_out = best;
    return FRAM_OK;
}

int fram_tuned_tile(const fram_scene* scene, const fram_params* p, int32_t* tile)
{
    int rc;
    if ((rc = check_params(p)) != FRAM_OK) return rc;
    if ((rc = check_scene(scene, false)) != FRAM_OK) return rc;
    if (!tile) return fail(FRAM_EINVAL, "tile is null");
    *tile = tile_for(scene, p);
    return FRAM_OK;
}

int fram_status(void* workspace, void* stream, int32_t* flags)
{
    if (!workspace || !flags) return fail(FRAM_EINVAL, "workspace and flags must not be null");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fram_status: stream synchronize");
    int32_t v = 0;
    e = cudaMemcpy(&v, workspace, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fram_status: reading the status word");
    *flags = v;
    if (v != 0) return fail(FRAM_EDEVICE, "device status 0x%x", v);
    return FRAM_OK;
}

}  // extern "C"
