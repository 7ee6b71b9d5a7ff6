// fram_noalloc.cu -- fram_synthesize_noalloc: RIR synthesis without a caller-provided
// workspace, for callers that cannot allocate device memory at all.
//
// Who needs it: code that runs where device allocation is off limits -- a plugin inside a
// host application whose memory is owned by that application's allocator, a real-time audio
// or streaming thread that must not block (cudaMalloc/cudaFree can synchronise the whole
// device), or a deployment with a fixed, preassigned device-memory budget.  Such callers can
// still hand over their input and output buffers, but they cannot create the scratch
// workspace that fram_synthesize needs.
//
// How: the scratch lives in one file-scope __device__ array of kStaticScratchBytes (16 MiB).
// Every GPU that loads libfram reserves it for the life of the process.  Host code cannot use
// the array's name as a device address; the address comes from cudaGetSymbolAddress, and it
// belongs to the CUDA context that is current (each context -- the device's primary context, a
// context a host application created with the driver API, or a primary context re-created after
// cudaDeviceReset -- has its own copy of the array).  So the address is looked up again on every
// call made outside stream capture, and remembered per context for calls made while the stream is
// being captured (a capture may not trigger the lookup).  No call here allocates memory.
#include <cstdio>
#include <mutex>
#include <utility>
#include <vector>

#include "fram_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

typedef int (*CtxGetCurrentFn)(void** ctx);   // cuCtxGetCurrent, through the runtime's entry-point query

std::mutex g_scratch_mu;
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_get_tried = false;
std::vector<std::pair<void*, void*>> g_scratch_by_ctx;   // (context, scratch address)

// The current context (null on error or when the driver entry point is unavailable).
void* current_context()
{
    if (!g_ctx_get_tried) {
        g_ctx_get_tried = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    void* ctx = nullptr;
    if (!g_ctx_get || g_ctx_get(&ctx) != 0) return nullptr;
    return ctx;
}

}  // namespace

extern "C" int fram_synthesize_noalloc(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                                       const float* vs_pos_lo, const float* vs_g, const float* r, float* rir,
                                       float* early, void* stream)
{
    size_t need = 0;
    const int rc = fram::workspace_bytes_at_launch_tile(scene, p, &need);
    if (rc != FRAM_OK) return rc;
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "fram_synthesize_noalloc: this scene needs %zu bytes of scratch but the static scratch holds %zu "
                 "(16 MiB); use fram_synthesize with a workspace",
                 need, kStaticScratchBytes);
        return fram::record_error(FRAM_EWORKSPACE, msg);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return fram::record_error(FRAM_ECUDA, cudaGetErrorString(e));
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        void* ctx = current_context();
        if (cap == cudaStreamCaptureStatusNone) {
            e = cudaGetSymbolAddress(&ws, g_static_scratch);
            if (e != cudaSuccess || !ws)
                return fram::record_error(FRAM_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
            if (ctx) {
                bool found = false;
                for (auto& kv : g_scratch_by_ctx)
                    if (kv.first == ctx) { kv.second = ws; found = true; }
                if (!found) g_scratch_by_ctx.emplace_back(ctx, ws);
            }
        } else {
            for (const auto& kv : g_scratch_by_ctx)
                if (ctx && kv.first == ctx) ws = kv.second;
            if (!ws)
                return fram::record_error(FRAM_ECUDA,
                                          "fram_synthesize_noalloc: the first call in this CUDA context must come "
                                          "before stream capture (the scratch address is looked up outside capture)");
        }
    }
    // The status word and work counters at the start of the scratch are cleared by the
    // preparation inside fram_synthesize; everything else is rewritten before it is read.
    return fram_synthesize(scene, p, vs_pos_hi, vs_pos_lo, vs_g, r, rir, early, ws, kStaticScratchBytes, stream);
}
