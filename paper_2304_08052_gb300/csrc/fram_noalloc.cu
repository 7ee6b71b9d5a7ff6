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
// the array's name as a device address, so the first call on each device (with that device
// current) asks the runtime for the address with cudaGetSymbolAddress and caches it; that
// first call should happen before any stream capture begins.  No call here allocates memory.
#include <cstdio>
#include <mutex>

#include "fram_internal.cuh"

namespace fram {
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int fram_synthesize_noalloc(const fram_scene* scene, const fram_params* p, const float* vs_pos_hi,
                                       const float* vs_pos_lo, const float* vs_g, const float* r, float* rir,
                                       float* early, void* stream)
{
    size_t need = 0;
    const int rc = fram_workspace_size(scene, p, &need);
    if (rc != FRAM_OK) return rc;
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "fram_synthesize_noalloc: this scene needs %zu bytes of scratch but the static scratch holds %zu "
                 "(16 MiB); use fram_synthesize with a workspace",
                 need, kStaticScratchBytes);
        return fram::record_error(FRAM_EWORKSPACE, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fram::record_error(FRAM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fram::record_error(FRAM_EINVAL, "device index out of range");
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr)
                return fram::record_error(FRAM_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
            g_scratch_ptr[dev] = ptr;
        }
        ws = g_scratch_ptr[dev];
    }
    // The status word and work counters at the start of the scratch are cleared by the
    // preparation inside fram_synthesize; everything else is rewritten before it is read.
    return fram_synthesize(scene, p, vs_pos_hi, vs_pos_lo, vs_g, r, rir, early, ws, kStaticScratchBytes, stream);
}
