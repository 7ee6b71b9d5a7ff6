// fram_peaks.cu -- throughput probes for the roofline's ALU denominators: scalar FP32 fused
// multiply-add, packed FP32 (fma.rn.f32x2) and the MUFU reciprocal (rcp.approx.ftz.f32), the
// three instruction kinds the synthesis and adjoint kernels spend their time in.  Each probe fills
// every SM with 8 CTAs of 256 threads; every thread runs 8 independent dependency chains so the
// pipes, not latencies, set the rate.  The SM clock counter (clock64) brackets each CTA's loop, so
// the result is reported per SM clock as well as per second.
#include <cstdint>
#include <vector>

#include "fram_internal.cuh"

namespace fram {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;
constexpr int kChains = 8;
constexpr int kUnroll = 64;
constexpr int kMaxProbeCtas = 64 * 1024;

__device__ float g_probe_sink[1];                    // written only if a chain hits a sentinel
__device__ long long g_probe_cycles[kMaxProbeCtas];  // SM cycles of each CTA's loop

__device__ __forceinline__ float rcp_chain(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kind 0: FFMA, kind 1: packed FFMA (two lanes of work per instruction), kind 2: MUFU reciprocal
// (each followed by an FP32 add of a runtime constant, so that the compiler cannot fold a
// reciprocal of a reciprocal back into its argument; the add runs on the FP32 pipe, which has
// several times the MUFU rate).
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, kProbeCtasPerSm) alu_probe(int64_t iters, float a, float b,
                                                                            float* __restrict__ sink,
                                                                            long long* __restrict__ cycles)
{
    float x[kChains];
    f32x2 y[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        x[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
        y[k] = pack2(x[k], x[k] + 0.5f);
    }
    const f32x2 a2 = pack2(a, a), b2 = pack2(b, b);
    __syncthreads();
    const long long t0 = clock64();
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (KIND == 0) x[k] = __fmaf_rn(x[k], a, b);
                else if (KIND == 1) y[k] = fma2(y[k], a2, b2);
                else x[k] = __fadd_rn(rcp_chain(x[k]), b);   // x -> 1/x + b: no fold of two reciprocals
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        unpack2(y[k], lo, hi);
        s += x[k] + lo + hi;
    }
    if (s == 1234.5f) sink[0] = s;   // keeps the chains live (a one-element sink)
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace fram

using namespace fram;

extern "C" int fram_measure_alu(int32_t kind, int64_t iters, double* result, void* stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || !result)
        return record_error(FRAM_EINVAL, "fram_measure_alu: kind must be 0, 1 or 2, iters >= 1, result non-null");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = device_sm_count();
    const int grid = sms * kProbeCtasPerSm;
    if (grid > kMaxProbeCtas) return record_error(FRAM_EINVAL, "fram_measure_alu: too many SMs");
    float* d_sink = nullptr;
    long long* d_cyc = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&d_sink, g_probe_sink);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d_cyc, g_probe_cycles);
    if (e != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    }
    const float a = 0.999f, b = 1e-4f;
    cudaEventRecord(e0, st);
    if (kind == 0) alu_probe<0><<<grid, kProbeThreads, 0, st>>>(iters, a, b, d_sink, d_cyc);
    else if (kind == 1) alu_probe<1><<<grid, kProbeThreads, 0, st>>>(iters, a, b, d_sink, d_cyc);
    else alu_probe<2><<<grid, kProbeThreads, 0, st>>>(iters, a, b, d_sink, d_cyc);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    std::vector<long long> host_cyc(grid);
    if ((e = cudaMemcpy(host_cyc.data(), d_cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return record_error(FRAM_ECUDA, cudaGetErrorString(e));
    long long mx = 0;
    for (int i = 0; i < grid; ++i) mx = host_cyc[i] > mx ? host_cyc[i] : mx;
    const double per_thread = (double)iters * kUnroll * kChains * (kind == 1 ? 2.0 : 1.0);
    result[0] = (double)ms;                                             // kernel time, ms
    result[1] = (double)mx;                                             // SM cycles of the longest CTA
    result[2] = per_thread * (double)grid * kProbeThreads;              // lane operations
    result[3] = (double)sms;
    return FRAM_OK;
}
