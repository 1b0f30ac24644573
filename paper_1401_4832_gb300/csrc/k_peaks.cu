// k_peaks.cu -- measured instruction-throughput peaks of the CUDA cores, the
// denominators of the ALU-bound rooflines (the method's own additions, the
// FP32 gather path and the popcount reweighting).
//
// Every thread runs 16 independent dependency chains of one instruction
// (inline PTX, volatile so that nothing is folded or dropped); with 32 warps
// per SM the issue slots, not the latencies, set the rate.  The chains'
// final values go to a file-scope device sink behind a condition that never
// holds in practice, so the compiler cannot discard them.
#include <cstdint>

#include "../../include/plmdca.h"
#include "plm_internal.cuh"

namespace {

constexpr int PK_CHAINS = 16;
constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 4;

__device__ unsigned long long g_peak_sink;

template <int KIND>
__global__ void __launch_bounds__(PK_THREADS) k_peak(int iters, float seed)
{
    float f[PK_CHAINS];
    double d[PK_CHAINS];
    uint32_t u[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) {
        f[c] = seed * (float)(threadIdx.x + c);
        d[c] = (double)f[c];
        u[c] = (uint32_t)(threadIdx.x * 2654435761u + c);
    }
    const float fb = seed * 1e-7f;
    const double db = (double)fb;
    const uint32_t ub = (uint32_t)blockIdx.x | 0x5A5A0000u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) {
            if (KIND == 0) {
                asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(f[c]) : "f"(fb));
            } else if (KIND == 1) {
                asm volatile("fma.rn.f32 %0, %0, %1, %1;" : "+f"(f[c]) : "f"(fb));
            } else if (KIND == 2) {
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[c]) : "d"(db));
            } else if (KIND == 3) {
                // x = x ^ (ub | x), one three-input logic op (table 0x1E)
                asm volatile("lop3.b32 %0, %0, %1, %0, 0x1E;" : "+r"(u[c]) : "r"(ub));
            } else {
                asm volatile("popc.b32 %0, %0;" : "+r"(u[c]));
            }
        }
    }
    unsigned long long acc = 0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c)
        acc += (unsigned long long)__float_as_uint(f[c]) + (unsigned long long)__double_as_longlong(d[c]) + u[c];
    if (acc == 0x0123456789ABCDEFull) g_peak_sink = acc;
}

template <int KIND>
cudaError_t launch_peak(int grid, int iters, float seed, cudaStream_t st)
{
    k_peak<KIND><<<grid, PK_THREADS, 0, st>>>(iters, seed);
    plm::count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int grid, int iters, cudaStream_t st)
{
    switch (kind) {
    case 0: return launch_peak<0>(grid, iters, 1.0f, st);
    case 1: return launch_peak<1>(grid, iters, 1.0f, st);
    case 2: return launch_peak<2>(grid, iters, 1.0f, st);
    case 3: return launch_peak<3>(grid, iters, 1.0f, st);
    default: return launch_peak<4>(grid, iters, 1.0f, st);
    }
}

}  // namespace

extern "C" plm_status plm_measure_peak(int kind, void *cuda_stream, double *ops_per_s)
{
    if (kind < 0 || kind > 4 || !ops_per_s) return PLM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    const int grid = sms * PK_BLOCKS_PER_SM;
    // FP64 runs at a small fraction of the FP32 rate on this GPU: fewer
    // iterations keep every launch near a millisecond
    const int iters = kind == 2 ? 256 : 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return PLM_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    float best = 0.0f;
    for (int rep = 0; rep < 7 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_kind(kind, grid, iters, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep >= 2 && (best == 0.0f || ms < best)) best = ms;  // 2 warm-ups
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || best <= 0.0f) {
        cudaGetLastError();
        return PLM_ECUDA;
    }
    const double ops = (double)grid * PK_THREADS * PK_CHAINS * (double)iters;
    *ops_per_s = ops / (best * 1e-3);
    return PLM_OK;
}
