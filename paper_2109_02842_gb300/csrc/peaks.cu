// Micro-benchmarks of the three units that bound the FP32 back-projection
// (FP32 FMA pipe, the MUFU sin/cos unit, shared-memory bandwidth), so that
// its roofline is taken against measured rather than nominal rates. Each one
// saturates every SM with independent work for a fixed number of iterations
// and is timed with CUDA events on the caller's stream; nothing is changed on
// the device (no clock, power or mode setting).
#include <cuda_runtime.h>

#include "../../include/polyline.h"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;          // independent dependency chains per thread

// Written only under a condition the inputs never meet (keeps the work live).
__device__ float g_sink[kThreads];

// kChains FMA chains per thread, `iters` x 16 FMAs each.
__global__ void __launch_bounds__(kThreads) k_peak_fma(int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) g_sink[threadIdx.x] = s;   // never true for the inputs used
}

// kChains sin chains per thread (the MUFU unit), `iters` x 16 each.
__global__ void __launch_bounds__(kThreads) k_peak_mufu(int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __sinf(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) g_sink[threadIdx.x] = s;
}

// Conflict-free 16-byte shared-memory loads: each warp reads 512 consecutive
// bytes per access; `iters` x 16 loads per thread.
__global__ void __launch_bounds__(kThreads) k_peak_smem(int iters) {
    __shared__ float4 buf[kThreads * 4];
    for (int i = threadIdx.x; i < kThreads * 4; i += kThreads)
        buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            // a volatile load, so neither compiler can keep the (repeating)
            // values in registers instead of reading them again
            float4 v;
            const unsigned a = (unsigned)__cvta_generic_to_shared(
                &buf[(idx + k * kThreads) & (kThreads * 4 - 1)]);
            asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "r"(a));
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx ^= 32;        // changes the address stream without bank conflicts
    }
    if (acc.x + acc.y + acc.z + acc.w == 12345.678f) g_sink[threadIdx.x] = acc.x;
}

}  // namespace

extern "C" pl_status pl_measure_peak(int which, void *stream, double *value) {
    if (!value || which < 0 || which > 2) return pl_internal_fail(PL_ERR_ARG, "bad pl_measure_peak");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "pl_measure_peak");
    const void *fn = which == 0 ? (const void *)k_peak_fma
                                : (which == 1 ? (const void *)k_peak_mufu : (const void *)k_peak_smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "pl_measure_peak");
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = which == 0 ? 4096 : (which == 1 ? 1024 : 2048);
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // first run warms up
        e = cudaEventRecord(a, st);
        if (e != cudaSuccess) break;
        if (which == 0)
            k_peak_fma<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-4f);
        else if (which == 1)
            k_peak_mufu<<<blocks, kThreads, 0, st>>>(iters);
        else
            k_peak_smem<<<blocks, kThreads, 0, st>>>(iters);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "pl_measure_peak");
    const double per_thread = (double)iters * 16 * (which == 2 ? 1 : kChains);
    const double ops = per_thread * blocks * kThreads;
    const double s = best * 1e-3;
    if (which == 0) *value = 2.0 * ops / s / 1e12;          // TFLOP/s (2 per FMA)
    else if (which == 1) *value = ops / s / 1e9;            // G sin/s
    else *value = 16.0 * ops / s / 1e9;                     // GB/s
    return PL_OK;
}
