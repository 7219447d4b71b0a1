// Scene simulation (input synthesis for benchmarks and training data, not a
// reconstruction step): echo of point scatterers, Eq. (1) / Eq. (10),
//   echo[c][n][m] = sum_t amp_t exp(-j k_m (R_T + R_R)).
// Thread = (channel, scan position, 8 frequencies); points staged in shared
// memory in chunks. FP32 ranges and phases (error ~2e-4 rad at 2 m, 34 GHz).
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kMC = 8;        // frequencies per thread
constexpr int kPts = 256;     // points per shared-memory chunk

__global__ void __launch_bounds__(128)
k_synth_echo(int n_chan, const float4 *__restrict__ ch, int n_scan, float z0, float dz, int n_f,
             const float *__restrict__ k, int n_pts, const float4 *__restrict__ pts,
             const float2 *__restrict__ amp, float2 *__restrict__ echo) {
    __shared__ float4 sp[kPts];
    __shared__ float2 sa[kPts];
    const int n_mc = (n_f + kMC - 1) / kMC;
    const long long total = (long long)n_chan * n_scan * n_mc;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = tid < total;
    int c = 0, n = 0, mc = 0;
    if (live) {
        mc = (int)(tid % n_mc);
        const long long cn = tid / n_mc;
        n = (int)(cn % n_scan);
        c = (int)(cn / n_scan);
    }
    const float4 cp = live ? ch[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float zs = z0 + n * dz;
    float km[kMC];
    float2 acc[kMC];
#pragma unroll
    for (int q = 0; q < kMC; ++q) {
        const int m = mc * kMC + q;
        km[q] = (live && m < n_f) ? k[m] : 0.f;
        acc[q] = make_float2(0.f, 0.f);
    }
    for (int t0 = 0; t0 < n_pts; t0 += kPts) {
        const int nt = min(kPts, n_pts - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            sp[i] = pts[t0 + i];
            sa[i] = amp[t0 + i];
        }
        __syncthreads();
        if (!live) continue;
        for (int i = 0; i < nt; ++i) {
            const float4 q = sp[i];
            const float dzz = q.z - zs;
            const float dxt = q.x - cp.x, dyt = q.y - cp.y;
            const float dxr = q.x - cp.z, dyr = q.y - cp.w;
            const float rs = sqrtf(dxt * dxt + dyt * dyt + dzz * dzz) +
                             sqrtf(dxr * dxr + dyr * dyr + dzz * dzz);
            const float2 a = sa[i];
#pragma unroll
            for (int qq = 0; qq < kMC; ++qq) {
                float s, co;
                __sincosf(-km[qq] * rs, &s, &co);
                acc[qq].x += a.x * co - a.y * s;
                acc[qq].y += a.x * s + a.y * co;
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int q = 0; q < kMC; ++q) {
        const int m = mc * kMC + q;
        if (m < n_f) echo[((size_t)c * n_scan + n) * n_f + m] = acc[q];
    }
}

}  // namespace

cudaError_t launch_synth_echo(int n_chan, const float4 *ch, int n_scan, float z0, float dz,
                              int n_f, const float *k, int n_pts, const float4 *pts,
                              const float2 *amp, float2 *echo, cudaStream_t st) {
    const long long total = (long long)n_chan * n_scan * ((n_f + kMC - 1) / kMC);
    const int blocks = (int)((total + 127) / 128);
    k_synth_echo<<<blocks, 128, 0, st>>>(n_chan, ch, n_scan, z0, dz, n_f, k, n_pts, pts, amp,
                                         echo);
    return cudaGetLastError();
}
