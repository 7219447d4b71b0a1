// Range-profile table, step (8a) / (19a) of the paper, per (channel, k_z bin):
//
//   b_i = sum_m S[c][u][m] alpha[u][m] e^{j theta_um (i - L/2)},  i < L
//
// where alpha folds the per-(k_z, f) compensation (the k weight of Eq. 7, the
// evanescent mask, the kernel deconvolution 1/phihat and the range-origin
// phase) and theta_um = kappa''_um h (see setup.cu). This is a type-1
// nonuniform FFT: the M sources are spread with an ES kernel onto a periodic
// fine grid of `fine` points using shared-memory atomics, transformed by a
// radix-2 FFT in shared memory, and divided by the spreading kernel's
// transform.
//
// One warp owns one (c, u) problem at a time and its fine grid in shared
// memory; a block of 8 warps covers 16 consecutive k_z bins of one channel
// and writes the [L][16] output panel as coalesced 128-byte rows of the
// table b[c][i][u] (u fastest, in planar pairs {re_u, re_u+1, im_u, im_u+1},
// N_p rounded up to even), the layout the back-projection stages.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kUB = 16;       // k_z bins per block
constexpr int kWarps = 8;

__global__ void __launch_bounds__(kWarps * 32)
k_range_table(NufftDesc d, const float2 *__restrict__ S, const float2 *__restrict__ alpha,
              const float *__restrict__ xg, const float *__restrict__ dec,
              const float2 *__restrict__ tw_g, void *__restrict__ table, int bf16) {
    extern __shared__ float2 smem[];
    const int fine = d.fine;
    const int lg = d.log2_fine;
    float2 *tw = smem;                                  // fine/2: e^{+2 pi i q / fine}
    float2 *panel = tw + fine / 2;                      // [L][kUB]
    float2 *grids = panel + d.L * kUB;                  // [kWarps][fine]
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float2 *grid = grids + warp * fine;
    const int c = blockIdx.y;
    const int u0 = blockIdx.x * kUB;
    const float two_over_w1 = 2.0f / d.w1;
    const float half_w1 = 0.5f * d.w1;

    for (int q = threadIdx.x; q < fine / 2; q += blockDim.x) tw[q] = tw_g[q];
    __syncthreads();

    for (int ul = warp; ul < kUB; ul += kWarps) {
        const int u = u0 + ul;
        if (u >= d.n_pad) {
            for (int i = lane; i < d.L; i += 32) panel[i * kUB + ul] = make_float2(0.f, 0.f);
            continue;
        }
        for (int g = lane; g < fine; g += 32) grid[g] = make_float2(0.f, 0.f);
        __syncwarp();
        // spread (compensation fused): sources to bit-reversed fine-grid slots
        const float2 *Su = S + ((size_t)c * d.n_pad + u) * d.n_f;
        for (int m = lane; m < d.n_f; m += 32) {
            const float2 a = cmul(Su[m], alpha[u * d.n_f + m]);
            if (a.x == 0.f && a.y == 0.f) continue;
            const float x = xg[u * d.n_f + m];
            const int g0 = (int)ceilf(x - half_w1);
            for (int t = 0; t < d.w1; ++t) {
                const int g = g0 + t;
                const float wgt = es_kernel((float)g - x, two_over_w1, d.beta1);
                const int gi = __brev((unsigned)(g & (fine - 1))) >> (32 - lg);
                atomicAdd(&grid[gi].x, a.x * wgt);
                atomicAdd(&grid[gi].y, a.y * wgt);
            }
        }
        __syncwarp();
        // in-place radix-2 decimation-in-time FFT, exponent +
        for (int s = 0; s < lg; ++s) {
            const int half = 1 << s;
            for (int bf = lane; bf < fine / 2; bf += 32) {
                const int k = bf & (half - 1);
                const int i0 = ((bf >> s) << (s + 1)) + k;
                const int i1 = i0 + half;
                const float2 w = tw[k << (lg - 1 - s)];
                const float2 v0 = grid[i0];
                const float2 v1 = cmul(grid[i1], w);
                grid[i0] = cadd(v0, v1);
                grid[i1] = csub(v0, v1);
            }
            __syncwarp();
        }
        // deconvolve and keep rows j = i - L/2
        for (int i = lane; i < d.L; i += 32) {
            const int gi = (i - d.L / 2) & (fine - 1);
            panel[i * kUB + ul] = cscale(grid[gi], dec[i]);
        }
        __syncwarp();
    }
    __syncthreads();

    // table rows hold k_z bins in planar pairs: {re_u, re_u+1, im_u, im_u+1}
    const int np2 = (d.n_pad + 1) / 2;
    const int p0 = u0 / 2;
    const int npair = min(kUB / 2, np2 - p0);
    if (!bf16) {
        float4 *b = reinterpret_cast<float4 *>(table) + (size_t)c * d.L * np2;
        for (int idx = threadIdx.x; idx < d.L * (kUB / 2); idx += blockDim.x) {
            const int i = idx / (kUB / 2);
            const int pp = idx - i * (kUB / 2);
            if (pp >= npair) continue;
            const float2 a = panel[i * kUB + 2 * pp];
            const float2 e = panel[i * kUB + 2 * pp + 1];
            b[(size_t)i * np2 + p0 + pp] = make_float4(a.x, e.x, a.y, e.y);
        }
    } else {
        uint2 *b = reinterpret_cast<uint2 *>(table) + (size_t)c * d.L * np2;
        for (int idx = threadIdx.x; idx < d.L * (kUB / 2); idx += blockDim.x) {
            const int i = idx / (kUB / 2);
            const int pp = idx - i * (kUB / 2);
            if (pp >= npair) continue;
            const float2 a = panel[i * kUB + 2 * pp];
            const float2 e = panel[i * kUB + 2 * pp + 1];
            __nv_bfloat162 re = __floats2bfloat162_rn(a.x, e.x);
            __nv_bfloat162 im = __floats2bfloat162_rn(a.y, e.y);
            uint2 v;
            v.x = *reinterpret_cast<unsigned *>(&re);
            v.y = *reinterpret_cast<unsigned *>(&im);
            b[(size_t)i * np2 + p0 + pp] = v;
        }
    }
}

}  // namespace

size_t range_table_smem_bytes(const NufftDesc &d) {
    return (size_t)(d.fine / 2 + d.L * kUB + kWarps * d.fine) * sizeof(float2);
}

cudaError_t launch_range_table(const NufftDesc &d, const float2 *S, const float2 *alpha,
                               const float *xg, const float *dec, const float2 *tw_fine,
                               void *table, int bf16, cudaStream_t st) {
    const size_t smem = range_table_smem_bytes(d);
    cudaError_t e = cudaFuncSetAttribute(k_range_table,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((d.n_pad + kUB - 1) / kUB, d.n_chan);
    k_range_table<<<grid, kWarps * 32, smem, st>>>(d, S, alpha, xg, dec, tw_fine, table, bf16);
    return cudaGetLastError();
}
