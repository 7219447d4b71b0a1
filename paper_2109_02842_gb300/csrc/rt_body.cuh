// Range-table block body shared by the per-scan kernel (range_table.cu) and
// the batched persistent kernel (batch.cu). See range_table.cu.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "stockham.cuh"

namespace rt {

// One block's work: channel c, k_z bins [ub UB, ub UB + UB).
template <int UB>
__device__ __forceinline__ void rt_block(const NufftDesc &d, const FftPlan &fp,
                                         const float2 *__restrict__ S,
                                         const float2 *__restrict__ alpha,
                                         const float *__restrict__ xg,
                                         const float *__restrict__ dec,
                                         const float2 *__restrict__ tw_g, void *__restrict__ table,
                                         int fmt, int c, int ub, float2 *smem) {
    const int fine = d.fine;
    float2 *tw = smem;                          // [fine]: exp(-2 pi i k / fine)
    float2 *buf0 = tw + fine;                   // [UB][fine]
    float2 *buf1 = buf0 + UB * fine;            // [UB][fine]
    const int u0 = ub * UB;
    const float two_over_w1 = 2.0f / d.w1;
    const float half_w1 = 0.5f * d.w1;

    for (int k = threadIdx.x; k < fine; k += blockDim.x) tw[k] = tw_g[k];
    for (int k = threadIdx.x; k < UB * fine; k += blockDim.x) buf0[k] = make_float2(0.f, 0.f);
    __syncthreads();

    // spread (compensation fused): source m of bin u onto row u of the grid
    for (int idx = threadIdx.x; idx < UB * d.n_f; idx += blockDim.x) {
        const int ul = idx / d.n_f;
        const int m = idx - ul * d.n_f;
        const int u = u0 + ul;
        if (u >= d.n_pad) continue;
        const float2 a = cmul(S[((size_t)c * d.n_pad + u) * d.n_f + m], alpha[u * d.n_f + m]);
        if (a.x == 0.f && a.y == 0.f) continue;
        const float x = xg[u * d.n_f + m];
        const int g0 = (int)ceilf(x - half_w1);
        float2 *row = buf0 + ul * fine;
        for (int t = 0; t < d.w1; ++t) {
            const int g = g0 + t;
            const float wgt = es_kernel((float)g - x, two_over_w1, d.beta1);
            float2 *cell = row + (g < 0 ? g + fine : g);   // |g| < fine: one wrap at most
            atomicAdd(&cell->x, a.x * wgt);
            atomicAdd(&cell->y, a.y * wgt);
        }
    }
    __syncthreads();

    // inverse transform of every row (exponent +)
    const float2 *res = stockham_run<false>(buf0, buf1, tw, fp, +1, UB, fine, 1);

    // deconvolve, keep rows j = i - L/2
    if (fmt == 4) {
        // tensor-core layout [c][plane hi/lo][row][column 2u + (re, im)], BF16,
        // hi = BF16(x) and lo = BF16(x - hi); bins past N_p stay zero
        __nv_bfloat16 *tb = reinterpret_cast<__nv_bfloat16 *>(table);
        for (int idx = threadIdx.x; idx < UB * d.L; idx += blockDim.x) {
            const int i = idx / UB;
            const int ul = idx - i * UB;
            if (u0 + ul >= d.n_pad) continue;
            const int j = i < d.L / 2 ? i - d.L / 2 + fine : i - d.L / 2;
            const float2 v = cscale(res[ul * fine + j], dec[i]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
            const size_t o = (((size_t)c * 2) * d.L + i) * d.tc_cols + 2 * (size_t)(u0 + ul);
            *reinterpret_cast<__nv_bfloat162 *>(tb + o) = h;
            *reinterpret_cast<__nv_bfloat162 *>(tb + o + (size_t)d.L * d.tc_cols) = l;
        }
        return;
    }
    // planar bin pairs
    const int np2 = (d.n_pad + 1) / 2;
    const int p0 = u0 / 2;
    constexpr int NPR = UB / 2;
    for (int idx = threadIdx.x; idx < d.L * NPR; idx += blockDim.x) {
        const int i = idx / NPR;
        const int q = idx - i * NPR;
        if (p0 + q >= np2) continue;
        const int j = i < d.L / 2 ? i - d.L / 2 + fine : i - d.L / 2;
        const float s = dec[i];
        const float2 a = cscale(res[(2 * q) * fine + j], s);
        const float2 e = cscale(res[(2 * q + 1) * fine + j], s);
        const size_t o = ((size_t)c * d.L + i) * np2 + p0 + q;
        if (fmt == 0) {
            reinterpret_cast<float4 *>(table)[o] = make_float4(a.x, e.x, a.y, e.y);
        } else {
            __nv_bfloat162 re = __floats2bfloat162_rn(a.x, e.x);
            __nv_bfloat162 im = __floats2bfloat162_rn(a.y, e.y);
            uint2 v;
            v.x = *reinterpret_cast<unsigned *>(&re);
            v.y = *reinterpret_cast<unsigned *>(&im);
            reinterpret_cast<uint2 *>(table)[o] = v;
        }
    }
}

inline int bins_per_block(int fine) { return fine <= 512 ? 16 : (fine <= 1024 ? 8 : 4); }

}  // namespace rt
