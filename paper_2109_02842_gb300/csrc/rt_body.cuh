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
    float2 *src_a = buf1 + UB * fine;           // [UB][M]: S alpha of every source
    float *src_x = reinterpret_cast<float *>(src_a + UB * d.n_f);   // [UB][M]: position
    const int u0 = ub * UB;
    const float two_over_w1 = 2.0f / d.w1;
    const float half_w1 = 0.5f * d.w1;

    for (int k = threadIdx.x; k < fine; k += blockDim.x) tw[k] = tw_g[k];
    for (int k = threadIdx.x; k < 2 * UB * fine; k += blockDim.x) buf0[k] = make_float2(0.f, 0.f);
    // compensation fused into the sources: a = S alpha (0 for bins past N_p)
    for (int idx = threadIdx.x; idx < UB * d.n_f; idx += blockDim.x) {
        const int ul = idx / d.n_f;
        const int m = idx - ul * d.n_f;
        const int u = u0 + ul;
        float2 a = make_float2(0.f, 0.f);
        float x = 0.f;
        if (u < d.n_pad) {
            const size_t si = ((size_t)c * d.n_pad + u) * d.n_f + m;
            const float2 sv = d.s_bf16
                                  ? __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(S)[si])
                                  : S[si];
            a = cmul(sv, alpha[(size_t)u * d.n_f + m]);
            x = xg[(size_t)u * d.n_f + m];
        }
        src_a[idx] = a;
        src_x[idx] = x;
    }
    __syncthreads();

    // spread: source m of bin u onto row u of the grid. Deterministic: the 8
    // lanes of a group own one bin and a tap each (the w1 <= 8 taps of one
    // source hit distinct cells) and add the sources in a fixed order, a
    // __syncwarp between successive sources; the first half of the sources
    // goes to buf0 (threads 0 .. 8 UB - 1), the second to buf1 (the next 8 UB),
    // and the two are added in a fixed order. No atomics: the sums do not
    // depend on scheduling.
    if (threadIdx.x < 2 * UB * 8) {
        const int half = threadIdx.x >= UB * 8;
        const int lt = threadIdx.x - half * UB * 8;
        const int ul = lt >> 3;
        const int t = lt & 7;
        const bool live = t < d.w1;
        float2 *row = (half ? buf1 : buf0) + ul * fine;
        const int mh = (d.n_f + 1) / 2;
        const int m0 = half ? mh : 0, m1 = half ? d.n_f : mh;
        const float2 *sa = src_a + ul * d.n_f;
        const float *sx = src_x + ul * d.n_f;
        for (int m = m0; m < m1; ++m) {
            const float2 a = sa[m];
            if (live && (a.x != 0.f || a.y != 0.f)) {
                const float x = sx[m];
                const int g = (int)ceilf(x - half_w1) + t;
                const float wgt = es_kernel((float)g - x, two_over_w1, d.beta1);
                float2 *cell = row + (g < 0 ? g + fine : g);   // |g| < fine: one wrap at most
                cell->x += a.x * wgt;
                cell->y += a.y * wgt;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < UB * fine; k += blockDim.x) buf0[k] = cadd(buf0[k], buf1[k]);
    __syncthreads();

    // inverse transform of every row (exponent +)
    const float2 *res = stockham_run<false, UB>(buf0, buf1, tw, fp, +1, fine, 1);

    // deconvolve, keep rows j = i - L/2
    if (fmt == 4) {
        // tensor-core layout [c][plane hi/lo][row][column 2u + (re, im)] (or
        // planar: Re at column u, Im at tc_cols / 2 + u), BF16,
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
            const size_t row = (((size_t)c * 2) * d.L + i) * d.tc_cols;
            const size_t lo = (size_t)d.L * d.tc_cols;
            if (d.tc_planar) {       // Re at column u, Im at column tc_cols / 2 + u
                const size_t o = row + (size_t)(u0 + ul), oi = o + d.tc_cols / 2;
                tb[o] = __low2bfloat16(h);
                tb[oi] = __high2bfloat16(h);
                tb[o + lo] = __low2bfloat16(l);
                tb[oi + lo] = __high2bfloat16(l);
            } else {
                const size_t o = row + 2 * (size_t)(u0 + ul);
                *reinterpret_cast<__nv_bfloat162 *>(tb + o) = h;
                *reinterpret_cast<__nv_bfloat162 *>(tb + o + lo) = l;
            }
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

// Shared memory of rt_block<UB>: twiddles, two fine grids per bin, the sources.
inline size_t smem_bytes(int fine, int ub, int n_f) {
    return (size_t)(fine + 2 * ub * fine + ub * n_f) * sizeof(float2) + (size_t)ub * n_f * sizeof(float);
}

}  // namespace rt
