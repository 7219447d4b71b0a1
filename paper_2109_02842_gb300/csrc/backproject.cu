// Back-projection, step (8b) / (19b) of the paper, with the coherent sum over
// every channel (all sections) and the k_z tile of one block:
//
//   G_u(x,y) = sum_c  h e^{j kappa_c,u a_c(x,y)}  sum_{t<w} phi(a_c - l_{i0+t}) b_c[i0+t][u]
//
// a_c = rho (monostatic) or rho_T + rho_R (multistatic), phi the ES kernel on
// the table grid l_i = l0 + i h (setup.cu explains the factorisation).
//
// Block = 16 x 16 pixels x `UT` consecutive k_z bins; thread = one pixel with
// UT complex accumulators in registers. Channels are processed in chunks of
// CC. For each chunk the block
//  1. forms, in FP64, the range a_c* of the tile centre for every channel and
//     the first table row i_lo of the R-row window that covers the tile;
//  2. stages b_c[i_lo .. i_lo+R)[u0 .. u0+UT) in shared memory, multiplied by
//     E_c,u = h e^{j kappa_c,u a_c*} -- the only place the large phase
//     kappa a (up to ~2e3 rad) is needed, so it is formed and range-reduced
//     in FP64 once per (block, channel, bin);
//  3. per pixel forms the small offset delta = a_c - a_c* in FP32 without
//     cancellation (difference of squares against the tile centre), the tap
//     weights once, and then for each bin one w-tap interpolation, the
//     residual carrier e^{j kappa_c,u delta} (|phase| < ~60 rad, FP32) and a
//     complex multiply-accumulate.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TX = 16, TY = 16;
constexpr int CC = 16;             // channels per staged chunk

struct ChanGeo {
    float dxt, dyt, rt;            // tile centre minus Tx position, its distance
    float dxr, dyr, rr;            // same for Rx (multistatic)
    float off;                     // a_c* - l_{i_lo} (m)
    int ilo;
};

template <int UT>
__device__ __forceinline__ float2 load_tab(const void *tab, size_t idx, int bf16) {
    if (bf16) {
        const __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(tab)[idx];
        return __bfloat1622float2(v);
    }
    return reinterpret_cast<const float2 *>(tab)[idx];
}

template <int UT, int W>
__global__ void __launch_bounds__(TX * TY)
k_backproject(BpDesc p, const void *__restrict__ table, const double *__restrict__ ch_xy,
              const double *__restrict__ kc, const float *__restrict__ kc_f,
              float2 *__restrict__ G) {
    constexpr int US = UT + 1;                         // padded row stride (float2)
    extern __shared__ float2 smem[];
    float2 *slab = smem;                               // [CC][R][US]
    float2 *Es = slab + CC * p.R * US;                 // [CC][UT]
    ChanGeo *geo = reinterpret_cast<ChanGeo *>(Es + CC * UT);
    double *ac = reinterpret_cast<double *>(geo + CC);

    const int lx = threadIdx.x % TX;
    const int ly = threadIdx.x / TX;
    const int ix_lo = blockIdx.x * TX;
    const int iy_lo = blockIdx.y * TY;
    const int u0 = blockIdx.z * UT;
    const int ix = ix_lo + lx;
    const int iy = iy_lo + ly;
    // tile centre (continuous) and this pixel's offset from it
    const double xc = p.x0 + (ix_lo + 0.5 * (TX - 1)) * p.dx;
    const double yc = p.y0 + (iy_lo + 0.5 * (TY - 1)) * p.dy;
    const float ddx = (float)((lx - 0.5 * (TX - 1)) * p.dx);
    const float ddy = (float)((ly - 0.5 * (TY - 1)) * p.dy);
    const double halfrows = 0.5 * (p.R - 1);

    float kcu[UT];
    float2 acc[UT];
#pragma unroll
    for (int u = 0; u < UT; ++u) {
        kcu[u] = (u0 + u < p.n_pad) ? kc_f[u0 + u] : 0.0f;
        acc[u] = make_float2(0.f, 0.f);
    }

    for (int c0 = 0; c0 < p.n_chan; c0 += CC) {
        const int ncc = min(CC, p.n_chan - c0);
        __syncthreads();
        if (threadIdx.x < ncc) {
            const int c = c0 + threadIdx.x;
            const double dxt = xc - ch_xy[4 * c + 0], dyt = yc - ch_xy[4 * c + 1];
            const double rt = sqrt(dxt * dxt + dyt * dyt);
            double a = rt;
            ChanGeo g;
            g.dxt = (float)dxt; g.dyt = (float)dyt; g.rt = (float)rt;
            g.dxr = g.dyr = g.rr = 0.f;
            if (p.mode == 1) {
                const double dxr = xc - ch_xy[4 * c + 2], dyr = yc - ch_xy[4 * c + 3];
                const double rr = sqrt(dxr * dxr + dyr * dyr);
                a += rr;
                g.dxr = (float)dxr; g.dyr = (float)dyr; g.rr = (float)rr;
            }
            int ilo = (int)floor((a - p.l0) / p.h - halfrows);
            ilo = max(0, min(ilo, p.L - p.R));
            g.ilo = ilo;
            g.off = (float)(a - (p.l0 + ilo * p.h));
            geo[threadIdx.x] = g;
            ac[threadIdx.x] = a;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < ncc * UT; idx += blockDim.x) {
            const int cl = idx / UT;
            const int u = idx - cl * UT;
            float2 e = make_float2(0.f, 0.f);
            if (u0 + u < p.n_pad) {
                const double ph = kc[u0 + u] * ac[cl];
                const double red = ph - PL_TWO_PI * rint(ph * (1.0 / PL_TWO_PI));
                float s, co;
                sincosf((float)red, &s, &co);
                e = make_float2((float)p.h * co, (float)p.h * s);
            }
            Es[idx] = e;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < ncc * p.R * UT; idx += blockDim.x) {
            const int cl = idx / (p.R * UT);
            const int rem = idx - cl * p.R * UT;
            const int r = rem / UT;
            const int u = rem - r * UT;
            float2 v = make_float2(0.f, 0.f);
            if (u0 + u < p.n_pad) {
                const size_t ti = ((size_t)(c0 + cl) * p.L + geo[cl].ilo + r) * p.n_pad + u0 + u;
                v = cmul(load_tab<UT>(table, ti, p.bf16), Es[cl * UT + u]);
            }
            slab[(cl * p.R + r) * US + u] = v;
        }
        __syncthreads();

        for (int cl = 0; cl < ncc; ++cl) {
            const ChanGeo g = geo[cl];
            // delta = a - a* from rho^2 - rho*^2 = d(2D + d), no cancellation
            float ex = g.dxt + ddx, ey = g.dyt + ddy;
            float num = ddx * (2.0f * g.dxt + ddx) + ddy * (2.0f * g.dyt + ddy);
            float delta = num / (sqrtf(ex * ex + ey * ey) + g.rt);
            if (p.mode == 1) {
                ex = g.dxr + ddx; ey = g.dyr + ddy;
                num = ddx * (2.0f * g.dxr + ddx) + ddy * (2.0f * g.dyr + ddy);
                delta += num / (sqrtf(ex * ex + ey * ey) + g.rr);
            }
            const float pos = (delta + g.off) * p.inv_h;
            int i0 = (int)ceilf(pos - 0.5f * W);
            i0 = max(0, min(i0, p.R - W));
            float wt[W];
#pragma unroll
            for (int t = 0; t < W; ++t) wt[t] = es_kernel(pos - (float)(i0 + t), p.two_over_w, p.beta);
            const float2 *row = slab + (cl * p.R + i0) * US;
#pragma unroll
            for (int u = 0; u < UT; ++u) {
                float2 v = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < W; ++t) {
                    const float2 bv = row[t * US + u];
                    v.x = fmaf(wt[t], bv.x, v.x);
                    v.y = fmaf(wt[t], bv.y, v.y);
                }
                float s, co;
                __sincosf(kcu[u] * delta, &s, &co);
                acc[u].x = fmaf(v.x, co, fmaf(-v.y, s, acc[u].x));
                acc[u].y = fmaf(v.x, s, fmaf(v.y, co, acc[u].y));
            }
        }
    }

    if (ix < p.nx && iy < p.ny) {
        const size_t plane = (size_t)p.nx * p.ny;
        const size_t pix = (size_t)iy * p.nx + ix;
#pragma unroll
        for (int u = 0; u < UT; ++u)
            if (u0 + u < p.n_pad) G[(u0 + u) * plane + pix] = acc[u];
    }
}

template <int UT, int W>
cudaError_t launch_t(const BpDesc &p, const void *table, const double *ch_xy, const double *kc,
                     const float *kc_f, float2 *G, cudaStream_t st) {
    const size_t smem = (size_t)CC * p.R * (UT + 1) * sizeof(float2) +
                        (size_t)CC * UT * sizeof(float2) + CC * sizeof(ChanGeo) +
                        CC * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_backproject<UT, W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.n_pad + UT - 1) / UT);
    k_backproject<UT, W><<<grid, TX * TY, smem, st>>>(p, table, ch_xy, kc, kc_f, G);
    return cudaGetLastError();
}

template <int UT>
cudaError_t launch_w(const BpDesc &p, const void *table, const double *ch_xy, const double *kc,
                     const float *kc_f, float2 *G, cudaStream_t st) {
    switch (p.w) {
        case 4: return launch_t<UT, 4>(p, table, ch_xy, kc, kc_f, G, st);
        case 6: return launch_t<UT, 6>(p, table, ch_xy, kc, kc_f, G, st);
        case 8: return launch_t<UT, 8>(p, table, ch_xy, kc, kc_f, G, st);
        case 10: return launch_t<UT, 10>(p, table, ch_xy, kc, kc_f, G, st);
        case 12: return launch_t<UT, 12>(p, table, ch_xy, kc, kc_f, G, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int backproject_tile_x() { return TX; }
int backproject_tile_y() { return TY; }

cudaError_t launch_backproject(const BpDesc &p, const void *table, const double *ch_xy,
                               const double *kc, const float *kc_f, float2 *G, cudaStream_t st) {
    if (p.tile_u == 8) return launch_w<8>(p, table, ch_xy, kc, kc_f, G, st);
    return launch_w<16>(p, table, ch_xy, kc, kc_f, G, st);
}
