// Back-projection tile body shared by the per-scan kernel (backproject.cu)
// and the batched persistent kernel (batch.cu). See backproject.cu.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bp {


constexpr int TX = 16, TY = 16;
constexpr float kTwoPiHi = 6.28318548202514648f;          // float(2 pi)
constexpr float kTwoPiLo = -1.7484556e-7f;                // 2 pi - float(2 pi)
constexpr float kInvTwoPi = 0.159154943091895336f;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// kappa * a mod 2 pi with kappa = kh + kl, a = ah + al (float pairs)
__device__ __forceinline__ float phase_ff(float kh, float kl, float ah, float al) {
    const float p = kh * ah;
    float e = fmaf(kh, ah, -p);
    e = fmaf(kh, al, e);
    e = fmaf(kl, ah, e);
    const float n = rintf(p * kInvTwoPi);
    float r = fmaf(-n, kTwoPiHi, p);
    r = fmaf(-n, kTwoPiLo, r);
    return r + e;
}

template <int UT, int W, int CC>
struct BpSmem {
    static constexpr int NP = UT / 2;
    static constexpr int RS = NP + 1;                   // padded row stride (float4)
    static size_t bytes(int R, int n_chan, int bf16) {
        size_t s = 2 * (size_t)CC * R * RS * sizeof(float4);       // slab, 2 buffers
        if (bf16) s += 2 * (size_t)CC * R * NP * sizeof(uint2);    // raw BF16 staging
        s += 2 * (size_t)CC * sizeof(TileGeo);                      // geometry, 2 buffers
        s += (size_t)CC * NP * sizeof(float4);                     // (kc, kc, phi, phi)
        s += (size_t)n_chan * sizeof(int);                          // i_lo of every channel
        return s;
    }
};

// One block's work: tile (bx, by) of a gx-wide tile grid, k_z tile bz.
// p holds the problem (it may live in shared memory), ct the tap polynomials
// (a kernel parameter, so the coefficients are constant-bank operands).
template <int UT, int W, int CC, int PX>
__device__ __forceinline__ void bp_tile(const BpDesc &p, const CoefTable &ct,
                                        const void *__restrict__ table,
                                        const TileGeo *__restrict__ tgeo,
                                        const float2 *__restrict__ kc_hl, float2 *__restrict__ G,
                                        int bx, int by, int bz, int gx, float4 *smem4) {
    using SM = BpSmem<UT, W, CC>;
    constexpr int NP = SM::NP;
    constexpr int RS = SM::RS;
    constexpr int ND = W + 2;                           // polynomial coefficients per tap
    constexpr int WT = W + PX - 1;                      // taps loaded per bin pair
    constexpr int TXP = TX * PX;                        // pixels per block along x
    float4 *slab = smem4;                                       // [2][CC][R][RS]
    uint2 *raw = reinterpret_cast<uint2 *>(slab + 2 * CC * p.R * RS);   // [2][CC][R][NP]
    TileGeo *geo = reinterpret_cast<TileGeo *>(p.bf16 ? (void *)(raw + 2 * CC * p.R * NP)
                                                        : (void *)raw);  // [2][CC]
    float4 *kphi = reinterpret_cast<float4 *>(geo + 2 * CC);          // [CC][NP]
    int *ilo_s = reinterpret_cast<int *>(kphi + CC * NP);             // [n_chan]

    const int lx = threadIdx.x % TX;
    const int ly = threadIdx.x / TX;
    const int tile = by * gx + bx;
    const int u0 = bz * UT;
    const int ix = bx * TXP + PX * lx;
    const int iy = by * TY + ly;
    const int np2 = (p.n_pad + 1) / 2;
    const int pair0 = u0 / 2;
    // pixel offsets from the tile centre, formed in FP32 only: under register
    // pressure the compiler may recompute them inside the channel loop, and a
    // double expression there would run on the (slow) FP64 pipe
    float ddx[PX];
#pragma unroll
    for (int k = 0; k < PX; ++k) ddx[k] = ((float)(PX * lx + k) - 0.5f * (TXP - 1)) * p.dxf;
    const float ddy = ((float)ly - 0.5f * (TY - 1)) * p.dyf;
    const TileGeo *tg = tgeo + (size_t)tile * p.n_chan;
    const size_t row_pairs = (size_t)np2;

    for (int c = threadIdx.x; c < p.n_chan; c += blockDim.x) ilo_s[c] = tg[c].ilo;
    __syncthreads();

    // issue the asynchronous copies of chunk `ck` into buffer `buf`
    auto issue = [&](int ck, int buf) {
        const int c0 = ck * CC;
        const int ncc = min(CC, p.n_chan - c0);
        const int per_c = p.R * NP;
        for (int idx = threadIdx.x; idx < ncc * per_c; idx += blockDim.x) {
            const int cl = idx / per_c;
            const int rem = idx - cl * per_c;
            const int r = rem / NP;
            const int q = rem - r * NP;
            const int pair = min(pair0 + q, np2 - 1);   // bins past N_p are masked by kc = 0
            const size_t ti = ((size_t)(c0 + cl) * p.L + ilo_s[c0 + cl] + r) * row_pairs + pair;
            if (p.bf16)
                cp_async8(raw + ((buf * CC + cl) * p.R + r) * NP + q,
                          reinterpret_cast<const uint2 *>(table) + ti);
            else
                cp_async16(slab + ((buf * CC + cl) * p.R + r) * RS + q,
                           reinterpret_cast<const float4 *>(table) + ti);
        }
        constexpr int G4 = sizeof(TileGeo) / 16;
        for (int idx = threadIdx.x; idx < ncc * G4; idx += blockDim.x)
            cp_async16(reinterpret_cast<float4 *>(geo + buf * CC) + idx,
                       reinterpret_cast<const float4 *>(tg + c0) + idx);
        cp_commit();
    };

    float2 aRe[PX][NP], aIm[PX][NP];
#pragma unroll
    for (int k = 0; k < PX; ++k)
#pragma unroll
        for (int q = 0; q < NP; ++q) aRe[k][q] = aIm[k][q] = f2(0.f, 0.f);

    const int n_chunks = (p.n_chan + CC - 1) / CC;
    issue(0, 0);
    for (int ck = 0; ck < n_chunks; ++ck) {
        const int buf = ck & 1;
        const int ncc = min(CC, p.n_chan - ck * CC);
        if (ck + 1 < n_chunks) {
            issue(ck + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        // per channel: the band centre kappa_T shared by the block's bins
        // (the table is built about it) and its reference phase at a*
        const float2 kT = kc_hl[u0];
        for (int cl = threadIdx.x; cl < ncc; cl += blockDim.x) {
            const TileGeo &g = geo[buf * CC + cl];
            kphi[cl * NP] = make_float4(kT.x, phase_ff(kT.x, kT.y, g.a_hi, g.a_lo), 0.f, 0.f);
        }
        if (p.bf16) {
            for (int idx = threadIdx.x; idx < ncc * p.R * NP; idx += blockDim.x) {
                const int cl = idx / (p.R * NP);
                const int rem = idx - cl * p.R * NP;
                const int r = rem / NP;
                const int q = rem - r * NP;
                const uint2 v = raw[((buf * CC + cl) * p.R + r) * NP + q];
                const float2 re = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
                const float2 im = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
                slab[((buf * CC + cl) * p.R + r) * RS + q] = make_float4(re.x, re.y, im.x, im.y);
            }
        }
        __syncthreads();

        const float4 *slab_b = slab + buf * CC * p.R * RS;
        for (int cl = 0; cl < ncc; ++cl) {
            const TileGeo g = geo[buf * CC + cl];
            float delta[PX], pos[PX];
            int i0[PX];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                // delta = a - a* from rho^2 - rho*^2 = d (2 D + d): no cancellation
                float ex = g.dxt + ddx[k], ey = g.dyt + ddy;
                float num = fmaf(ddx[k], 2.0f * g.dxt + ddx[k], ddy * (2.0f * g.dyt + ddy));
                float r2 = fmaf(ex, ex, ey * ey);
                float dl = num * __frcp_rn(fmaf(r2, rsqrtf(r2), g.rt));
                if (p.mode == 1) {
                    ex = g.dxr + ddx[k]; ey = g.dyr + ddy;
                    num = fmaf(ddx[k], 2.0f * g.dxr + ddx[k], ddy * (2.0f * g.dyr + ddy));
                    r2 = fmaf(ex, ex, ey * ey);
                    dl += num * __frcp_rn(fmaf(r2, rsqrtf(r2), g.rr));
                }
                delta[k] = dl;
                pos[k] = (dl + g.off) * p.inv_h;
                i0[k] = (int)ceilf(pos[k] - 0.5f * W);
            }
            int base = i0[0];
#pragma unroll
            for (int k = 1; k < PX; ++k) base = min(base, i0[k]);
            base = max(0, min(base, p.R - WT));
            // tap weights: per-tap polynomial in s = 2 (pos - i0 - (w/2 - 1)) - 1,
            // placed at slot (i0 - base) + t of the WT loaded taps
            float2 wt[PX][WT];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                const int o = min(max(i0[k] - base, 0), PX - 1);
                const float s = fmaf(2.0f, pos[k] - (float)(base + o), -(float)(W - 1));
                float w[W];
#pragma unroll
                for (int t = 0; t < W; ++t) {
                    float acc = ct.c[t][ND - 1];
#pragma unroll
                    for (int d = ND - 2; d >= 0; --d) acc = fmaf(acc, s, ct.c[t][d]);
                    w[t] = acc;
                }
#pragma unroll
                for (int t = 0; t < WT; ++t) {
                    float v = 0.f;
#pragma unroll
                    for (int oo = 0; oo < PX; ++oo)
                        if (t - oo >= 0 && t - oo < W && o == oo) v = w[t - oo];
                    wt[k][t] = f2(v, v);
                }
            }
            const float4 *row = slab_b + (cl * p.R + base) * RS;
            // the carrier e^{j kappa_T a} of each pixel: one sin/cos pair per
            // (pixel, channel), shared by all the block's bins
            const float4 kk = kphi[cl * NP];
            float2 C[PX], S[PX], nS[PX];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                float sv, cv;
                __sincosf(fmaf(kk.x, delta[k], kk.y), &sv, &cv);
                C[k] = f2(cv, cv);
                S[k] = f2(sv, sv);
                nS[k] = f2(-sv, -sv);
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 X[PX], Y[PX];
#pragma unroll
                for (int k = 0; k < PX; ++k) X[k] = Y[k] = f2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < WT; ++t) {
                    const float4 b = row[t * RS + q];
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        X[k] = __ffma2_rn(wt[k][t], f2(b.x, b.y), X[k]);
                        Y[k] = __ffma2_rn(wt[k][t], f2(b.z, b.w), Y[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    aRe[k][q] = __ffma2_rn(Y[k], nS[k], __ffma2_rn(X[k], C[k], aRe[k][q]));
                    aIm[k][q] = __ffma2_rn(Y[k], C[k], __ffma2_rn(X[k], S[k], aIm[k][q]));
                }
            }
        }
        __syncthreads();
    }

    if (iy < p.ny) {
        const size_t plane = (size_t)p.nx * p.ny;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            if (ix + k >= p.nx) continue;
            const size_t pix = (size_t)iy * p.nx + ix + k;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int u = u0 + 2 * q;
                if (u < p.n_pad) G[u * plane + pix] = f2(aRe[k][q].x, aIm[k][q].x);
                if (u + 1 < p.n_pad) G[(u + 1) * plane + pix] = f2(aRe[k][q].y, aIm[k][q].y);
            }
        }
    }
}


}  // namespace bp
