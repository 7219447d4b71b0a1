// The two comparison algorithms of Sec. III (Table II), on the GPU:
//
//  * exact-sum hybrid ("omega-K-BP", the method without the NUFFT): after the
//    z-FFT, per k_z bin u and pixel
//      G_u(x,y) = sum_c sum_m S[c][u][m] k_m e^{+j kappa_um a_c(x,y)}
//    (Eq. 7 mono, Eq. 19 multistatic, evanescent terms dropped), then the
//    inverse transform over k_z (Eq. 9);
//  * direct back-projection (BP), the time-domain matched filter of the echo
//    model (Eq. 1 / 10) with the k weight:
//      g(x,y,z) = sum_c sum_n sum_m s[c][n][m] k_m e^{+j k_m (R_T + R_R)}.
//
// Both in FP32 with float-float ranges and phases (kappa a and k R reach
// ~2e3 rad; a float-float product reduced modulo 2 pi leaves ~1e-7 rad), one
// thread per output pixel / voxel, the per-channel data read with warp-uniform
// loads (the same address for every lane: one broadcast). With an evenly
// spaced band the direct BP forms e^{j k_m R} by rotation from k_0 in steps
// of dk (one sin/cos pair per (voxel, channel, scan) instead of one per term).
#include "bp_body.cuh"
#include "common.cuh"
#include "kernels.h"

namespace {

struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_of(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, s.lo + x.lo + y.lo);
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_sqr(ff x) {
    const float p = x.hi * x.hi;
    const float e = fmaf(x.hi, x.hi, -p) + 2.0f * x.hi * x.lo;
    return quick_two_sum(p, e);
}
// sqrt of a positive float pair: one correction step of the float root
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float r = sqrtf(x.hi);
    const float p = r * r;
    const float e = fmaf(r, r, -p);
    const float d = ((x.hi - p) - e + x.lo) / (2.0f * r);
    return quick_two_sum(r, d);
}
// |(x, y) - (px, py)| as a float pair
__device__ __forceinline__ ff ff_dist2d(ff x, ff y, ff px, ff py) {
    const ff dx = ff_add(x, ff_neg(px)), dy = ff_add(y, ff_neg(py));
    return ff_sqrt(ff_add(ff_sqr(dx), ff_sqr(dy)));
}

// G[u][pixel] of the exact sum, UT bins per block.
template <int UT>
__global__ void __launch_bounds__(128)
k_exact_sum(ExactDesc e, const float2 *__restrict__ S, const float2 *__restrict__ kap,
            const float *__restrict__ wum, const float4 *__restrict__ chff, float2 *__restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int u0 = blockIdx.y * UT;
    const int np = e.nx * e.ny;
    const bool live = p < np;
    const int ix = live ? p % e.nx : 0, iy = live ? p / e.nx : 0;
    const ff px = ff_of(e.x0 + ix * e.dx), py = ff_of(e.y0 + iy * e.dy);
    float2 acc[UT];
#pragma unroll
    for (int j = 0; j < UT; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int c = 0; c < e.n_chan; ++c) {
        const float4 t = chff[2 * c], r = chff[2 * c + 1];
        // a = rho (mono: kappa = sqrt(4k^2 - k_z^2) carries the factor 2) or
        // rho_T + rho_R (multi: kappa = sqrt(k^2 - k_z^2 / 4))
        ff a = ff_dist2d(px, py, {t.x, t.y}, {t.z, t.w});
        if (e.mode == 1) a = ff_add(a, ff_dist2d(px, py, {r.x, r.y}, {r.z, r.w}));
#pragma unroll
        for (int j = 0; j < UT; ++j) {
            const int u = u0 + j;
            if (u >= e.n_pad) break;
            const float2 *Su = S + ((size_t)c * e.n_pad + u) * e.n_f;
            const float2 *ku = kap + (size_t)u * e.n_f;
            const float *wu = wum + (size_t)u * e.n_f;
            for (int m = 0; m < e.n_f; ++m) {
                const float w = wu[m];
                if (w == 0.f) continue;              // evanescent (uniform across the block)
                const float2 k = ku[m];
                const float2 s = Su[m];
                float sn, cs;
                __sincosf(bp::phase_ff(k.x, k.y, a.hi, a.lo), &sn, &cs);
                const float sr = s.x * w, si = s.y * w;
                acc[j].x = fmaf(sr, cs, fmaf(-si, sn, acc[j].x));
                acc[j].y = fmaf(sr, sn, fmaf(si, cs, acc[j].y));
            }
        }
    }
    if (live) {
#pragma unroll
        for (int j = 0; j < UT; ++j)
            if (u0 + j < e.n_pad) G[(size_t)(u0 + j) * np + p] = acc[j];
    }
}

// Direct back-projection onto the voxel grid, one voxel per thread.
template <bool UNIFORM>
__global__ void __launch_bounds__(128)
k_bp_direct(DirectDesc e, const float2 *__restrict__ s, const float4 *__restrict__ chff,
            const float2 *__restrict__ zs, const float2 *__restrict__ kff, float2 *__restrict__ img) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nv = (long long)e.nx * e.ny * e.nz;
    const bool live = v < nv;
    const int ix = live ? (int)(v % e.nx) : 0;
    const int iy = live ? (int)((v / e.nx) % e.ny) : 0;
    const int iz = live ? (int)(v / ((long long)e.nx * e.ny)) : 0;
    const ff px = ff_of(e.x0 + ix * e.dx), py = ff_of(e.y0 + iy * e.dy);
    const ff pz = ff_of(e.z0 + iz * e.dz);
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < e.n_chan; ++c) {
        const float4 t = chff[2 * c], r = chff[2 * c + 1];
        const ff dxt = ff_add(px, ff_neg({t.x, t.y})), dyt = ff_add(py, ff_neg({t.z, t.w}));
        const ff rho_t = ff_add(ff_sqr(dxt), ff_sqr(dyt));
        ff rho_r = rho_t;
        if (e.mode == 1) {
            const ff dxr = ff_add(px, ff_neg({r.x, r.y})), dyr = ff_add(py, ff_neg({r.z, r.w}));
            rho_r = ff_add(ff_sqr(dxr), ff_sqr(dyr));
        }
        const float2 *sc = s + (size_t)c * e.n_scan * e.n_f;
        for (int n = 0; n < e.n_scan; ++n) {
            const float2 zn = zs[n];
            const ff dz2 = ff_sqr(ff_add(pz, ff_neg({zn.x, zn.y})));
            ff a = ff_sqrt(ff_add(rho_t, dz2));
            a = e.mode == 0 ? ff_add(a, a) : ff_add(a, ff_sqrt(ff_add(rho_r, dz2)));
            const float2 *sn_ = sc + (size_t)n * e.n_f;
            if (UNIFORM) {
                // e^{j k_m a} = e^{j k_0 a} (e^{j dk a})^m
                float s0, c0, s1, c1;
                __sincosf(bp::phase_ff(e.k0_hi, e.k0_lo, a.hi, a.lo), &s0, &c0);
                __sincosf(bp::phase_ff(e.dk_hi, e.dk_lo, a.hi, a.lo), &s1, &c1);
                float er = c0, ei = s0;
                for (int m = 0; m < e.n_f; ++m) {
                    const float2 x = sn_[m];
                    const float k = kff[m].x;
                    const float sr = x.x * k, si = x.y * k;
                    acc.x = fmaf(sr, er, fmaf(-si, ei, acc.x));
                    acc.y = fmaf(sr, ei, fmaf(si, er, acc.y));
                    const float nr = fmaf(er, c1, -ei * s1);
                    ei = fmaf(er, s1, ei * c1);
                    er = nr;
                }
            } else {
                for (int m = 0; m < e.n_f; ++m) {
                    const float2 x = sn_[m];
                    const float2 k = kff[m];
                    float sv, cv;
                    __sincosf(bp::phase_ff(k.x, k.y, a.hi, a.lo), &sv, &cv);
                    const float sr = x.x * k.x, si = x.y * k.x;
                    acc.x = fmaf(sr, cv, fmaf(-si, sv, acc.x));
                    acc.y = fmaf(sr, sv, fmaf(si, cv, acc.y));
                }
            }
        }
    }
    if (live) img[v] = acc;
}

}  // namespace

cudaError_t launch_exact_sum(const ExactDesc &e, const float2 *S, const float2 *kap,
                             const float *wum, const float4 *chff, float2 *G, cudaStream_t st) {
    constexpr int UT = 8;
    dim3 grid((e.nx * e.ny + 127) / 128, (e.n_pad + UT - 1) / UT);
    k_exact_sum<UT><<<grid, 128, 0, st>>>(e, S, kap, wum, chff, G);
    return cudaGetLastError();
}

cudaError_t launch_bp_direct(const DirectDesc &e, const float2 *s, const float4 *chff,
                             const float2 *zs, const float2 *kff, float2 *img, cudaStream_t st) {
    const long long nv = (long long)e.nx * e.ny * e.nz;
    const unsigned blocks = (unsigned)((nv + 127) / 128);
    if (e.uniform)
        k_bp_direct<true><<<blocks, 128, 0, st>>>(e, s, chff, zs, kff, img);
    else
        k_bp_direct<false><<<blocks, 128, 0, st>>>(e, s, chff, zs, kff, img);
    return cudaGetLastError();
}
