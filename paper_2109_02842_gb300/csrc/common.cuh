// Internal helpers shared by the CUDA translation units of libpolyline.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PL_C0 299792458.0
#define PL_TWO_PI 6.283185307179586476925286766559

// ---------------------------------------------------------------------------
// complex helpers (float2 = (re, im))
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
    return make_float2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ---------------------------------------------------------------------------
// "exponential of semicircle" kernel, Barnett, Magland & af Klinteberg,
// SIAM J. Sci. Comput. 41 (2019): ES(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1))
// for |t| < w/2 (t in grid cells), else 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float es_kernel(float t, float two_over_w, float beta) {
    float z = t * two_over_w;
    float q = 1.0f - z * z;
    return q > 0.0f ? __expf(beta * (sqrtf(q) - 1.0f)) : 0.0f;
}
__device__ __forceinline__ double es_kernel_d(double t, double two_over_w, double beta) {
    double z = t * two_over_w;
    double q = 1.0 - z * z;
    return q > 0.0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
}

// Radix plan of a 5-smooth length (at most 16 stages of radix 2, 3, 4 or 5).
struct FftPlan {
    int n;
    int n_stages;
    int radix[16];
};

// Problem description shared by the range-table and back-projection kernels.
struct NufftDesc {
    int mode;          // 0 mono, 1 multi
    int n_chan, n_pad, n_f;
    int L;             // table rows
    int fine;          // type-1 fine grid length (2^a 3^b 5^c)
    int log2_fine;
    int w;             // interpolation taps
    int w1;            // type-1 spreading taps
    float beta, beta1;
    double h, l0;      // table step and origin (m)
    int tc_cols;       // tensor-core table layout: columns (2 per bin) per row
    int tc_planar;     // 1: [Re of the bins | Im of the bins] per row, 0: (re, im) pairs
    int s_bf16;        // 1: the spectrum S is stored as bfloat16 (re, im) pairs
};
