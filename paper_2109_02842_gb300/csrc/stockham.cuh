// Mixed-radix (2, 3, 4, 5) Stockham autosort FFT stage on a batch of columns
// in shared memory. Element (column col, index n) lives at col*cs + n*ns.
// One stage of radix R with Ns = product of the previous radices:
//   v_r = src[j + r N/R] * W_N^{(j mod Ns) r N/(Ns R)},  r < R
//   dst[(j/Ns) Ns R + (j mod Ns) + q Ns] = sum_r v_r W_R^{r q},  q < R
// for j < N/R. After all stages the data are in natural order. tw holds
// exp(-2 pi i k / N), k < N; sgn = +1 conjugates it (inverse transform).
#pragma once

#include "common.cuh"

template <int R>
__device__ __forceinline__ void stockham_small_dft(float2 (&v)[5], const float2 *tw, int N,
                                                   int sgn) {
    float2 o[R];
    const int step = N / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        float2 acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[((r * q) % R) * step];
            if (sgn > 0) w.y = -w.y;
            acc = cadd(acc, cmul(v[r], w));
        }
        o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = o[q];
}

// COL_FAST: consecutive threads take consecutive columns (use when columns
// are the contiguous axis); otherwise consecutive j.
template <int R, bool COL_FAST>
__device__ __forceinline__ void stockham_stage(const float2 *src, float2 *dst, const float2 *tw,
                                               int N, int Ns, int sgn, int ncol, int cs, int ns) {
    const int nr = N / R;
    const int items = nr * ncol;
    const int tw_step = N / (Ns * R);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int j, col;
        if (COL_FAST) { j = it / ncol; col = it - j * ncol; }
        else { col = it / nr; j = it - col * nr; }
        const int k = j % Ns;
        const float2 *s = src + col * cs;
        float2 v[5];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = s[(j + r * nr) * ns];
            if (r > 0) {
                float2 w = tw[(k * r * tw_step) % N];
                if (sgn > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        stockham_small_dft<R>(v, tw, N, sgn);
        float2 *d = dst + col * cs;
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) d[(base + q * Ns) * ns] = v[q];
    }
}

// Runs every stage of `plan`; returns the buffer holding the result. Ends
// with a __syncthreads().
template <bool COL_FAST>
__device__ __forceinline__ float2 *stockham_run(float2 *buf0, float2 *buf1, const float2 *tw,
                                                const FftPlan &plan, int sgn, int ncol, int cs,
                                                int ns) {
    float2 *src = buf0, *dst = buf1;
    int Ns = 1;
    const int N = plan.n;
    for (int s = 0; s < plan.n_stages; ++s) {
        const int R = plan.radix[s];
        if (R == 4) stockham_stage<4, COL_FAST>(src, dst, tw, N, Ns, sgn, ncol, cs, ns);
        else if (R == 2) stockham_stage<2, COL_FAST>(src, dst, tw, N, Ns, sgn, ncol, cs, ns);
        else if (R == 3) stockham_stage<3, COL_FAST>(src, dst, tw, N, Ns, sgn, ncol, cs, ns);
        else stockham_stage<5, COL_FAST>(src, dst, tw, N, Ns, sgn, ncol, cs, ns);
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}
