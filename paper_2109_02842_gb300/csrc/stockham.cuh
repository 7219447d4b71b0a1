// Mixed-radix (2, 3, 4, 5, 8) Stockham autosort FFT stage on a batch of columns
// in shared memory. Element (column col, index n) lives at col*cs + n*ns.
// One stage of radix R with Ns = product of the previous radices:
//   v_r = src[j + r N/R] * W_N^{(j mod Ns) r N/(Ns R)},  r < R
//   dst[(j/Ns) Ns R + (j mod Ns) + q Ns] = sum_r v_r W_R^{r q},  q < R
// for j < N/R. After all stages the data are in natural order. tw holds
// exp(-2 pi i k / N), k < N; sgn = +1 conjugates it (inverse transform).
// The small DFTs W_R use the exact values of the R-th roots of unity,
// and the twiddle index (j mod Ns) r N/(Ns R) is below N (no reduction).
#pragma once

#include "common.cuh"

namespace stockham_detail {

// v <- DFT_R(v) with exponent sign -1 (sgn < 0) or +1 (sgn > 0)
template <int R>
__device__ __forceinline__ void small_dft(float2 (&v)[8], int sgn);

template <>
__device__ __forceinline__ void small_dft<2>(float2 (&v)[8], int) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void small_dft<4>(float2 (&v)[8], int sgn) {
    // W_4 = -i (forward) / +i (inverse)
    const float2 s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
    const float2 s1 = cadd(v[1], v[3]), d1 = csub(v[1], v[3]);
    // d1 * W_4: forward (x, y) -> (y, -x); inverse (x, y) -> (-y, x)
    const float2 r1 = sgn < 0 ? make_float2(d1.y, -d1.x) : make_float2(-d1.y, d1.x);
    v[0] = cadd(s0, s1);
    v[2] = csub(s0, s1);
    v[1] = cadd(d0, r1);
    v[3] = csub(d0, r1);
}

template <>
__device__ __forceinline__ void small_dft<3>(float2 (&v)[8], int sgn) {
    // W_3 = -1/2 -+ i sqrt(3)/2
    const float c = -0.5f, s = (sgn < 0 ? -1.f : 1.f) * 0.866025403784438647f;
    const float2 t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(v[0].x + c * t.x, v[0].y + c * t.y);
    const float2 r = make_float2(-s * d.y, s * d.x);    // i s d
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

template <>
__device__ __forceinline__ void small_dft<5>(float2 (&v)[8], int sgn) {
    // cos / sin of 2 pi / 5 and 4 pi / 5
    const float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;
    const float sg = sgn < 0 ? -1.f : 1.f;
    const float s1 = sg * 0.951056516295153572f, s2 = sg * 0.587785252292473129f;
    const float2 t1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
    const float2 t2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
    const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    // b1 = i (s1 d1 + s2 d2), b2 = i (s2 d1 - s1 d2)
    const float2 e1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
    const float2 e2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
    const float2 b1 = make_float2(-e1.y, e1.x), b2 = make_float2(-e2.y, e2.x);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <>
__device__ __forceinline__ void small_dft<8>(float2 (&v)[8], int sgn) {
    // two DFT_4 on the even and odd entries, combined with W_8^q; W_8 =
    // (1 -+ i) / sqrt 2, W_8^2 = -+ i, W_8^3 = (-1 -+ i) / sqrt 2
    float2 e[8] = {v[0], v[2], v[4], v[6]}, o[8] = {v[1], v[3], v[5], v[7]};
    small_dft<4>(e, sgn);
    small_dft<4>(o, sgn);
    const float h = 0.707106781186547524f;
    const float sg = sgn < 0 ? -1.f : 1.f;
    float2 t[4];
    t[0] = o[0];
    t[1] = make_float2(h * (o[1].x - sg * o[1].y), h * (o[1].y + sg * o[1].x));
    t[2] = make_float2(-sg * o[2].y, sg * o[2].x);
    t[3] = make_float2(-h * (o[3].x + sg * o[3].y), h * (sg * o[3].x - o[3].y));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = cadd(e[q], t[q]);
        v[q + 4] = csub(e[q], t[q]);
    }
}

}  // namespace stockham_detail

// NCOL columns (compile time). COL_FAST: consecutive threads take consecutive
// columns (use when columns are the contiguous axis); otherwise consecutive j.
template <int R, bool COL_FAST, int NCOL>
__device__ __forceinline__ void stockham_stage(const float2 *src, float2 *dst, const float2 *tw,
                                               int N, int Ns, int sgn, int cs, int ns) {
    const int nr = N / R;
    const int items = nr * NCOL;
    const int tw_step = N / (Ns * R);
    // j / Ns as floor((j + 1/2) / Ns) in float: exact for j < 2^20 (the
    // fraction stays at least 1/(2 Ns) away from an integer), and three
    // instructions instead of an integer division
    const float inv_ns = 1.0f / (float)Ns;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int j, col;
        if (COL_FAST) { j = it / NCOL; col = it - j * NCOL; }
        else { col = it / nr; j = it - col * nr; }
        const int jh = __float2int_rz(((float)j + 0.5f) * inv_ns);
        const int k = j - jh * Ns;
        const float2 *s = src + col * cs;
        float2 v[8];
        v[0] = s[j * ns];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[k * r * tw_step];
            if (sgn > 0) w.y = -w.y;
            v[r] = cmul(s[(j + r * nr) * ns], w);
        }
        stockham_detail::small_dft<R>(v, sgn);
        float2 *d = dst + col * cs;
        const int base = jh * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) d[(base + q * Ns) * ns] = v[q];
    }
}

// Runs every stage of `plan` on NCOL columns; returns the buffer holding the
// result. Ends with a __syncthreads().
template <bool COL_FAST, int NCOL>
__device__ __forceinline__ float2 *stockham_run(float2 *buf0, float2 *buf1, const float2 *tw,
                                                const FftPlan &plan, int sgn, int cs, int ns) {
    float2 *src = buf0, *dst = buf1;
    int Ns = 1;
    const int N = plan.n;
    for (int s = 0; s < plan.n_stages; ++s) {
        const int R = plan.radix[s];
        if (R == 8) stockham_stage<8, COL_FAST, NCOL>(src, dst, tw, N, Ns, sgn, cs, ns);
        else if (R == 4) stockham_stage<4, COL_FAST, NCOL>(src, dst, tw, N, Ns, sgn, cs, ns);
        else if (R == 2) stockham_stage<2, COL_FAST, NCOL>(src, dst, tw, N, Ns, sgn, cs, ns);
        else if (R == 3) stockham_stage<3, COL_FAST, NCOL>(src, dst, tw, N, Ns, sgn, cs, ns);
        else stockham_stage<5, COL_FAST, NCOL>(src, dst, tw, N, Ns, sgn, cs, ns);
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}

// The same stage on column pairs: NCOL (even) columns stored at n * NCOL +
// col, one thread item = two adjacent columns as a float4, so the index
// arithmetic, the twiddle loads and the shared-memory accesses are shared by
// both columns.
template <int R, int NCOL>
__device__ __forceinline__ void stockham_stage_pairs(const float2 *src, float2 *dst,
                                                     const float2 *tw, int N, int Ns, int sgn) {
    constexpr int NP = NCOL / 2;
    const int nr = N / R;
    const int items = nr * NP;
    const int tw_step = N / (Ns * R);
    const float inv_ns = 1.0f / (float)Ns;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / NP;
        const int cp = it - j * NP;
        const int jh = __float2int_rz(((float)j + 0.5f) * inv_ns);
        const int k = j - jh * Ns;
        float2 a[8], b[8];
        float4 x = s4[j * NP + cp];
        a[0] = make_float2(x.x, x.y);
        b[0] = make_float2(x.z, x.w);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[k * r * tw_step];
            if (sgn > 0) w.y = -w.y;
            x = s4[(j + r * nr) * NP + cp];
            a[r] = cmul(make_float2(x.x, x.y), w);
            b[r] = cmul(make_float2(x.z, x.w), w);
        }
        stockham_detail::small_dft<R>(a, sgn);
        stockham_detail::small_dft<R>(b, sgn);
        const int base = jh * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q)
            d4[(base + q * Ns) * NP + cp] = make_float4(a[q].x, a[q].y, b[q].x, b[q].y);
    }
}

// Every stage of `plan` on NCOL columns (column pairs); returns the buffer
// holding the result. Both buffers 16-byte aligned. Ends with a
// __syncthreads().
template <int NCOL>
__device__ __forceinline__ float2 *stockham_run_pairs(float2 *buf0, float2 *buf1, const float2 *tw,
                                                      const FftPlan &plan, int sgn) {
    float2 *src = buf0, *dst = buf1;
    int Ns = 1;
    const int N = plan.n;
    for (int s = 0; s < plan.n_stages; ++s) {
        const int R = plan.radix[s];
        if (R == 8) stockham_stage_pairs<8, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 4) stockham_stage_pairs<4, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 2) stockham_stage_pairs<2, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 3) stockham_stage_pairs<3, NCOL>(src, dst, tw, N, Ns, sgn);
        else stockham_stage_pairs<5, NCOL>(src, dst, tw, N, Ns, sgn);
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}

// First stage (N_s = 1, so every twiddle is 1) on column pairs when the
// input is the sum of two panels: reads a + b, and after a barrier writes the
// stage's output over b. Needs (N / R) * NCOL / 2 <= blockDim.x (one item per
// thread), so that every read precedes every write.
template <int R, int NCOL>
__device__ __forceinline__ void stockham_first_stage_sum_pairs(const float2 *a_buf, float2 *b_buf,
                                                               int N, int sgn) {
    constexpr int NP = NCOL / 2;
    const int nr = N / R;
    const int it = threadIdx.x;
    const bool act = it < nr * NP;
    const int j = it / NP;
    const int cp = it - j * NP;
    float2 a[8], b[8];
    if (act) {
        const float4 *s4 = reinterpret_cast<const float4 *>(a_buf);
        const float4 *t4 = reinterpret_cast<const float4 *>(b_buf);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 x = s4[(j + r * nr) * NP + cp], y = t4[(j + r * nr) * NP + cp];
            a[r] = make_float2(x.x + y.x, x.y + y.y);
            b[r] = make_float2(x.z + y.z, x.w + y.w);
        }
        stockham_detail::small_dft<R>(a, sgn);
        stockham_detail::small_dft<R>(b, sgn);
    }
    __syncthreads();
    if (act) {
        float4 *d4 = reinterpret_cast<float4 *>(b_buf);
#pragma unroll
        for (int q = 0; q < R; ++q)
            d4[(j * R + q) * NP + cp] = make_float4(a[q].x, a[q].y, b[q].x, b[q].y);
    }
}

// Last stage (N_s = N / R: every output row is j + q N_s, twiddle step 1) on
// column pairs, handing each output row to emit(row, column pair, first
// column, second column) instead of writing shared memory.
template <int R, int NCOL, class Emit>
__device__ __forceinline__ void stockham_last_stage_pairs(const float2 *src, const float2 *tw,
                                                          int N, int sgn, const Emit &emit) {
    constexpr int NP = NCOL / 2;
    const int nr = N / R;
    const int items = nr * NP;
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int j = it / NP;
        const int cp = it - j * NP;
        float2 a[8], b[8];
        float4 x = s4[j * NP + cp];
        a[0] = make_float2(x.x, x.y);
        b[0] = make_float2(x.z, x.w);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[j * r];
            if (sgn > 0) w.y = -w.y;
            x = s4[(j + r * nr) * NP + cp];
            a[r] = cmul(make_float2(x.x, x.y), w);
            b[r] = cmul(make_float2(x.z, x.w), w);
        }
        stockham_detail::small_dft<R>(a, sgn);
        stockham_detail::small_dft<R>(b, sgn);
#pragma unroll
        for (int q = 0; q < R; ++q) emit(j + q * nr, cp, a[q], b[q]);
    }
}

// Every stage of `plan` on NCOL columns (column pairs), the input the sum of
// buf0 and buf1 when `sum2` (else buf0 alone), the last stage's rows handed
// to `emit`. Both buffers 16-byte aligned.
template <int NCOL, class Emit>
__device__ __forceinline__ void stockham_run_pairs_emit(float2 *buf0, float2 *buf1, const float2 *tw,
                                                        const FftPlan &plan, int sgn, bool sum2,
                                                        const Emit &emit) {
    const int N = plan.n;
    const int S = plan.n_stages;
    float2 *src = buf0, *dst = buf1;
    int Ns = 1;
    int s = 0;
    if (sum2) {
        const int R = plan.radix[0];
        if (S >= 2 && (N / R) * (NCOL / 2) <= (int)blockDim.x) {
            if (R == 8) stockham_first_stage_sum_pairs<8, NCOL>(buf0, buf1, N, sgn);
            else if (R == 4) stockham_first_stage_sum_pairs<4, NCOL>(buf0, buf1, N, sgn);
            else if (R == 2) stockham_first_stage_sum_pairs<2, NCOL>(buf0, buf1, N, sgn);
            else if (R == 3) stockham_first_stage_sum_pairs<3, NCOL>(buf0, buf1, N, sgn);
            else stockham_first_stage_sum_pairs<5, NCOL>(buf0, buf1, N, sgn);
            __syncthreads();
            src = buf1;
            dst = buf0;
            Ns = R;
            s = 1;
        } else {     // a separate pass: buf0 += buf1
            for (int idx = threadIdx.x; idx < N * NCOL / 2; idx += blockDim.x) {
                float4 *p = reinterpret_cast<float4 *>(buf0) + idx;
                const float4 c = reinterpret_cast<const float4 *>(buf1)[idx];
                *p = make_float4(p->x + c.x, p->y + c.y, p->z + c.z, p->w + c.w);
            }
            __syncthreads();
        }
    }
    for (; s < S - 1; ++s) {
        const int R = plan.radix[s];
        if (R == 8) stockham_stage_pairs<8, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 4) stockham_stage_pairs<4, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 2) stockham_stage_pairs<2, NCOL>(src, dst, tw, N, Ns, sgn);
        else if (R == 3) stockham_stage_pairs<3, NCOL>(src, dst, tw, N, Ns, sgn);
        else stockham_stage_pairs<5, NCOL>(src, dst, tw, N, Ns, sgn);
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    const int R = plan.radix[S - 1];
    if (R == 8) stockham_last_stage_pairs<8, NCOL>(src, tw, N, sgn, emit);
    else if (R == 4) stockham_last_stage_pairs<4, NCOL>(src, tw, N, sgn, emit);
    else if (R == 2) stockham_last_stage_pairs<2, NCOL>(src, tw, N, sgn, emit);
    else if (R == 3) stockham_last_stage_pairs<3, NCOL>(src, tw, N, sgn, emit);
    else stockham_last_stage_pairs<5, NCOL>(src, tw, N, sgn, emit);
}
