// Transforms along the scan axis (Sec. II-A, Eq. 2) and along k_z (Eq. 9).
//
// Both act on the middle axis of a [batch][n][inner] complex64 array whose
// inner axis is contiguous: the echo s[c][n][m] (forward, zero-padded to N_p)
// and the image spectrum G[u][pixel] (inverse; the sum of the two channel
// parts' spectra, added as the first stage reads them). One block stages a
// [n][IB] column panel in shared memory (coalesced row segments), runs a
// mixed-radix (2, 3, 4, 5, 8) Stockham autosort FFT on all IB columns at once
// (column pairs), and its last stage writes the requested output rows to
// global memory (complex64 rows, or the range table's BF16 hi/lo operand). A
// launch may cover a range of columns of wider rows (row stride ld). Lengths
// with another prime factor, and inverse transforms onto voxel heights off
// the scan grid, use the tiled direct DFT kernel below with a precomputed
// phase matrix.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>


#include "common.cuh"
#include "kernels.h"
#include "stockham.cuh"

namespace {

constexpr int kFftIB = 16;        // columns per block (128-byte rows)
constexpr int kFftThreads = 256;  // threads per block

// in:  [batch][n_in][ld], columns i < I  (rows n >= n_in are zero padding)
// out: [batch][out_rows][ld], out row r = transform index (r + out_off) mod N
// (complex64, or with sp.bf16_rows set bfloat16 (re, im) pairs in the same
// layout); or, with sp.A set, the tensor-core range table's operand instead:
// A[r][re hi, re lo, im hi, im lo][batch][Kp] = split(X[r][i]) (BF16; with
// sp.hi_only only the hi planes are written)
struct SplitOut {
    __nv_bfloat16 *A;        // nullptr: plain output
    int batch, Kp;
    int hi_only;             // split output: hi planes only (BF16 spectrum)
    int bf16_rows;           // plain output as bfloat16 (re, im) pairs
};
// PAIRS (I even): every access moves two adjacent columns (16-byte copies,
// float4 shared-memory accesses, column pairs through the FFT stages).
// SPLIT: the output is the range table's operand (sp.A), else `out`.
template <bool PAIRS, bool SPLIT>
__global__ void __launch_bounds__(kFftThreads)
k_fft_strided(const float2 *__restrict__ in, const float2 *__restrict__ in2, float2 *__restrict__ out,
              int n_in, int I, int ld, FftPlan plan, const float2 *__restrict__ tw_g, int sgn,
              float scale, int out_rows, int out_off, SplitOut sp) {
    extern __shared__ __align__(16) float2 smem[];
    const int N = plan.n;
    float2 *buf0 = smem;
    float2 *buf1 = smem + N * kFftIB;
    float2 *tw = smem + 2 * N * kFftIB;
    const int i0 = blockIdx.x * kFftIB;
    const size_t b = blockIdx.y;
    constexpr int CW = PAIRS ? 2 : 1;          // columns per access
    constexpr int NG = kFftIB / CW;            // accesses per row

    // the whole panel in flight at once: asynchronous copies, zeros for the
    // padding rows and the columns past I. Each thread keeps one column group
    // (CW columns) and walks the rows RPS apart with running pointers.
    constexpr int RPS = kFftThreads / NG;      // rows per sweep of the block
    const int col = (threadIdx.x % NG) * CW;
    const int n_first = threadIdx.x / NG;
    const bool col_ok = i0 + col < I;
    for (int k = threadIdx.x; k < N; k += kFftThreads) tw[k] = tw_g[k];
    // in2 (optional): a second array of the same shape, added on load (into
    // buf1 first, which the transform then reuses)
    for (int part = 0; part < (in2 ? 2 : 1); ++part) {
        const float2 *src = (part ? in2 : in) + (b * n_in + n_first) * (size_t)ld + i0 + col;
        float2 *dst = (part ? buf1 : buf0) + n_first * kFftIB + col;
        const size_t src_step = (size_t)RPS * ld;
        for (int n = n_first; n < N; n += RPS, src += src_step, dst += RPS * kFftIB) {
            if (col_ok && n < n_in) {
                if (PAIRS)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(
                                     (unsigned)__cvta_generic_to_shared(dst)),
                                 "l"(src)
                                 : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                                     (unsigned)__cvta_generic_to_shared(dst)),
                                 "l"(src)
                                 : "memory");
            } else if (PAIRS) {
                *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                *dst = make_float2(0.f, 0.f);
            }
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    if constexpr (PAIRS) {
        // the last FFT stage writes the output rows itself: transform index t
        // goes to output row (t - out_off) mod N when that is below out_rows
        if constexpr (SPLIT) {
            const size_t plane = (size_t)sp.batch * sp.Kp;
            __nv_bfloat16 *A = sp.A + b * sp.Kp + i0;
            auto emit = [&](int t, int cp, float2 x0, float2 x1) {
                int r = t - out_off;
                if (r < 0) r += N;
                if (r >= out_rows || i0 + 2 * cp >= I) return;
                const float2 v0 = cscale(x0, scale), v1 = cscale(x1, scale);
                const __nv_bfloat16 h0 = __float2bfloat16(v0.x), h1 = __float2bfloat16(v1.x);
                const __nv_bfloat16 g0 = __float2bfloat16(v0.y), g1 = __float2bfloat16(v1.y);
                __nv_bfloat16 *o = A + (size_t)r * 4 * plane + 2 * cp;
                *reinterpret_cast<__nv_bfloat162 *>(o) = __halves2bfloat162(h0, h1);
                *reinterpret_cast<__nv_bfloat162 *>(o + 2 * plane) = __halves2bfloat162(g0, g1);
                if (sp.hi_only) return;
                *reinterpret_cast<__nv_bfloat162 *>(o + plane) = __halves2bfloat162(
                    __float2bfloat16(v0.x - __bfloat162float(h0)),
                    __float2bfloat16(v1.x - __bfloat162float(h1)));
                *reinterpret_cast<__nv_bfloat162 *>(o + 3 * plane) = __halves2bfloat162(
                    __float2bfloat16(v0.y - __bfloat162float(g0)),
                    __float2bfloat16(v1.y - __bfloat162float(g1)));
            };
            stockham_run_pairs_emit<kFftIB>(buf0, buf1, tw, plan, sgn, in2 != nullptr, emit);
        } else {
            float2 *o0 = out + b * out_rows * (size_t)ld + i0;
            __nv_bfloat162 *ob = reinterpret_cast<__nv_bfloat162 *>(out) + b * out_rows * (size_t)ld + i0;
            auto emit = [&](int t, int cp, float2 x0, float2 x1) {
                int r = t - out_off;
                if (r < 0) r += N;
                if (r >= out_rows || i0 + 2 * cp >= I) return;
                if (sp.bf16_rows) {
                    __nv_bfloat162 q[2] = {__floats2bfloat162_rn(scale * x0.x, scale * x0.y),
                                           __floats2bfloat162_rn(scale * x1.x, scale * x1.y)};
                    *reinterpret_cast<uint2 *>(ob + (size_t)r * ld + 2 * cp) =
                        *reinterpret_cast<const uint2 *>(q);
                    return;
                }
                *reinterpret_cast<float4 *>(o0 + (size_t)r * ld + 2 * cp) =
                    make_float4(scale * x0.x, scale * x0.y, scale * x1.x, scale * x1.y);
            };
            stockham_run_pairs_emit<kFftIB>(buf0, buf1, tw, plan, sgn, in2 != nullptr, emit);
        }
        return;
    }

    if (in2) {
        for (int idx = threadIdx.x; idx < N * kFftIB / 2; idx += kFftThreads) {
            float4 *a = reinterpret_cast<float4 *>(buf0) + idx;
            const float4 c = reinterpret_cast<const float4 *>(buf1)[idx];
            *a = make_float4(a->x + c.x, a->y + c.y, a->z + c.z, a->w + c.w);
        }
        __syncthreads();
    }
    // single columns (I odd or unaligned buffers)
    const float2 *src = stockham_run<true, kFftIB>(buf0, buf1, tw, plan, sgn, 1, kFftIB);
    // out_off < N and r < out_rows <= N: one conditional subtraction wraps
    if (!col_ok) return;
    if constexpr (SPLIT) {
        const size_t plane = (size_t)sp.batch * sp.Kp;
        __nv_bfloat16 *o = sp.A + (size_t)n_first * 4 * plane + b * sp.Kp + i0 + col;
        for (int r = n_first; r < out_rows; r += RPS, o += (size_t)RPS * 4 * plane) {
            int sr = r + out_off;
            if (sr >= N) sr -= N;
            const float2 t = cscale(src[sr * kFftIB + col], scale);
            const __nv_bfloat16 h = __float2bfloat16(t.x), g = __float2bfloat16(t.y);
            o[0] = h;
            o[2 * plane] = g;
            if (!sp.hi_only) {
                o[plane] = __float2bfloat16(t.x - __bfloat162float(h));
                o[3 * plane] = __float2bfloat16(t.y - __bfloat162float(g));
            }
        }
    } else if (sp.bf16_rows) {
        __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(out) +
                            (b * out_rows + n_first) * (size_t)ld + i0 + col;
        for (int r = n_first; r < out_rows; r += RPS, o += (size_t)RPS * ld) {
            int sr = r + out_off;
            if (sr >= N) sr -= N;
            const float2 t = cscale(src[sr * kFftIB + col], scale);
            *o = __floats2bfloat162_rn(t.x, t.y);
        }
    } else {
        float2 *o = out + (b * out_rows + n_first) * (size_t)ld + i0 + col;
        for (int r = n_first; r < out_rows; r += RPS, o += (size_t)RPS * ld) {
            int sr = r + out_off;
            if (sr >= N) sr -= N;
            *o = cscale(src[sr * kFftIB + col], scale);
        }
    }
}

// Direct DFT along the middle axis with an explicit phase matrix:
//   out[b][r][i] = scale * sum_{n < n_in} in[b][n][i] * T[r][n]
// 32 x 32 output tile per block, 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256)
k_dft_strided(const float2 *__restrict__ in, const float2 *__restrict__ in2, float2 *__restrict__ out,
              int n_in, int I, int out_rows, const float2 *__restrict__ T, float scale,
              int out_bf16) {
    __shared__ float2 xs[32][33];
    __shared__ float2 ts[32][33];
    const int tx = threadIdx.x & 31;
    const int ty = threadIdx.x >> 5;   // 0..7
    const int i = blockIdx.x * 32 + tx;
    const int r0 = blockIdx.y * 32;
    const size_t b = blockIdx.z;
    float2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int n0 = 0; n0 < n_in; n0 += 32) {
        for (int q = 0; q < 4; ++q) {
            const int nn = ty * 4 + q;
            const int n = n0 + nn;
            float2 x = make_float2(0.f, 0.f);
            if (n < n_in && i < I) {
                const size_t o = (b * n_in + n) * (size_t)I + i;
                x = in[o];
                if (in2) x = cadd(x, in2[o]);
            }
            xs[nn][tx] = x;
            const int rr = r0 + ty * 4 + q;
            ts[ty * 4 + q][tx] = (rr < out_rows && n0 + tx < n_in)
                                     ? T[(size_t)rr * n_in + n0 + tx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int nn = 0; nn < 32; ++nn) {
            const float2 x = xs[nn][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 t = ts[ty * 4 + q][nn];
                acc[q].x += x.x * t.x - x.y * t.y;
                acc[q].y += x.x * t.y + x.y * t.x;
            }
        }
        __syncthreads();
    }
    if (i < I) {
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + ty * 4 + q;
            if (r >= out_rows) continue;
            const float2 v = cscale(acc[q], scale);
            const size_t o = (b * out_rows + r) * (size_t)I + i;
            if (out_bf16)
                reinterpret_cast<__nv_bfloat162 *>(out)[o] = __floats2bfloat162_rn(v.x, v.y);
            else
                out[o] = v;
        }
    }
}

}  // namespace

size_t fft_strided_smem_bytes(int n) { return (size_t)(2 * n * kFftIB + n) * sizeof(float2); }

cudaError_t launch_fft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               const FftPlan &plan, const float2 *tw, int sgn, float scale,
                               int out_rows, int out_off, cudaStream_t st,
                               void *split_A, int split_Kp, const float2 *in2, int ld,
                               int bf16_out) {
    const size_t smem = fft_strided_smem_bytes(plan.n);
    // column pairs need 16-byte aligned rows: I even, 16-byte aligned
    // buffers, and (split output) an even operand row length
    if (ld <= 0) ld = I;
    if (ld < I) return cudaErrorInvalidValue;
    const bool pairs = (I % 2 == 0) && (ld % 2 == 0) && ((uintptr_t)in % 16 == 0) &&
                       ((uintptr_t)in2 % 16 == 0) &&
                       (split_A ? (split_Kp % 2 == 0 && (uintptr_t)split_A % 4 == 0)
                                : (uintptr_t)out % 16 == 0);
    auto kern = split_A ? (pairs ? k_fft_strided<true, true> : k_fft_strided<false, true>)
                        : (pairs ? k_fft_strided<true, false> : k_fft_strided<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((I + kFftIB - 1) / kFftIB, batch);
    // bf16_out: with split_A, the hi planes only; else bfloat16 (re, im) rows
    const SplitOut sp{(__nv_bfloat16 *)split_A, batch, split_Kp, split_A ? bf16_out : 0,
                      split_A ? 0 : bf16_out};
    kern<<<grid, kFftThreads, smem, st>>>(in, in2, out, n_in, I, ld, plan, tw, sgn, scale, out_rows, out_off,
                                  sp);
    return cudaGetLastError();
}

cudaError_t launch_dft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               int out_rows, const float2 *T, float scale, cudaStream_t st,
                               const float2 *in2, int bf16_out) {
    dim3 grid((I + 31) / 32, (out_rows + 31) / 32, batch);
    k_dft_strided<<<grid, 256, 0, st>>>(in, in2, out, n_in, I, out_rows, T, scale, bf16_out);
    return cudaGetLastError();
}

namespace {

// Exponent all ones <=> NaN or Inf, decided on the bits (no float compare).
__device__ __forceinline__ bool nonfinite_bits(float v) {
    return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

__global__ void __launch_bounds__(256) k_check_finite(const float4 *__restrict__ x4, size_t n4,
                                                     const float2 *__restrict__ tail, int n_tail,
                                                     int *flag) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(&x4[i]);
        bad |= nonfinite_bits(v.x) | nonfinite_bits(v.y) | nonfinite_bits(v.z) |
               nonfinite_bits(v.w);
    }
    if (blockIdx.x == 0 && (int)threadIdx.x < n_tail) {
        const float2 v = tail[threadIdx.x];
        bad |= nonfinite_bits(v.x) | nonfinite_bits(v.y);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, PL_FLAG_NONFINITE);
}

}  // namespace

cudaError_t launch_check_finite(const float2 *x, size_t n, int *flag, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (!x || !flag) return cudaErrorInvalidValue;
    // float4 body from the first 16-byte boundary; the rest (at most two
    // leading or one trailing complex value) read as float2
    const size_t lead = ((uintptr_t)x % 16) ? 1 : 0;       // x is 8-byte aligned
    if (lead && n == 1) {
        k_check_finite<<<1, 32, 0, st>>>(nullptr, 0, x, 1, flag);
        return cudaGetLastError();
    }
    const size_t body = (n - lead) / 2;                      // float4 = two complex values
    const size_t rest = n - lead - 2 * body;                 // 0 or 1
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t want = (body + 255) / 256;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)sms * 8));
    if (lead) {
        k_check_finite<<<1, 32, 0, st>>>(nullptr, 0, x, 1, flag);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_check_finite<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(x + lead), body,
                                           x + lead + 2 * body, (int)rest, flag);
    return cudaGetLastError();
}
