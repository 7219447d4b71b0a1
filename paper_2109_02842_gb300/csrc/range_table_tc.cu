// Range-profile table of step (8a) / (19a) for the tensor-core back-projection,
// evaluated as exact sums on the tensor cores instead of a type-1 NUFFT:
//
//   b[c][i][u] = sum_m a[c][u][m] e^{+j theta_um (i - L/2)},   a = S alpha,
//
// theta_um = kappa''_um h and alpha as in setup.cu (k weight, 1/phihat of the
// interpolation kernel, range-origin phase). For one k_z bin u this is a
// complex matrix product over the frequencies: channels (M = 128 per block) x
// table rows (N = L rounded up to 16) x frequencies (K). Operands are BF16
// split hi + lo (three products per real product), the complex product is
// four real ones with the imaginary-by-imaginary term negated through the
// instruction descriptor, and the two accumulators (Re, Im) live in TMEM.
//
//   k_rt_prep          S [C][N_p][M] x alpha -> A [u][re hi, re lo, im hi, im lo][C][K] BF16
//   k_range_table_tc   per (128-channel block, bin, row part): TMA (128-byte
//                      swizzled, K-major) A and E tiles, 12 MMAs per
//                      16-frequency step, tcgen05.ld, BF16 hi/lo, staged per warp
//                      and stored as full lines of each channel's consecutive
//                      rows into prod [u][hi, lo][part][C][Lh] of (re, im) pairs
//                      (Lh rows per part, a multiple of 16). Two row parts when that lets two
//                      blocks share an SM (256 TMEM columns, ~107 KB of shared
//                      memory each), so one block's loads, products and stores
//                      overlap the other's.
//   k_rt_transpose     prod -> table [c][hi, lo][L][column 2u + (re, im)] (or
//                      planar: Re at column u, Im at row_words + u), the layout
//                      the back-projection streams (u innermost)
//
// E [u][re hi, re lo, im hi, im lo][L'][K] = e^{+j theta (i - L/2)} is a plan-time table.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

namespace {

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16(x);
    lo = __float2bfloat16(x - __bfloat162float(hi));
}

__device__ __forceinline__ double kz_at(int u, int n_pad, double dz) {
    const int ut = (2 * u < n_pad) ? u : u - n_pad;
    return PL_TWO_PI * (double)ut / ((double)n_pad * dz);
}

__global__ void k_setup_rt_E(NufftDesc d, double dz, const double *k, const double *kc, int Lp,
                             int Kp, __nv_bfloat16 *E) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)d.n_pad * Lp * Kp) return;
    const int m = (int)(idx % Kp);
    const int i = (int)((idx / Kp) % Lp);
    const int u = (int)(idx / ((long long)Kp * Lp));
    double re = 0.0, im = 0.0;
    if (i < d.L && m < d.n_f) {
        const double kz = kz_at(u, d.n_pad, dz);
        const double q = d.mode == 0 ? 4.0 * k[m] * k[m] - kz * kz : k[m] * k[m] - 0.25 * kz * kz;
        if (q > 0.0) {
            const double ph = (sqrt(q) - kc[u]) * d.h * (double)(i - d.L / 2);
            re = cos(ph);
            im = sin(ph);
        }
    }
    __nv_bfloat16 h, l;
    const size_t plane = (size_t)Lp * Kp;
    const size_t base = (size_t)u * 4 * plane + (size_t)i * Kp + m;
    split_bf16((float)re, h, l);
    E[base] = h;
    E[base + plane] = l;
    split_bf16((float)im, h, l);
    E[base + 2 * plane] = h;
    E[base + 3 * plane] = l;
}

// A[u][plane][c][m] = split(S[c][u][m] alpha[u][m]) (zero for m >= M)
__global__ void k_rt_prep(const float2 *__restrict__ S, const float2 *__restrict__ alpha, int C,
                          int Np, int M, int Kp, __nv_bfloat16 *__restrict__ A) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)C * Np * Kp) return;
    const int m = (int)(idx % Kp);
    const int u = (int)((idx / Kp) % Np);
    const int c = (int)(idx / ((long long)Kp * Np));
    float2 a = make_float2(0.f, 0.f);
    if (m < M) a = cmul(S[((size_t)c * Np + u) * M + m], alpha[(size_t)u * M + m]);
    __nv_bfloat16 h, l;
    const size_t plane = (size_t)C * Kp;
    const size_t base = (size_t)u * 4 * plane + (size_t)c * Kp + m;
    split_bf16(a.x, h, l);
    A[base] = h;
    A[base + plane] = l;
    split_bf16(a.y, h, l);
    A[base + 2 * plane] = h;
    A[base + 3 * plane] = l;
}

__global__ void __launch_bounds__(128, 1)
k_range_table_tc(RtTcArgs ra, const __grid_constant__ CUtensorMap tmA,
                 const __grid_constant__ CUtensorMap tmB, uint32_t *__restrict__ prod, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * 128, u = blockIdx.y, h = blockIdx.z;
    const uint32_t a_tile = 128 * 128;                 // one plane x 64-frequency atom of A
    const uint32_t b_tile = (uint32_t)ra.Lh * 128;     // of E (this part's rows)
    const uint32_t tcols = 2 * ra.Lh > 256 ? 512 : (2 * ra.Lh > 128 ? 256 : 128);
    unsigned char *As = smem;
    unsigned char *Bs = smem + 4 * ra.natoms * a_tile;

    if (threadIdx.x == 0) {
        tc05::mbar_init(&bar_tma, 1);
        tc05::mbar_init(&bar_mma, 1);
        tc05::fence_mbar_init();
    }
    if (warp == 0) {
        tc05::tmem_alloc(&tmem_slot, tcols);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (threadIdx.x == 0) {
        tc05::mbar_arrive_expect_tx(&bar_tma, 4 * ra.natoms * (a_tile + b_tile));
        for (int p = 0; p < 4; ++p)
            for (int at = 0; at < ra.natoms; ++at) {
                const int t = p * ra.natoms + at;
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(tc05::smem_addr(As + t * a_tile)),
                    "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(64 * at), "r"(c0), "r"(4 * u + p),
                    "r"(tc05::smem_addr(&bar_tma))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(tc05::smem_addr(Bs + t * b_tile)),
                    "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(64 * at), "r"(h * ra.Lh), "r"(4 * u + p),
                    "r"(tc05::smem_addr(&bar_tma))
                    : "memory");
            }
        bool ok = tc05::mbar_wait(&bar_tma, 0, ra.budget);
        if (ok) {
            tc05::fence_after_sync();
            const uint32_t id = ra.idesc, idn = ra.idesc | (1u << 13);   // negate A
            const uint32_t dre = tmem, dim = tmem + ra.Lh;
            for (int ks = 0; ks < ra.natoms * 4; ++ks) {
                const int at = ks >> 2;
                const uint32_t ko = (ks & 3) * 32;
                auto da = [&](int p) {
                    return tc05::smem_desc_sw128(tc05::smem_addr(As + (p * ra.natoms + at) * a_tile) + ko,
                                                 16, 1024);
                };
                auto db = [&](int p) {
                    return tc05::smem_desc_sw128(tc05::smem_addr(Bs + (p * ra.natoms + at) * b_tile) + ko,
                                                 16, 1024);
                };
                const uint32_t acc = ks > 0 ? 1u : 0u;
                // planes: 0 re hi, 1 re lo, 2 im hi, 3 im lo
                // Re += a_r b_r - a_i b_i
                tc05::mma_ss(dre, da(0), db(0), id, acc);
                tc05::mma_ss(dre, da(0), db(1), id, 1u);
                tc05::mma_ss(dre, da(1), db(0), id, 1u);
                tc05::mma_ss(dre, da(2), db(2), idn, 1u);
                tc05::mma_ss(dre, da(2), db(3), idn, 1u);
                tc05::mma_ss(dre, da(3), db(2), idn, 1u);
                // Im += a_r b_i + a_i b_r
                tc05::mma_ss(dim, da(0), db(2), id, acc);
                tc05::mma_ss(dim, da(0), db(3), id, 1u);
                tc05::mma_ss(dim, da(1), db(2), id, 1u);
                tc05::mma_ss(dim, da(2), db(0), id, 1u);
                tc05::mma_ss(dim, da(2), db(1), id, 1u);
                tc05::mma_ss(dim, da(3), db(0), id, 1u);
            }
        } else {
            atomicOr(err, 1);
        }
        tc05::mma_commit(&bar_mma);   // arrives once every issued MMA completed
    }
    __syncwarp();
    bool done = tc05::mbar_wait(&bar_mma, 0, ra.budget);
    done = __all_sync(0xffffffffu, done);
    // output in 32-row chunks: each thread (one channel: its TMEM lane)
    // converts its rows to BF16 hi/lo pairs and puts them in its warp's
    // staging rows (33 words apart: conflict-free), then the warp writes one
    // channel's 32 consecutive rows per store instruction (a full 128-byte
    // line of prod, where a channel's rows are contiguous). The operand tiles
    // are dead by now and hold the staging.
    const int rows_here = min(ra.Lh, ra.L - h * ra.Lh);     // table rows of this part
    if (done) {
        tc05::fence_after_sync();
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        uint32_t *st = reinterpret_cast<uint32_t *>(smem) + warp * (2 * 32 * 33);
        const int cw = c0 + 32 * warp;                       // the warp's first channel
        uint32_t *g_hi = prod + ((size_t)(2 * u + 0) * ra.nh + h) * ra.C * ra.Lh;
        uint32_t *g_lo = prod + ((size_t)(2 * u + 1) * ra.nh + h) * ra.C * ra.Lh;
        for (int i0 = 0; i0 < rows_here; i0 += 32) {
            const int nrow = min(32, ra.Lh - i0);            // 16 or 32 columns of the part
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (16 * half >= nrow) break;
                uint32_t vr[16], vi[16];
                tc05::tmem_ld16(lane_base + i0 + 16 * half, vr);
                tc05::tmem_ld16(lane_base + ra.Lh + i0 + 16 * half, vi);
                tc05::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float re = __uint_as_float(vr[j]), im = __uint_as_float(vi[j]);
                    __nv_bfloat162 hv = __floats2bfloat162_rn(re, im);
                    const float2 hf = __bfloat1622float2(hv);
                    __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
                    st[lane * 33 + 16 * half + j] = *reinterpret_cast<uint32_t *>(&hv);
                    st[32 * 33 + lane * 33 + 16 * half + j] = *reinterpret_cast<uint32_t *>(&l);
                }
            }
            __syncwarp();
            if (lane < nrow) {
                for (int rr = 0; rr < 32 && cw + rr < ra.C; ++rr) {
                    const size_t o = (size_t)(cw + rr) * ra.Lh + i0 + lane;
                    g_hi[o] = st[rr * 33 + lane];
                    g_lo[o] = st[32 * 33 + rr * 33 + lane];
                }
            }
            __syncwarp();
        }
    } else if (lane == 0) {
        atomicOr(err, 2);
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, tcols);
}

// prod [u][plane][part][C][Lh] (uint32 = (re, im) BF16 pair) -> table
// [c][plane][L][u], u beyond N_p written as zeros so the padding columns stay
// zero. Interleaved rows hold row_words (re, im) pairs; planar rows hold
// row_words Re entries, then row_words Im. A block covers 64 rows x 64 bins;
// each thread transposes a 4 x 4 block in registers: four independent 16-byte
// loads (4 rows i of one bin each) and four row stores, so a warp (16 rows x
// 32 bins) reads and writes 64-byte runs with no shared memory or barrier.
__device__ __forceinline__ uint32_t word_of(const uint4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

template <bool PLANAR>
__global__ void __launch_bounds__(256)
k_rt_transpose(const uint32_t *__restrict__ prod, uint32_t *__restrict__ table, int C, int L,
               int nh, int Lh, int Np, int row_words) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 64 + 16 * (warp & 3) + 4 * (lane & 3);
    const int u = blockIdx.y * 64 + 32 * (warp >> 2) + 4 * (lane >> 2);
    const int cp = blockIdx.z;                 // c * 2 + plane
    const int c = cp >> 1, p = cp & 1;
    if (i >= L || u >= row_words) return;      // row_words is a multiple of 4
    // row i lives in part i / Lh (Lh is a multiple of 16: rows i..i+3 stay in
    // one part; those at L and beyond are padding, loaded but never stored)
    const int hp = i / Lh;
    const uint32_t *src = prod + ((size_t)hp * C + c) * Lh + (i - hp * Lh);
    const size_t bin_stride = (size_t)2 * nh * C * Lh;
    uint4 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        v[r] = u + r < Np ? *reinterpret_cast<const uint4 *>(src + (size_t)(u + r) * bin_stride +
                                                              (size_t)p * nh * C * Lh)
                          : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (i + e >= L) break;
        const uint32_t w0 = word_of(v[0], e), w1 = word_of(v[1], e);
        const uint32_t w2 = word_of(v[2], e), w3 = word_of(v[3], e);
        uint32_t *row = table + ((size_t)cp * L + i + e) * row_words;
        if (PLANAR) {
            // low halves (Re) of the four bins, then the high halves (Im)
            __nv_bfloat16 *rb = reinterpret_cast<__nv_bfloat16 *>(row);
            *reinterpret_cast<uint2 *>(rb + u) =
                make_uint2(__byte_perm(w0, w1, 0x5410), __byte_perm(w2, w3, 0x5410));
            *reinterpret_cast<uint2 *>(rb + row_words + u) =
                make_uint2(__byte_perm(w0, w1, 0x7632), __byte_perm(w2, w3, 0x7632));
        } else {
            *reinterpret_cast<uint4 *>(row + u) = make_uint4(w0, w1, w2, w3);
        }
    }
}

}  // namespace

size_t range_table_tc_smem_bytes(const RtTcArgs &ra) {
    return 1024 + (size_t)4 * ra.natoms * (128 * 128 + (size_t)ra.Lh * 128);
}

cudaError_t launch_setup_rt_E(const NufftDesc &d, double dz, const double *k, const double *kc,
                              int Lp, int Kp, void *E, cudaStream_t st) {
    const long long n = (long long)d.n_pad * Lp * Kp;
    k_setup_rt_E<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, dz, k, kc, Lp, Kp,
                                                              (__nv_bfloat16 *)E);
    return cudaGetLastError();
}

cudaError_t launch_range_table_tc(const RtTcArgs &ra, const CUtensorMap &tmA,
                                  const CUtensorMap &tmB, const float2 *S, const float2 *alpha,
                                  void *A, void *prod, void *table, int row_words, int planar,
                                  int *err, bool prepared, cudaStream_t st) {
    cudaError_t e;
    if (!prepared) {     // the z transform wrote S, not the split operand
        const long long n = (long long)ra.C * ra.Np * ra.Kp;
        k_rt_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, alpha, ra.C, ra.Np, ra.M,
                                                               ra.Kp, (__nv_bfloat16 *)A);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const size_t smem = range_table_tc_smem_bytes(ra);
    e = cudaFuncSetAttribute(k_range_table_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((ra.C + 127) / 128, ra.Np, ra.nh);
    k_range_table_tc<<<grid, 128, smem, st>>>(ra, tmA, tmB, (uint32_t *)prod, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (row_words % 4 != 0 || ra.Lh % 16 != 0) return cudaErrorInvalidValue;
    dim3 tg((ra.L + 63) / 64, (row_words + 63) / 64, 2 * ra.C);
    if (planar)
        k_rt_transpose<true><<<tg, 256, 0, st>>>((const uint32_t *)prod, (uint32_t *)table, ra.C,
                                                 ra.L, ra.nh, ra.Lh, ra.Np, row_words);
    else
        k_rt_transpose<false><<<tg, 256, 0, st>>>((const uint32_t *)prod, (uint32_t *)table, ra.C,
                                                  ra.L, ra.nh, ra.Lh, ra.Np, row_words);
    return cudaGetLastError();
}
