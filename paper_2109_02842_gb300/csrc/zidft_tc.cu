// Inverse transform over k_z (step 9) at voxel heights off the scan grid, on
// the fifth-generation tensor cores:
//
//   image[z][p] = sum_u T[z][u] G[u][p],   T[z][u] = e^{j k_z(u) (z_v - z_0)} / N_p,
//
// with G the sum of the back-projection's channel parts. It is a complex
// matrix product with K = N_p bins; the FP32 DFT kernel spends ~4 flop per
// byte of G on the CUDA cores, which leaves it far from the memory bound. Here
// a block takes 128 pixels (the MMA's M, one TMEM lane each) and NZC output
// heights (the MMA's N) over every bin, 16 bins (one K step) at a time:
//  * A = G^T [pixel][bin]: warps 0-7 (two classes of four, one lane quarter
//    each) load their pixel's 16 bins of both channel parts (coalesced rows of
//    G), add them, split Re and Im into BF16 hi + lo and write the four
//    planes to the class's A buffer in tensor memory (tcgen05.st); the
//    classes take alternate K steps so one class's loads overlap the other's
//    products;
//  * B = T^T [bin][height]: a BF16 table of four planes (Re hi, Re lo, Im hi,
//    Im lo), rows = heights, bins contiguous (K-major), built at plan time
//    with 1 / N_p folded in; warp 9 streams one box of 16 bins x NZC heights
//    per plane per K step (32-byte swizzle, the layout the MMA reads) into a
//    ring of stages;
//  * warp 8 (one lane) issues per K step the twelve products of the
//    hi/lo-split complex product into the planar accumulators Re D and Im D
//    (NZC columns each; the minus of Re G Re T - Im G Im T through the
//    descriptor's negate-A bit);
//  * at the end warps 0-7 read the accumulators back (lane = pixel, column =
//    height) and write image rows, 32 consecutive pixels per warp and height.
// Relative error of the split products ~1e-5 (as the back-projection's).
// Every wait is bounded; an expired wait sets a bit (1 << 8 .. 1 << 11) in
// *err and the block drains its copies and products before it releases
// tensor memory. (a.dbg_wait makes the MMA warp wait first on a barrier
// nothing completes, so that tests can run these exit paths.)
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc05.cuh"

namespace {

constexpr int kAWarps = 8;                       // two classes of four warps
constexpr int kThreads = (kAWarps + 2) * 32;     // + MMA warp + TMA warp
constexpr int kStages = 4;
constexpr uint32_t kTmemCols = 256;              // 2 NZC accumulators + 2 x 32 A columns

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
// BF16 pair (a, b) and the BF16 pair of its residuals
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = bf2(a, b);
    lo = bf2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}
// K-major operand, 32-byte swizzle: rows of 32 B, 8-row groups 256 B apart
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
    return tc05::smem_desc(saddr, 16, 256) | (6ull << 61);
}

__global__ void __launch_bounds__(kThreads, 2)
k_zidft_tc(const __grid_constant__ CUtensorMap tmap, const float2 *__restrict__ G,
           const float2 *__restrict__ G2, float2 *__restrict__ out, ZidftTcArgs a, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], a_full[2], a_done[2], acc_full,
        dbg_bar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NZC = a.nzc;
    const uint32_t plane = (uint32_t)a.plane_bytes;
    const uint32_t stage = 4 * plane;
    const int zc = (int)blockIdx.x % a.zchunks;
    const int p0 = ((int)blockIdx.x / a.zchunks) * 128;
    const int z0 = zc * NZC;
    const long long budget = a.budget;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc05::mbar_init(&full[s], 1);
            tc05::mbar_init(&empty[s], 1);
        }
        for (int k = 0; k < 2; ++k) {
            tc05::mbar_init(&a_full[k], 4);
            tc05::mbar_init(&a_done[k], 1);
        }
        tc05::mbar_init(&acc_full, 1);
        tc05::mbar_init(&dbg_bar, 1);      // never arrived on (test hook)
        tc05::fence_mbar_init();
    }
    if (warp == 0) {
        tc05::tmem_alloc(&tmem_slot, kTmemCols);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t acol = 2 * (uint32_t)NZC;          // A buffers follow the accumulators
    int issued = 0, committed = 0;

    if (warp < kAWarps) {
        // ------------------------------------------------ A (G^T, split)
        const int cls = warp >> 2, q = warp & 3;
        const int col = p0 + 32 * q + lane;
        const bool live = col < a.n_cols;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t abuf = lane_base + acol + 32 * cls;
        bool ok = true;
        int r = 0;
        for (int s = cls; s < a.ksteps; s += 2, ++r) {
            float2 v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int u = 16 * s + j;
                v[j] = make_float2(0.f, 0.f);
                if (live && u < a.n_in) {
                    const size_t o = (size_t)u * a.ld + col;
                    v[j] = G[o];
                    if (G2) {
                        const float2 w = G2[o];
                        v[j].x += w.x;
                        v[j].y += w.y;
                    }
                }
            }
            // the products of the class's previous K step have read its buffer
            if (r > 0) ok = tc05::mbar_wait(&a_done[cls], (uint32_t)(r - 1) & 1u, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc05::fence_after_sync();
            uint32_t rh[8], rl[8], ih[8], il[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                split2(v[2 * j].x, v[2 * j + 1].x, rh[j], rl[j]);
                split2(v[2 * j].y, v[2 * j + 1].y, ih[j], il[j]);
            }
            tc05::tmem_st8(abuf, rh);
            tc05::tmem_st8(abuf + 8, rl);
            tc05::tmem_st8(abuf + 16, ih);
            tc05::tmem_st8(abuf + 24, il);
            tc05::tmem_wait_st();
            tc05::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&a_full[cls]);
        }
        // the release of the class's last K step has arrived
        if (ok && r > 0)
            ok = __all_sync(0xffffffffu,
                            tc05::mbar_wait(&a_done[cls], (uint32_t)(r - 1) & 1u, budget));
        if (!ok && lane == 0) atomicOr(err, 1 << 8);

        // ------------------------------------------------ epilogue
        bool done = __all_sync(0xffffffffu, tc05::mbar_wait(&acc_full, 0, budget));
        if (done) {
            tc05::fence_after_sync();
            for (int ch = cls; ch < NZC / 16; ch += 2) {
                uint32_t re[16], im[16];
                tc05::tmem_ld16(lane_base + 16 * ch, re);
                tc05::tmem_ld16(lane_base + NZC + 16 * ch, im);
                tc05::tmem_wait_ld();
                if (!live) continue;
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    const int z = z0 + 16 * ch + b;
                    if (z < a.nz)
                        out[(size_t)z * a.out_ld + col] =
                            make_float2(__uint_as_float(re[b]), __uint_as_float(im[b]));
                }
            }
        } else if (lane == 0) {
            atomicOr(err, 1 << 9);
        }
    } else if (warp == kAWarps) {
        // ------------------------------------------------ MMA issue
        const uint32_t idesc = tc05::idesc_bf16(128, NZC, 0);
        const uint32_t idn = idesc | (1u << 13);        // negated A
        const uint32_t dre = tmem, dim = tmem + (uint32_t)NZC;
        bool ok = true;
        if (a.dbg_wait) ok = __all_sync(0xffffffffu, tc05::mbar_wait(&dbg_bar, 0, budget));
        for (int s = 0; s < a.ksteps && ok; ++s) {
            const int st = s % kStages, cls = s & 1;
            ok = tc05::mbar_wait(&full[st], (uint32_t)(s / kStages) & 1u, budget) &&
                 tc05::mbar_wait(&a_full[cls], (uint32_t)(s >> 1) & 1u, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc05::fence_after_sync();
            if (lane == 0) {
                const uint32_t base = tc05::smem_addr(smem + (size_t)st * stage);
                const uint64_t bh = desc_sw32(base), bl = desc_sw32(base + plane);
                const uint64_t bi = desc_sw32(base + 2 * plane), bil = desc_sw32(base + 3 * plane);
                const uint32_t ar = tmem + acol + 32 * cls, arl = ar + 8, ai = ar + 16, ail = ar + 24;
                const uint32_t acc = s > 0 ? 1u : 0u;
                // Re D += Re G Re T - Im G Im T
                tc05::mma_ts(dre, ar, bh, idesc, acc);
                tc05::mma_ts(dre, ar, bl, idesc, 1u);
                tc05::mma_ts(dre, arl, bh, idesc, 1u);
                tc05::mma_ts(dre, ai, bi, idn, 1u);
                tc05::mma_ts(dre, ai, bil, idn, 1u);
                tc05::mma_ts(dre, ail, bi, idn, 1u);
                // Im D += Re G Im T + Im G Re T
                tc05::mma_ts(dim, ar, bi, idesc, acc);
                tc05::mma_ts(dim, ar, bil, idesc, 1u);
                tc05::mma_ts(dim, arl, bi, idesc, 1u);
                tc05::mma_ts(dim, ai, bh, idesc, 1u);
                tc05::mma_ts(dim, ai, bl, idesc, 1u);
                tc05::mma_ts(dim, ail, bh, idesc, 1u);
                tc05::mma_commit(&a_done[cls]);
                tc05::mma_commit(&empty[st]);
            }
            __syncwarp();
            committed = s + 1;
        }
        if (lane == 0) {
            if (!ok) atomicOr(err, 1 << 10);
            tc05::mma_commit(&acc_full);
        }
    } else {
        // ------------------------------------------------ TMA producer
        bool ok = true;
        for (int s = 0; s < a.ksteps; ++s) {
            const int st = s % kStages;
            if (s >= kStages) ok = tc05::mbar_wait(&empty[st], (uint32_t)(s / kStages - 1) & 1u, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (lane == 0) {
                unsigned char *dst = smem + (size_t)st * stage;
                tc05::mbar_arrive_expect_tx(&full[st], 4u * (uint32_t)NZC * 32u);
#pragma unroll
                for (int pl = 0; pl < 4; ++pl)
                    tc05::tma_load_2d(dst + pl * plane, &tmap, &full[st], 16 * s, pl * a.nzp + z0);
            }
            __syncwarp();
            issued = s + 1;
        }
        if (!ok && lane == 0) atomicOr(err, 1 << 11);
    }
    // before shared and tensor memory are released: every copy issued has
    // landed and every product issued has completed (waiting again on a
    // completed phase returns at once)
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == kAWarps + 1 && lane == 0)
        for (int s = issued > kStages ? issued - kStages : 0; s < issued; ++s)
            tc05::mbar_wait(&full[s % kStages], (uint32_t)(s / kStages) & 1u, budget);
    if (warp == kAWarps && lane == 0 && committed > 0)
        tc05::mbar_wait(&empty[(committed - 1) % kStages],
                        (uint32_t)((committed - 1) / kStages) & 1u, budget);
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
}

// The BF16 table of the transform: plane 0 / 1 = Re T hi / lo, 2 / 3 = Im T
// hi / lo, [plane][nzp][kp] with the scale folded in and zeros past (nz, n_in).
__global__ void k_zidft_tc_table(const float2 *__restrict__ T, int nz, int n_in, float scale,
                                 int nzp, int kp, __nv_bfloat16 *__restrict__ tb) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nzp * kp) return;
    const int z = (int)(idx / kp), u = (int)(idx - (long long)z * kp);
    float re = 0.f, im = 0.f;
    if (z < nz && u < n_in) {
        const float2 t = T[(size_t)z * n_in + u];
        re = t.x * scale;
        im = t.y * scale;
    }
    const __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
    const size_t pl = (size_t)nzp * kp;
    tb[idx] = rh;
    tb[pl + idx] = __float2bfloat16_rn(re - __bfloat162float(rh));
    tb[2 * pl + idx] = ih;
    tb[3 * pl + idx] = __float2bfloat16_rn(im - __bfloat162float(ih));
}

}  // namespace

ZidftTcArgs zidft_tc_shape(int n_in, int n_cols, int nz) {
    ZidftTcArgs a{};
    a.n_in = n_in;
    a.ksteps = (n_in + 15) / 16;
    a.n_cols = n_cols;
    a.ld = n_cols;
    a.out_ld = n_cols;
    a.nz = nz;
    // heights per block: at most 96 (two accumulators of 96 columns and two
    // A buffers of 32 fit 256 TMEM columns: two blocks per SM), evenly split
    const int nz16 = (nz + 15) / 16 * 16;
    a.zchunks = (nz16 + 95) / 96;
    a.nzc = ((nz + a.zchunks - 1) / a.zchunks + 15) / 16 * 16;
    a.nzp = a.zchunks * a.nzc;
    a.plane_bytes = (a.nzc * 32 + 1023) / 1024 * 1024;
    return a;
}

size_t zidft_tc_table_elems(const ZidftTcArgs &a) { return (size_t)4 * a.nzp * (16 * a.ksteps); }

cudaError_t launch_zidft_tc_table(const ZidftTcArgs &a, const float2 *T, float scale,
                                  __nv_bfloat16 *tb, cudaStream_t st) {
    const int kp = 16 * a.ksteps;
    const long long n = (long long)a.nzp * kp;
    k_zidft_tc_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T, a.nz, a.n_in, scale, a.nzp, kp,
                                                                tb);
    return cudaGetLastError();
}

bool zidft_tc_make_map(const ZidftTcArgs &a, const __nv_bfloat16 *tb, CUtensorMap *map,
                       TmapEncodeFn enc) {
    if (!enc) return false;
    const int kp = 16 * a.ksteps;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)4 * a.nzp};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {16, (cuuint32_t)a.nzc};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(tb), dims,
               strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

size_t zidft_tc_smem_bytes(const ZidftTcArgs &a) {
    return 1024 + (size_t)kStages * 4 * a.plane_bytes;
}

cudaError_t launch_zidft_tc(const ZidftTcArgs &a, const CUtensorMap *map, const float2 *G,
                            const float2 *G2, float2 *out, int *err, cudaStream_t st) {
    if (a.n_cols <= 0 || a.nz <= 0 || a.ksteps <= 0) return cudaSuccess;
    if (a.nzc < 16 || a.nzc > 96 || a.nzc % 16 || 2 * a.nzc + 64 > (int)kTmemCols)
        return cudaErrorInvalidValue;
    const size_t smem = zidft_tc_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(k_zidft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)((a.n_cols + 127) / 128) * a.zchunks;
    k_zidft_tc<<<(unsigned)blocks, kThreads, smem, st>>>(*map, G, G2, out, a, err);
    return cudaGetLastError();
}
