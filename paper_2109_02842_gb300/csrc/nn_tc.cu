// The learned path's 3 x 3 x 3 convolution on the fifth-generation tensor
// cores (tcgen05), for the shapes the network runs at full size: Cin a
// multiple of 16, Cout in 1..16 (the MMA's N = 16) or {32, 64, 128}, rows of W
// in {16, 32, 64, 128} voxels with 128 / W dividing H. Other shapes (the
// 3-channel input layer, odd sizes) keep the mma.sync kernel of nn.cu.
//
// Implicit GEMM: out[v][co] = act(bias[co] + sum_{tap, ci} x[v + off(tap)][ci]
// w[co][tap Cin + ci]). A tile is 128 consecutive voxels (the MMA's M: 128 / W
// whole rows of one z slice); its K runs over 27 taps x Cin / 16 channel
// chunks. For tap (dz, dy, dx) and chunk j the A operand is a TMA box
// {16 channels, W, 128 / W, 1} of the activations [D][H][W][Cin] at
// (16 j, dx - 1, y0 + dy - 1, z + dz - 1): the row shifted by the tap, with the
// zero padding of the convolution supplied by the out-of-bounds fill. The B
// operand is the box {16, Cout} of the weights [Cout][Kp] at (tap Cin + 16 j,
// 0). Both land 32-byte swizzled in shared memory -- the K-major layout the
// MMA reads (16 BF16 = one K step per row).
//
// Block (persistent, tiles gridDim.x apart): warps 0-3 read the accumulator
// back (TMEM lanes = the tile's voxels), add the bias, apply the ReLU and
// store; warp 4 (one lane) issues the copies into a ring of stages; warp 5
// (one lane) issues one M = 128, N = Cout, K = 16 product per stage into one of
// two TMEM accumulators, so that a tile's epilogue overlaps the next tile's
// products. Every wait is bounded; a wait that runs out sets g_conv_tc_err and
// the block drains its copies and products before it releases tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/polyline.h"
#include "kernels.h"
#include "tc05.cuh"

namespace {

constexpr int kStages = 8;
constexpr int kThreads = 192;     // 4 epilogue warps + producer warp + MMA warp
constexpr uint32_t kABytes = 128 * 32;

__device__ int g_conv_tc_err;     // wait-expired bits (kept until the process ends)

struct ConvTcArgs {
    int tiles;          // V / 128
    int tiles_per_z;    // H W / 128
    int bh;             // rows of y per tile (128 / W)
    int chunks;         // Cin / 16
    int relu;
    int Cout;
    long long budget;   // wait budget, SM clock cycles
};

// K-major operand, 32-byte swizzle: rows of 32 B, 8-row groups 256 B apart
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
    return tc05::smem_desc(saddr, 16, 256) | (6ull << 61);
}

template <int N, bool OUT_BF16>
__global__ void __launch_bounds__(kThreads)
k_conv3d_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
            const float *__restrict__ bias, void *__restrict__ out, ConvTcArgs a) {
    constexpr uint32_t kBBytes = N * 32;
    constexpr uint32_t kStage = kABytes + kBBytes;
    constexpr int kTmemCols = 2 * N < 32 ? 32 : 2 * N;     // two accumulators
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float s_bias[N];
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int steps = 27 * a.chunks;
    const int my_tiles = (a.tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc05::mbar_init(&full[s], 1);
            tc05::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc05::mbar_init(&acc_full[b], 1);
            tc05::mbar_init(&acc_empty[b], 4);
        }
        tc05::fence_mbar_init();
        abort_flag = 0;
    }
    for (int i = threadIdx.x; i < N; i += kThreads) s_bias[i] = (bias && i < a.Cout) ? bias[i] : 0.f;
    if (warp == 0) {
        tc05::tmem_alloc(&tmem_slot, kTmemCols);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    int issued = 0, committed = 0;       // stages copied (warp 4) / multiplied (warp 5)

    if (warp == 4) {
        // ---------------------------------------------------------- copies
        if (lane == 0) {
            int it = 0;
            for (int t = 0; t < my_tiles && !abort_flag; ++t) {
                const int tile = (int)blockIdx.x + t * (int)gridDim.x;
                const int z = tile / a.tiles_per_z;
                const int y0 = (tile - z * a.tiles_per_z) * a.bh;
                for (int st = 0; st < steps; ++st, ++it) {
                    const int s = it % kStages, round = it / kStages;
                    if (round > 0 &&
                        !tc05::mbar_wait(&empty[s], (uint32_t)(round - 1) & 1u, a.budget)) {
                        atomicOr(&g_conv_tc_err, 1);
                        abort_flag = 1;
                        break;
                    }
                    const int tap = st / a.chunks, j = st - tap * a.chunks;
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                    unsigned char *As = smem + (size_t)s * kStage;
                    tc05::mbar_arrive_expect_tx(&full[s], kStage);
                    tc05::tma_load_4d(As, &tmX, &full[s], 16 * j, dx - 1, y0 + dy - 1, z + dz - 1);
                    tc05::tma_load_2d(As + kABytes, &tmW, &full[s], tap * 16 * a.chunks + 16 * j, 0);
                    issued = it + 1;
                }
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- products
        if (lane == 0) {
            const uint32_t idesc = tc05::idesc_bf16(128, N, 0);
            int it = 0;
            for (int t = 0; t < my_tiles && !abort_flag; ++t) {
                const int b = t & 1;
                // the epilogue of tile t - 2 has read this accumulator
                if (t >= 2 &&
                    !tc05::mbar_wait(&acc_empty[b], (uint32_t)((t >> 1) - 1) & 1u, a.budget)) {
                    atomicOr(&g_conv_tc_err, 2);
                    abort_flag = 1;
                    break;
                }
                tc05::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * N);
                bool ok = true;
                for (int st = 0; st < steps; ++st, ++it) {
                    const int s = it % kStages, round = it / kStages;
                    if (!tc05::mbar_wait(&full[s], (uint32_t)round & 1u, a.budget)) {
                        ok = false;
                        break;
                    }
                    tc05::fence_after_sync();
                    const uint32_t as = tc05::smem_addr(smem + (size_t)s * kStage);
                    tc05::mma_ss(d, desc_sw32(as), desc_sw32(as + kABytes), idesc, st > 0 ? 1u : 0u);
                    tc05::mma_commit(&empty[s]);          // frees the stage once read
                    committed = it + 1;
                }
                if (!ok) {
                    atomicOr(&g_conv_tc_err, 4);
                    abort_flag = 1;
                    break;
                }
                tc05::mma_commit(&acc_full[b]);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        for (int t = 0; t < my_tiles; ++t) {
            const int b = t & 1;
            bool ok = tc05::mbar_wait(&acc_full[b], (uint32_t)(t >> 1) & 1u, a.budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicOr(&g_conv_tc_err, 8);
                abort_flag = 1;
                break;
            }
            tc05::fence_after_sync();
            const int tile = (int)blockIdx.x + t * (int)gridDim.x;
            const size_t v = (size_t)tile * 128 + 32 * warp + lane;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t r[16];
                tc05::tmem_ld16(lane_base + (uint32_t)(b * N + c0), r);
                tc05::tmem_wait_ld();
                float f[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    f[i] = __uint_as_float(r[i]) + s_bias[c0 + i];
                    if (a.relu) f[i] = fmaxf(f[i], 0.f);
                }
                if (a.Cout < N) {
                    // fewer real output channels than the MMA's N (the head):
                    // the weight rows past Cout were zero-filled by the copy
                    for (int i = 0; i < 16 && c0 + i < a.Cout; ++i) {
                        if (OUT_BF16)
                            reinterpret_cast<__nv_bfloat16 *>(out)[v * a.Cout + c0 + i] =
                                __float2bfloat16(f[i]);
                        else
                            reinterpret_cast<float *>(out)[v * a.Cout + c0 + i] = f[i];
                    }
                } else if (OUT_BF16) {
                    uint32_t p[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                        p[i] = *reinterpret_cast<uint32_t *>(&h);
                    }
                    uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(out) +
                                                         v * N + c0);
                    o[0] = make_uint4(p[0], p[1], p[2], p[3]);
                    o[1] = make_uint4(p[4], p[5], p[6], p[7]);
                } else {
                    float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + v * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        o[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
                }
            }
            // the accumulator is free for tile t + 2
            tc05::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&acc_empty[b]);
        }
    }
    // before shared and tensor memory are released: every copy issued has
    // landed and every product issued has completed (only the last stages can
    // be outstanding after an expired wait; waiting again on a completed
    // phase returns at once)
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 4 && lane == 0)
        for (int it = issued > kStages ? issued - kStages : 0; it < issued; ++it)
            tc05::mbar_wait(&full[it % kStages], (uint32_t)(it / kStages) & 1u, a.budget);
    if (warp == 5 && lane == 0 && committed > 0)
        tc05::mbar_wait(&empty[(committed - 1) % kStages],
                        (uint32_t)((committed - 1) / kStages) & 1u, a.budget);
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

template <int N, bool OUT_BF16>
cudaError_t launch_n(const CUtensorMap &tx, const CUtensorMap &tw, const float *bias, void *out,
                     const ConvTcArgs &a, cudaStream_t st) {
    auto kern = k_conv3d_tc<N, OUT_BF16>;
    const size_t smem = 1024 + (size_t)kStages * (kABytes + N * 32);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    // all of the unified L1 / shared storage as shared memory, so that several
    // blocks share an SM (their copies and products overlap)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0, smem_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    // blocks per SM: the occupancy limit, at least what shared memory allows
    // (1 KB of static shared memory and 1 KB the system reserves per block),
    // and at most what tensor memory allows (512 columns per SM)
    const int cols = 2 * N < 32 ? 32 : 2 * N;
    const int by_smem = smem_sm / (int)(smem + 2048);
    per_sm = per_sm < by_smem ? by_smem : per_sm;
    per_sm = per_sm < 1 ? 1 : per_sm;
    if (per_sm > 2048 / kThreads) per_sm = 2048 / kThreads;
    if (per_sm * cols > 512) per_sm = 512 / cols;
    const int grid = a.tiles < sms * per_sm ? a.tiles : sms * per_sm;
    kern<<<grid, kThreads, smem, st>>>(tx, tw, bias, out, a);
    return cudaGetLastError();
}

}  // namespace

bool nn_conv3d_tc_supported(int D, int H, int W, int Cin, int Cout, const void *x, const void *w,
                            const void *out) {
    const bool w_ok = W == 16 || W == 32 || W == 64 || W == 128;
    return Cin % 16 == 0 && Cin >= 16 && ((Cout >= 1 && Cout <= 16) || Cout == 32 || Cout == 64 || Cout == 128) &&
           w_ok && H % (128 / W) == 0 && D >= 1 && ((uintptr_t)x % 16) == 0 &&
           ((uintptr_t)w % 16) == 0 && ((uintptr_t)out % 16) == 0 && encode_fn() != nullptr;
}

cudaError_t nn_conv3d_tc(const void *x, const void *w, const float *bias, void *out, int D, int H,
                         int W, int Cin, int Cout, int Kp, int relu, int out_bf16,
                         cudaStream_t st) {
    if (!nn_conv3d_tc_supported(D, H, W, Cin, Cout, x, w, out)) return cudaErrorNotSupported;
    EncodeTiledFn enc = encode_fn();
    CUtensorMap tx{}, tw{};
    {
        const cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
        const cuuint64_t strides[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2,
                                       (cuuint64_t)H * W * Cin * 2};
        const cuuint32_t box[4] = {16, (cuuint32_t)W, (cuuint32_t)(128 / W), 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(x), dims, strides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // a box of N rows (N = Cout, or 16 for fewer channels: the rows past
        // Cout are out of bounds and land as zeros)
        const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Cout};
        const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
        const cuuint32_t box[2] = {16, (cuuint32_t)(Cout < 16 ? 16 : Cout)};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(w), dims, strides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    ConvTcArgs a{};
    a.tiles = D * H * W / 128;
    a.tiles_per_z = H * W / 128;
    a.bh = 128 / W;
    a.chunks = Cin / 16;
    a.relu = relu;
    a.Cout = Cout;
    a.budget = 4ll << 30;
    switch (Cout < 16 ? 16 : Cout) {
        case 16: return out_bf16 ? launch_n<16, true>(tx, tw, bias, out, a, st)
                                 : launch_n<16, false>(tx, tw, bias, out, a, st);
        case 32: return out_bf16 ? launch_n<32, true>(tx, tw, bias, out, a, st)
                                 : launch_n<32, false>(tx, tw, bias, out, a, st);
        case 64: return out_bf16 ? launch_n<64, true>(tx, tw, bias, out, a, st)
                                 : launch_n<64, false>(tx, tw, bias, out, a, st);
        default: return out_bf16 ? launch_n<128, true>(tx, tw, bias, out, a, st)
                                 : launch_n<128, false>(tx, tw, bias, out, a, st);
    }
}
