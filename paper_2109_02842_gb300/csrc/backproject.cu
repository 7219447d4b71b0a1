// Back-projection, step (8b) / (19b) of the paper, with the coherent sum over
// every channel (all sections) and the k_z tile of one block:
//
//   G_u(x,y) = sum_c  e^{j kappa_T a_c(x,y)}  sum_{t<w} phi(a_c - l_{i0+t}) b_c[i0+t][u]
//
// a_c = rho (monostatic) or rho_T + rho_R (multistatic), phi the ES kernel on
// the table grid l_i = l0 + i h (setup.cu explains the factorisation; the
// table already carries the factor h), kappa_T the band centre of the block's
// UT bins (the range table is built about it for each of them).
//
// Block = (16 PX) x 16 pixels x UT consecutive k_z bins; thread = PX
// x-adjacent pixels with their UT bins in registers. With PX = 2 the two
// pixels' table windows differ by at most one row (the plan checks that the
// range step between neighbours is below h), so the thread loads w + 1 taps
// once per bin pair and uses them for both pixels: 1.75 instead of 3 shared
// 128-bit loads per update, which is what bounds this kernel (each such load
// costs a warp four shared-memory wavefronts). Channels are processed in chunks of CC, with the
// table window of chunk k+1 copied into shared memory (cp.async, double
// buffered) while chunk k is computed. Per chunk:
//  * the plan-time geometry of (tile, channel) gives the range a* of the tile
//    centre as a float pair and the first row i_lo of the R-row window;
//  * phi_c = kappa_T a* mod 2 pi is formed once per (block, channel) as a
//    float-float product with a two-constant reduction (Dekker / Cody-Waite;
//    phases reach ~2e3 rad, the result is good to ~3e-7 rad);
//  * per pixel: delta = a - a* in FP32 without cancellation (difference of
//    squares against the tile centre), tap weights from per-tap polynomials
//    of the ES kernel (fitted at plan time), the carrier
//    e^{j (kappa_T delta + phi_c)} (|arg| < ~70 rad, one FP32 sin/cos pair for
//    all bins), then for each pair of bins: w 128-bit shared loads, the
//    interpolation and the complex multiply-accumulate, as packed FP32x2
//    operations.
//
// The table holds bins in planar pairs {re_u, re_u+1, im_u, im_u+1}, so one
// shared load feeds two bins and the complex multiply-accumulate needs no
// shuffles: with X = (re_u, re_u+1), Y = (im_u, im_u+1) interpolated and
// C, S the cosine and sine of the carrier, Re += X.C - Y.S and
// Im += X.S + Y.C as four FP32x2 FMAs into two FP32x2 accumulators.
#include "bp_body.cuh"

namespace {

using bp::TX;
using bp::TY;
using bp::BpSmem;

template <int UT, int W, int CC, int MINB, int PX>
__global__ void __launch_bounds__(TX * TY, MINB)
k_backproject(BpDesc p, CoefTable ct, const void *__restrict__ table,
              const TileGeo *__restrict__ tgeo, const float2 *__restrict__ kc_hl,
              float2 *__restrict__ G) {
    extern __shared__ float4 smem4[];
    bp::bp_tile<UT, W, CC, PX>(p, ct, table, tgeo, kc_hl, G, blockIdx.x, blockIdx.y, blockIdx.z,
                               gridDim.x, smem4);
}

template <int UT, int W, int CC, int MINB, int PX>
cudaError_t launch_t(const BpDesc &p, const CoefTable &ct, const void *table, const TileGeo *tgeo, const float2 *kc_hl,
                     float2 *G, cudaStream_t st) {
    const size_t smem = BpSmem<UT, W, CC>::bytes(p.R, p.n_chan, p.bf16);
    cudaError_t e = cudaFuncSetAttribute(k_backproject<UT, W, CC, MINB, PX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + TX * PX - 1) / (TX * PX), (p.ny + TY - 1) / TY, (p.n_pad + UT - 1) / UT);
    k_backproject<UT, W, CC, MINB, PX><<<grid, TX * TY, smem, st>>>(p, ct, table, tgeo,
                                                                        kc_hl, G);
    return cudaGetLastError();
}

// Block configurations: k_z bins per block (UT), channels per staged chunk
// (CC), resident blocks per SM (MINB) and pixels per thread (PX).
//   block_config 1: CC = 8,  3 blocks/SM (80 registers per thread), PX = 1
//   block_config 2: CC = 16, 2 blocks/SM (128 registers per thread), PX = 1
//   block_config 3: CC = 8,  2 blocks/SM, PX = 2 (two pixels share the taps)
template <int UT, int CC, int MINB, int PX>
cudaError_t launch_w(const BpDesc &p, const CoefTable &ct, const void *table, const TileGeo *tgeo, const float2 *kc_hl,
                     float2 *G, cudaStream_t st) {
    switch (p.w) {
        case 4: return launch_t<UT, 4, CC, MINB, PX>(p, ct, table, tgeo, kc_hl, G, st);
        case 6: return launch_t<UT, 6, CC, MINB, PX>(p, ct, table, tgeo, kc_hl, G, st);
        case 8: return launch_t<UT, 8, CC, MINB, PX>(p, ct, table, tgeo, kc_hl, G, st);
        case 10: return launch_t<UT, 10, 8, 2, 1>(p, ct, table, tgeo, kc_hl, G, st);
        case 12: return launch_t<UT, 12, 8, 2, 1>(p, ct, table, tgeo, kc_hl, G, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int UT>
cudaError_t launch_u(const BpDesc &p, const CoefTable &ct, const void *table, const TileGeo *tgeo, const float2 *kc_hl,
                     float2 *G, cudaStream_t st) {
    if (p.block_config == 2) return launch_w<UT, 16, 2, 1>(p, ct, table, tgeo, kc_hl, G, st);
    if (p.block_config == 3) return launch_w<UT, 8, 2, 2>(p, ct, table, tgeo, kc_hl, G, st);
    return launch_w<UT, 8, 3, 1>(p, ct, table, tgeo, kc_hl, G, st);
}

}  // namespace

int backproject_tile_x(int block_config) { return block_config == 3 ? 2 * TX : TX; }
int backproject_tile_y() { return TY; }

size_t backproject_smem_bytes(int R, int tile_u, int n_chan, int bf16, int block_config) {
    const int CC = block_config == 2 ? 16 : 8;   // configs 1 and 3 stage 8 channels
    const int np = tile_u / 2;
    size_t s = 2 * (size_t)CC * R * (np + 1) * sizeof(float4);
    if (bf16) s += 2 * (size_t)CC * R * np * sizeof(uint2);
    s += 2 * (size_t)CC * sizeof(TileGeo) + (size_t)CC * np * sizeof(float4);
    s += (size_t)n_chan * sizeof(int);
    return s;
}

cudaError_t launch_backproject(const BpDesc &p, const CoefTable &ct, const void *table, const TileGeo *tgeo,
                               const float2 *kc_hl, float2 *G, cudaStream_t st) {
    switch (p.tile_u) {
        case 8: return launch_u<8>(p, ct, table, tgeo, kc_hl, G, st);
        case 16: return launch_u<16>(p, ct, table, tgeo, kc_hl, G, st);
        case 20: return launch_u<20>(p, ct, table, tgeo, kc_hl, G, st);
        case 24: return launch_u<24>(p, ct, table, tgeo, kc_hl, G, st);
        default: return cudaErrorInvalidValue;
    }
}
