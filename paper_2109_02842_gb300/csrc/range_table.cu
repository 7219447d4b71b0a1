// Range-profile table, step (8a) / (19a) of the paper, per (channel, k_z bin):
//
//   b_i = sum_m S[c][u][m] alpha[u][m] e^{j theta_um (i - L/2)},  i < L
//
// where alpha folds the per-(k_z, f) compensation (the k weight of Eq. 7, the
// evanescent mask, the kernel deconvolution 1/phihat and the range-origin
// phase) and theta_um = kappa''_um h (see setup.cu). This is a type-1
// nonuniform FFT: the M sources are spread with an ES kernel onto a periodic
// fine grid of `fine` points in shared memory (one 8-lane group per bin, a
// lane per tap, the sources in a fixed order: no atomics, so the table does
// not depend on scheduling), transformed by a mixed-radix FFT in shared
// memory, and divided by the spreading kernel's transform.
//
// A block covers UB consecutive k_z bins of one channel: their fine grids are
// the rows of a [UB][fine] array in shared memory (bin-major, so the atomics
// of a bin's row hit neighbouring banks), transformed
// together by the block-wide mixed-radix Stockham FFT, and the deconvolved
// rows j = i - L/2 are written as coalesced rows of the table b[c][i][u]
// (u fastest; planar pairs {re_u, re_u+1, im_u, im_u+1} for the FP32
// back-projection, BF16 hi/lo planes of (re_u, im_u) columns for the tensor-core
// one).
#include "rt_body.cuh"

namespace {

using rt::bins_per_block;

template <int UB>
__global__ void __launch_bounds__(256)
k_range_table(NufftDesc d, FftPlan fp, const float2 *__restrict__ S,
              const float2 *__restrict__ alpha, const float *__restrict__ xg,
              const float *__restrict__ dec, const float2 *__restrict__ tw_g,
              void *__restrict__ table, int fmt) {
    extern __shared__ float2 smem[];
    rt::rt_block<UB>(d, fp, S, alpha, xg, dec, tw_g, table, fmt, blockIdx.y, blockIdx.x, smem);
}

}  // namespace

size_t range_table_smem_bytes(const NufftDesc &d) {
    return rt::smem_bytes(d.fine, bins_per_block(d.fine), d.n_f);
}

template <int UB>
cudaError_t launch_ub(const NufftDesc &d, const FftPlan &fp, const float2 *S, const float2 *alpha,
                      const float *xg, const float *dec, const float2 *tw_fine, void *table,
                      int fmt, cudaStream_t st) {
    const size_t smem = range_table_smem_bytes(d);
    cudaError_t e = cudaFuncSetAttribute(k_range_table<UB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((d.n_pad + UB - 1) / UB, d.n_chan);
    k_range_table<UB><<<grid, 256, smem, st>>>(d, fp, S, alpha, xg, dec, tw_fine, table, fmt);
    return cudaGetLastError();
}

cudaError_t launch_range_table(const NufftDesc &d, const FftPlan &fp, const float2 *S,
                               const float2 *alpha, const float *xg, const float *dec,
                               const float2 *tw_fine, void *table, int fmt, cudaStream_t st) {
    switch (bins_per_block(d.fine)) {
        case 16: return launch_ub<16>(d, fp, S, alpha, xg, dec, tw_fine, table, fmt, st);
        case 8: return launch_ub<8>(d, fp, S, alpha, xg, dec, tw_fine, table, fmt, st);
        default: return launch_ub<4>(d, fp, S, alpha, xg, dec, tw_fine, table, fmt, st);
    }
}
