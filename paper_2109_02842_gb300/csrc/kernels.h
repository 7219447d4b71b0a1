// Launch wrappers of the CUDA kernels (internal to libpolyline).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

// ---- zfft.cu ---------------------------------------------------------------
size_t fft_strided_smem_bytes(int n);
cudaError_t launch_fft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               const FftPlan &plan, const float2 *tw, int sgn, float scale,
                               int out_rows, int out_off, cudaStream_t st);
cudaError_t launch_dft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               int out_rows, const float2 *T, float scale, cudaStream_t st);

// ---- setup.cu --------------------------------------------------------------
// Per k_z bin: kappa range over propagating frequencies; kc = centre (double),
// kspan = kappa_max - kappa_min (0 when every frequency is evanescent).
cudaError_t launch_setup_kz(int mode, int n_pad, double dz, int n_f, const double *k,
                            double *kc, float *kc_f, double *kspan, cudaStream_t st);
// Per (k_z, f): spreading position (fine cells) and source factor alpha.
cudaError_t launch_setup_sources(const NufftDesc &d, double dz, const double *k,
                                 const double *kc, const double *gl_x, const double *gl_w,
                                 int n_gl, float *xg, float2 *alpha, cudaStream_t st);
// Type-1 deconvolution factors for table rows i < L.
cudaError_t launch_setup_deconv(const NufftDesc &d, const double *gl_x, const double *gl_w,
                                int n_gl, float *dec, cudaStream_t st);
// out[k] = exp(sgn 2 pi i k / n), k < count.
cudaError_t launch_twiddles(int n, int count, int sgn, float2 *out, cudaStream_t st);
// Phase matrix of the zero-padded forward DFT: T[u][n] = exp(-2 pi i (u n mod Np) / Np).
cudaError_t launch_dft_matrix_fwd(int n_pad, int n_scan, float2 *T, cudaStream_t st);
// Phase matrix of the z inverse transform onto voxel heights:
// T[p][u] = exp(+i kz_u (z_p - z0_scan)), z_p = zv0 + p dzv.
cudaError_t launch_dft_matrix_inv(int n_pad, double dz, double z0_scan, int nz, double zv0,
                                  double dzv, float2 *T, cudaStream_t st);

// ---- range_table.cu ----------------------------------------------------------
size_t range_table_smem_bytes(const NufftDesc &d);
cudaError_t launch_range_table(const NufftDesc &d, const float2 *S, const float2 *alpha,
                               const float *xg, const float *dec, const float2 *tw_fine,
                               void *table, int bf16, cudaStream_t st);

// ---- backproject.cu ------------------------------------------------------------
struct BpDesc {
    int mode, n_chan, n_pad, L, R;
    int nx, ny;
    double x0, dx, y0, dy;
    double h, l0;
    float inv_h;
    float beta, two_over_w;
    int w, tile_u;
    int bf16;
};
cudaError_t launch_backproject(const BpDesc &p, const void *table, const double *ch_xy,
                               const double *kc, const float *kc_f, float2 *G, cudaStream_t st);
int backproject_tile_x();
int backproject_tile_y();

// ---- synth.cu ----------------------------------------------------------------
cudaError_t launch_synth_echo(int n_chan, const float4 *ch, int n_scan, float z0, float dz,
                              int n_f, const float *k, int n_pts, const float4 *pts,
                              const float2 *amp, float2 *echo, cudaStream_t st);
