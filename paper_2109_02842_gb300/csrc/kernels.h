// Launch wrappers of the CUDA kernels (internal to libpolyline).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

// ---- zfft.cu ---------------------------------------------------------------
size_t fft_strided_smem_bytes(int n);
cudaError_t launch_fft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               const FftPlan &plan, const float2 *tw, int sgn, float scale,
                               int out_rows, int out_off, cudaStream_t st,
                               void *split_A = nullptr, int split_Kp = 0,
                               const float2 *in2 = nullptr, int ld = 0, int bf16_out = 0);
// (ld: row stride in elements, 0 = I; a launch may cover columns [0, I) of
// wider rows, the pointers offset by the first column)
// in2 (optional): a second input of the same shape, added to `in` on load
cudaError_t launch_dft_strided(const float2 *in, float2 *out, int batch, int n_in, int I,
                               int out_rows, const float2 *T, float scale, cudaStream_t st,
                               const float2 *in2 = nullptr, int bf16_out = 0);

// Status bit a kernel sets in the plan's mapped status word when the echo
// holds NaN or Inf (the tensor-core kernels' expired waits use bits 0..5).
constexpr int PL_FLAG_NONFINITE = 1 << 20;
// Sets PL_FLAG_NONFINITE in *flag if any of the n complex values is NaN or Inf
// (a test of the exponent bits; one read of the buffer).
cudaError_t launch_check_finite(const float2 *x, size_t n, int *flag, cudaStream_t st);

// ---- zidft_tc.cu -----------------------------------------------------------
// Inverse z transform at off-grid heights on the tensor cores: image[z][p] =
// sum_u T[z][u] (G[u][p] + G2[u][p]), T from a BF16 hi/lo table (scale folded in).
struct ZidftTcArgs {
    int n_in;          // N_p: rows (bins) of G
    int ksteps;        // ceil(n_in / 16)
    int n_cols;        // columns (pixels) of G and of the image
    int ld, out_ld;    // row strides of G and of the image, elements
    int nz;            // output heights
    int nzc;           // heights per block (the MMA's N, multiple of 16, <= 96)
    int zchunks;       // ceil(nz / nzc)
    int nzp;           // table rows per plane (zchunks nzc)
    int plane_bytes;   // shared memory of one plane of a stage
    long long budget;  // wait budget, SM clock cycles
    int dbg_wait;      // test hook: the MMA warp first waits on a barrier nothing completes
};
typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
ZidftTcArgs zidft_tc_shape(int n_in, int n_cols, int nz);
size_t zidft_tc_table_elems(const ZidftTcArgs &a);       // BF16 elements of the table
cudaError_t launch_zidft_tc_table(const ZidftTcArgs &a, const float2 *T, float scale,
                                  __nv_bfloat16 *tb, cudaStream_t st);
bool zidft_tc_make_map(const ZidftTcArgs &a, const __nv_bfloat16 *tb, CUtensorMap *map,
                       TmapEncodeFn enc);
size_t zidft_tc_smem_bytes(const ZidftTcArgs &a);
cudaError_t launch_zidft_tc(const ZidftTcArgs &a, const CUtensorMap *map, const float2 *G,
                            const float2 *G2, float2 *out, int *err, cudaStream_t st);

// ---- setup.cu --------------------------------------------------------------
// Per k_z bin: kappa range over propagating frequencies; kc = centre (double
// and as a float pair hi + lo), kspan = kappa_max - kappa_min (0 when every
// frequency is evanescent). With group > 1 the range is taken over the group
// of bins [group floor(u / group), + group) and every bin of it gets the
// group's centre and span. band: scratch of 2 n_pad doubles (each bin's own
// kappa range, the first pass).
cudaError_t launch_setup_kz(int mode, int n_pad, double dz, int n_f, const double *k, int group,
                            double *band, double *kc, float2 *kc_hl, double *kspan,
                            cudaStream_t st);
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
// tw_fine: exp(-2 pi i k / fine), k < fine; fp: radix plan of `fine`.
cudaError_t launch_range_table(const NufftDesc &d, const FftPlan &fp, const float2 *S,
                               const float2 *alpha, const float *xg, const float *dec,
                               const float2 *tw_fine, void *table, int fmt, cudaStream_t st);

// ---- backproject.cu ------------------------------------------------------------
// Plan-time geometry of one (pixel tile, channel): offsets of the tile centre
// from the Tx / Rx position and their distances (FP32), the tile-centre range
// a* as a float pair, the first table row i_lo of the R-row window covering the
// tile, and off = a* - l_{i_lo}. 48 bytes (three 16-byte copies).
struct TileGeo {
    float dxt, dyt, rt, dxr;
    float dyr, rr, off, a_hi;
    float a_lo;
    int ilo;
    float pad0, pad1;
};
struct BpDesc {
    int mode, n_chan, n_pad, L, R;
    int nx, ny;
    double x0, dx, y0, dy;
    double h, l0;
    float inv_h;
    float dxf, dyf;       // dx, dy in FP32
    float beta, two_over_w;
    int w, tile_u;
    int block_config;     // 1: 8-channel chunks, 3 blocks/SM; 2: 16-channel chunks, 2 blocks/SM;
                          // 3: 8-channel chunks, 2 blocks/SM, two pixels per thread
    int tile_px;          // pixels per block along x (16 or 32)
    int tile_py;          // pixels per block along y (16, or 8 for block_config 4)
    int bf16;
};
// ES kernel tap weights as polynomials: weight_t(s) = sum_d c[t][d] s^d,
// s in (-1, 1] the offset of the pixel inside its first table cell.
struct CoefTable {
    float c[12][14];
};
size_t backproject_smem_bytes(int R, int tile_u, int n_chan, int bf16, int block_config);
cudaError_t launch_backproject(const BpDesc &p, const CoefTable &ct, const void *table,
                               const TileGeo *tgeo, const float2 *kc_hl, float2 *G,
                               cudaStream_t st);
cudaError_t launch_setup_tile_geo(const BpDesc &p, const double *ch_xy, TileGeo *tgeo,
                                  cudaStream_t st);
int backproject_tile_x(int block_config);
// tensor-core variant (block_config 4), backproject_tc.cu
struct TcArgs {
    int UT;              // k_z bins per block (the MMA's N: UT planar, 2 UT interleaved)
    int planar;          // 1: table rows [Re of every bin | Im of every bin], accumulators
                         //    Re G and Im G, 12 products per K step; 0: (re, im) pairs, P and Q
    int nsplit;          // channel parts per tile (blocks adding into G: 1 or 2)
    int im_col;          // planar: table column of the first Im entry
    unsigned im_off;     // planar: smem offset of a window's Im columns (ncb x cb_bytes)
    int ncb;             // 64-column blocks of a block's window: ceil(N / 64)
    int n_utiles;        // blocks along k_z
    int nst;             // table-window slots in shared memory (groups of npar x cpr)
    unsigned cb_bytes;   // one column block: planes x 16 ks rows x 128 B
    unsigned slot_bytes; // one channel's window: ncb x cb_bytes (x 2 planar)
    unsigned idesc;      // tcgen05 instruction descriptor
    int acol;            // first TMEM column of the A buffers (after P and Q)
    int tmem_cols;       // TMEM columns per block (256 or 512)
    int ks;              // 16-row K steps per channel (1 or 2)
    int split;           // 3: BF16 hi/lo products, 1: BF16 only
    int npar;            // channel classes of A-building warps (2: 2 blocks/SM, 3: 1 block/SM)
    int cpr;             // channels per class round (1, or 2 with npar 3): A buffers of cpr
                         // channels, one A-ready wait and one release per round
    long long budget;    // wait budget, SM clock cycles
    int dbg_wait;        // test hook: the MMA warp first waits on a barrier nothing
                         // completes, so the bounded-wait exit paths run
    int blk0, nblk;      // the launch's blocks: linear indices [blk0, blk0 + nblk) of
                         // (tile x, tile y, bin block x part), x fastest; nblk 0: to the end
    int sparse;          // 1: 2:4-sparse products (planar, 16-row windows, cpr 1): window rows
                         // taken in residue order, K = [Re rows; Im rows] of the table, six
                         // sparse products per channel (split 3); 5-D table map
    int mcol;            // sparse: first TMEM column of the classes' metadata (8 apart)
    int rw;              // sparse: window rows, 16 (residues mod 4) or 12 (mod 3, w <= 6;
                         // each window slot then ends in a 1 KB zero pad)
    int g_atomic;        // 1: the channel parts add their sums into one spectrum G
                         // (atomic adds onto a zeroed G: two terms per value, in either
                         // order the same sum); 0: part p writes spectrum p
};
// blocks of a whole back-projection
int backproject_tc_blocks(const BpDesc &p, const TcArgs &ta);
// One scene of a batch whose back-projections run as ONE persistent launch
// (every scene in the one-block-per-SM layout: npar 3, cpr 1, 512 TMEM
// columns; w = 6; one precision; the same tap polynomials).
struct TcScene {
    BpDesc bp;
    TcArgs ta;
    const TileGeo *tgeo;
    const float2 *kc_hl;
    float2 *G;
    int begin;           // the scene's first item in the work queue
    int nblk;            // its items (back-projection blocks)
};
constexpr int kTcBatchMaxScenes = 96;
// the scenes' table maps, a kernel parameter (TMA reads them from there)
struct TcBatchMaps {
    CUtensorMap m[kTcBatchMaxScenes];
};
// counters[0]: next item (zeroed before the launch); err: wait-expired bits
// (any set bit also stops the blocks from taking further items)
cudaError_t launch_backproject_tc_batch(const TcBatchMaps &maps, const CoefTable &ct,
                                        const TcScene *scenes, int n_scenes, int total, int split,
                                        int *counters, int *err, int grid, size_t smem,
                                        cudaStream_t st);
size_t backproject_tc_batch_smem_bytes(const TcArgs &ta);
int backproject_tc_tile_x();
int backproject_tc_tile_y();
size_t backproject_tc_smem_bytes(const TcArgs &ta);
cudaError_t launch_backproject_tc(const BpDesc &p, const CoefTable &ct, const TcArgs &ta,
                                  const CUtensorMap &tm, const TileGeo *tgeo, const float2 *kc_hl,
                                  float2 *G, int *err, cudaStream_t st);
// window of every (16 x 8 tile, channel): first row i_lo = the lowest first tap
// of its 128 pixels; stats[0] = max rows spanned, stats[1] = max i_lo
cudaError_t launch_setup_tile_geo_tc(const BpDesc &p, const double *ch_xy, TileGeo *tgeo,
                                     int *stats, cudaStream_t st);
int backproject_tile_y();

// ---- range_table_tc.cu: the range table as exact sums on the tensor cores ------
struct RtTcArgs {
    int C, Np, M;
    int Kp;              // frequencies rounded up to 64 (the K of the products)
    int natoms;          // Kp / 64
    int L, Lp;           // table rows; rounded up to 16
    int nh, Lh;          // row parts per bin (blocks along the rows) and rows per part,
                         // a multiple of 16 (the N of the products)
    unsigned idesc;      // tcgen05 instruction descriptor (M 128, N Lh, both K-major)
    long long budget;    // wait budget, SM clock cycles
    int grid;            // persistent blocks (one per SM)
    int a_hi_only;       // 1: the spectrum operand is BF16 (hi planes only): 8 products
                         // per K step instead of 12
    int dbg_wait;        // test hook: the first stage's operand wait is replaced by a
                         // wait on a barrier nothing completes
};
size_t range_table_tc_smem_bytes(const RtTcArgs &ra);
// E [N_p][re hi, re lo, im hi, im lo][Lp][Kp] BF16: alpha_um e^{+j theta_um (i - L/2)}
cudaError_t launch_setup_rt_E(const NufftDesc &d, double dz, const double *k, const double *kc,
                              const float2 *alpha, int Lp, int Kp, void *E, cudaStream_t st);
// S -> A (scratch [N_p][4][C][Kp] BF16; skipped when `prepared`: the
// z-FFT wrote A) -> prod (scratch [N_p][2][nh * Lh][C rounded up to 128] uint32) -> table
// [C][2][L][row_words uint32]
cudaError_t launch_range_table_tc(const RtTcArgs &ra, const CUtensorMap &tmA,
                                  const CUtensorMap &tmB, const float2 *S,
                                  void *A, void *prod, void *table, int row_words, int planar, int *err,
                                  bool prepared, cudaStream_t st);

// ---- comparison.cu: exact-sum hybrid and direct back-projection (Sec. III) ------
struct ExactDesc {
    int mode, n_chan, n_pad, n_f, nx, ny;
    double x0, dx, y0, dy;
};
struct DirectDesc {
    int mode, n_chan, n_scan, n_f, nx, ny, nz;
    int uniform;                    // evenly spaced band: rotation from k_0 by dk
    double x0, dx, y0, dy, z0, dz;
    float k0_hi, k0_lo, dk_hi, dk_lo;
};
// S [C][N_p][M]; kap [N_p][M] kappa as float pairs; wum [N_p][M] k_m or 0
// (evanescent); chff [C][2] float4 (xT hi, lo, yT hi, lo), (xR ..); G [N_p][ny][nx]
cudaError_t launch_exact_sum(const ExactDesc &e, const float2 *S, const float2 *kap,
                             const float *wum, const float4 *chff, float2 *G, cudaStream_t st);
// s [C][N][M] echo; zs [N] scan heights and kff [M] wavenumbers as float pairs;
// img [nz][ny][nx]
cudaError_t launch_bp_direct(const DirectDesc &e, const float2 *s, const float4 *chff,
                             const float2 *zs, const float2 *kff, float2 *img, cudaStream_t st);
// kap / wum of the exact sum, per (k_z bin, frequency)
cudaError_t launch_setup_exact(int mode, int n_pad, double dz, int n_f, const double *k,
                               float2 *kap, float *wum, cudaStream_t st);

// ---- plan.cu: error reporting for other translation units ----------------------
#include "../../include/polyline.h"
pl_status pl_internal_fail(pl_status s, const char *msg);
pl_status pl_internal_cuda_fail(cudaError_t e, const char *where);

// ---- synth.cu ----------------------------------------------------------------
// device arrays in the caller's FP64 layouts: tx_xy, rx_xy [n_chan][2], f_hz [n_f],
// pts [n_pts][3], amp [n_pts][2]
cudaError_t launch_synth_echo(int n_chan, const double *tx_xy, const double *rx_xy, int n_scan,
                              double z0, double dz, int n_f, const double *f_hz, int n_pts,
                              const double *pts, const double *amp, float2 *echo,
                              cudaStream_t st);

// ---- nn_tc.cu: the convolution on the tensor cores (tcgen05) -------------------
bool nn_conv3d_tc_supported(int D, int H, int W, int Cin, int Cout, const void *x, const void *w,
                            const void *out);
cudaError_t nn_conv3d_tc(const void *x, const void *w, const float *bias, void *out, int D, int H,
                         int W, int Cin, int Cout, int Kp, int relu, int out_bf16,
                         cudaStream_t st);

// ---- nn.cu: learned fast path -------------------------------------------------
cudaError_t nn_conv3d(const void *x, const void *w, const float *bias, void *out, int D, int H,
                      int W, int Cin, int Cout, int Kp, int relu, int out_bf16, cudaStream_t st);
size_t nn_wgrad_work_floats(int D, int H, int W, int Cin, int Cout, int Kp);
cudaError_t nn_conv3d_wgrad(const void *x, const void *gy, float *gw, float *gb, float *work,
                            int D, int H, int W, int Cin, int Cout, int Kp, cudaStream_t st);
cudaError_t nn_check(const float *corr, const void *img, const float *scale, float gain, size_t n,
                     float *out, cudaStream_t st);
cudaError_t nn_residual(float *pred, const void *img, const float *scale, float gain, size_t n,
                        cudaStream_t st);
cudaError_t nn_weight_flip(const void *w, void *wt, int Cin, int Cout, int Kp, int Kpt,
                           cudaStream_t st);
cudaError_t nn_elementwise(int op, const void *a, const void *b, void *out, size_t n,
                           cudaStream_t st);
cudaError_t nn_resample(int op, const void *x, void *y, int D, int H, int W, int C, cudaStream_t st);
cudaError_t nn_features(const void *img, void *feat, float *scale, size_t n, cudaStream_t st);
cudaError_t nn_loss(const float *pred, const void *target, const float *scale, float *sums,
                    float *grad, size_t n, cudaStream_t st);
cudaError_t nn_to_complex(const float *pred, const float *scale, void *img, size_t n,
                          cudaStream_t st);
cudaError_t nn_adam(float *p, const float *g, float *m, float *v, void *pb, size_t n, float lr,
                    float b1, float b2, float eps, int step, cudaStream_t st);
