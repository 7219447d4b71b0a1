/*
 * polyline.h -- C ABI of the GB300 (sm_103a) hybrid 3-D reconstruction for
 * mechanically scanned polyline arrays.
 *
 * Method: Wang, Li, Zhao, Sun, "Near-Field Millimeter-Wave Imaging via Arrays
 * in the Shape of Polyline" (arXiv 2109.02842), Sec. II. Equation numbers are
 * the paper's printed numbering: (1) monostatic echo, (2) FT over the scan
 * axis, (5) monostatic dispersion, (7) time-domain inversion, (8a)/(8b)
 * filtered back-projection with an inverse NUFFT, (9) inverse FFT over k_z,
 * (10) multistatic echo, (18) multistatic dispersion, (19a)/(19b)
 * multistatic filtered back-projection.
 *
 * Problem statement (Sec. II-A/B): array geometry (circle radius, section
 * count, chord length, element positions), scan positions, frequency samples
 * and complex echoes in; a complex 3-D image out.
 *
 * Conventions for every call:
 *  - Every call returns a pl_status; nothing throws across the ABI. On an
 *    error, pl_last_error() returns a message for the calling thread.
 *  - Complex data are interleaved single precision (re, im) = 8 bytes, C order.
 *  - "device" pointers are CUDA global-memory pointers on the current device
 *    (e.g. a torch tensor's data_ptr()); "host" pointers are CPU memory.
 *  - The caller owns echo and image buffers. A plan owns its workspace and
 *    copies the geometry, scan, frequency and grid descriptions at creation.
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy default).
 *  - A plan is not thread-safe: one execute at a time per plan.
 *  - There is no CPU fallback: without a usable CUDA device every compute
 *    call fails with PL_ERR_CUDA.
 */
#ifndef POLYLINE_H
#define POLYLINE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PL_OK = 0,
    PL_ERR_ARG = 1,          /* NULL pointer, bad size or bad option */
    PL_ERR_GEOMETRY = 2,     /* element/pair indices or positions invalid */
    PL_ERR_FREQ = 3,         /* frequencies not finite, positive, strictly ascending */
    PL_ERR_EVANESCENT = 4,   /* every (k_z, f) term is evanescent */
    PL_ERR_NONFINITE = 5,    /* NaN/Inf in an input description */
    PL_ERR_CUDA = 6,         /* a CUDA runtime call or kernel failed */
    PL_ERR_OOM = 7,          /* device allocation failed */
    PL_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
    PL_ERR_UNSUPPORTED = 9   /* valid request this build does not support */
} pl_status;

/* Array topology, Sec. II-A (monostatic) and II-B (multistatic), Fig. 1.
 * mode 0: one channel per element, Tx = Rx at elem_xy[c]; echo model Eq. (1).
 * mode 1: one channel per (Tx, Rx) pair, pair c uses elem_xy[pair_tx[c]] and
 *         elem_xy[pair_rx[c]]; echo model Eq. (10). Pairs may be any subset
 *         (the paper pairs within a section, Sec. III).
 * radius, n_sections, chord_len describe the polyline (informational; the
 * element positions are authoritative). All arrays are host memory and are
 * copied by pl_plan_create. elem_section may be NULL. */
typedef struct {
    int mode;
    double radius;
    int n_sections;
    double chord_len;
    int n_elem;
    const double *elem_xy;      /* host [n_elem][2], metres */
    const int *elem_section;    /* host [n_elem] or NULL */
    int n_pairs;                /* mode 1 only */
    const int *pair_tx;         /* host [n_pairs], mode 1 only */
    const int *pair_rx;         /* host [n_pairs], mode 1 only */
} pl_geometry;

/* Mechanical scan along z (Sec. II-A): z'_n = z0 + n*dz, n < n.
 * n_pad: length N_p >= n of the zero-padded transform over z (Eq. 2);
 * 0 selects n. The image is periodic in z with period N_p*dz. */
typedef struct {
    double z0;
    double dz;
    int n;
    int n_pad;
} pl_scan;

/* Frequency samples f_m (Hz), finite, positive, strictly ascending. k_0 of
 * Eq. (8a) is the wavenumber of f_hz[0]. Host memory, copied. */
typedef struct {
    const double *f_hz;
    int n;
} pl_freqs;

/* Voxel centres x0 + i*dx (i < nx), y0 + j*dy, z0 + p*dz. The image is
 * complex64 [nz][ny][nx]. When z0 = scan.z0 + q*scan.dz for an integer q,
 * dz = scan.dz and q + nz <= N_p, the z inverse transform is an FFT;
 * otherwise it is an explicit DFT onto the voxel heights (Eq. 9). */
typedef struct {
    double x0, dx;
    double y0, dy;
    double z0, dz;
    int nx, ny, nz;
} pl_grid;

/* Numerical options. Zero-initialise and set what you need.
 * precision: 0 = FP32 everywhere (default);
 *            1 = range-profile table stored as BF16 pairs (FP32 accumulate);
 *            2 = as 1, and the spectrum S of Eq. (2) stored in BF16 as well
 *                (FP32 kernels: S as bfloat16 (re, im) pairs; block_config 4:
 *                the exact-sum range table takes the spectrum's BF16 part
 *                only, two products per real product instead of three).
 * nufft_sigma: oversampling of the range-profile grid (default 2.0).
 * nufft_w: interpolation taps (even, 4..12; default 6).
 * tile_u: k_z bins per back-projection block (8, 16, 20 or 24; with
 *         block_config 4 a multiple of 8 in 16..112, which selects the
 *         interleaved layout below; 0 = chosen from n_pad).
 * block_config: back-projection kernel (0 = default: 4 when nufft_w is 4, 6
 *         or 8, tile_u is 0 and the grid allows it, else 3 when the x step is
 *         below the table step, else 1; 1 = FP32, one pixel per thread,
 *         8-channel chunks, 3 blocks per SM; 2 = FP32, one pixel per thread,
 *         16-channel chunks; 3 = FP32, two pixels per thread sharing the tap
 *         window; 4 = tensor cores (tcgen05): 16 x 8 pixels x tile_u bins per
 *         block, the channel sum accumulated in tensor memory, one band centre
 *         per block of bins, BF16 operands split hi + lo (precision 0) or BF16
 *         only (precision 1); needs nufft_w 4, 6 or 8. With 4 the range-table
 *         workspace holds [channel][hi/lo][row][column] BF16, hi = BF16(x),
 *         lo = BF16(x - hi): by default (tile_u = 0) planar, every bin in one
 *         block (tile_u = n_pad rounded up to 16), column u = Re b_u and
 *         column tile_u + u = Im b_u, and each tile's channels in two parts;
 *         where that does not fit tensor memory, or with an explicit tile_u,
 *         interleaved, column 2u + (re, im) within blocks of tile_u bins.
 *         A bounded device wait of block_config 4 that runs out makes the next
 *         pl_execute / pl_execute_host call return PL_ERR_TIMEOUT.) */
typedef struct {
    int precision;
    double nufft_sigma;
    int nufft_w;
    int tile_u;
    int block_config;
    /* Bounded waits of the tensor-core kernels (block_config 4):
     * wait_timeout_us = how long one wait may last before it gives up
     * (0 = about 2 s); debug_unsatisfiable (a test hook) = 1 makes the
     * back-projection's MMA warp, 2 the range-table kernel's first stage, 3
     * the MMA warp of the inverse z transform at off-grid heights, wait first
     * on a barrier nothing completes, so that the wait runs out
     * and the kernel takes its exit path (the next pl_execute returns
     * PL_ERR_TIMEOUT; no device fault, the context stays usable). */
    int debug_unsatisfiable;
    int wait_timeout_us;
    /* block_config 4: 1 = the one-block-per-SM layout (three channel classes,
     * one channel per round, 512 TMEM columns) whatever fits, the layout a
     * batch's persistent back-projection runs every scene in; 0 = chosen by
     * size (default). */
    int one_block_per_sm;
    /* check_nonfinite = 1: every execution first scans its echo for NaN or
     * Inf (one read of the echo on the device, a flag in mapped host memory).
     * pl_execute_host and pl_execute_host_stream then return
     * PL_ERR_NONFINITE from the call itself; pl_execute, which does not
     * synchronise, returns it from the next pl_execute / pl_execute_host call
     * on the plan (after pl_execute, synchronise the stream before relying on
     * that report). The image of an echo with such values is not defined.
     * 0 = no scan (default). */
    int check_nonfinite;
    /* debug_fail_alloc (a test hook) = n > 0: the n-th device allocation that
     * pl_plan_create makes for this plan fails as if the device were out of
     * memory, so that the call returns PL_ERR_OOM and frees what it had
     * allocated. 0 = off (default). */
    int debug_fail_alloc;
    /* block_config 4: by default the back-projection's products are 2:4
     * sparse (tcgen05.mma.sp) in the planar layout (16- and 32-row windows)
     * and in the interleaved layout (16-row windows with the hi/lo split,
     * 32-row windows). A window's rows are taken in residue order (K index
     * 4 j + e <-> row j + 4 e; over 32 rows 8 j + e), in which a pixel's w
     * consecutive taps leave at most two nonzeros in every group of four. The
     * K = 32 operand is the window's [Re rows; Im rows] (planar, 16 rows: six
     * sparse products per channel instead of twelve dense), its Re rows and
     * its Im rows (planar, 32 rows: twelve instead of 24), its [hi rows; lo
     * rows] (interleaved, 16 rows: four instead of six) or its 32 rows
     * (interleaved, 32 rows: six instead of twelve). The sums are the same up
     * to rounding order. dense_products = 1 keeps the dense products
     * (pl_info.sparse_products says which run). */
    int dense_products;
    /* The sparse products' window: 0 = 16 rows (default); 12 = 12 rows
     * (residues mod 3) where every tile's taps span at most 12 rows and
     * nufft_w <= 6, else 16. (12-row windows copy a quarter fewer table
     * bytes; on the full-size monostatic workload they are not faster.) */
    int sparse_window_rows;
    int reserved[1];
} pl_options;

typedef struct pl_plan pl_plan;

/* Read-only description of a plan (sizes a caller may need). */
typedef struct {
    int mode, n_chan, n_scan, n_pad, n_f;
    int nx, ny, nz;
    int table_len;        /* L: rows of the range-profile table */
    int fine_len;         /* n_f of the type-1 NUFFT grid */
    int slab_rows;        /* R: table rows a back-projection block stages */
    int nufft_w;
    double nufft_sigma;
    double table_h;       /* range step h of the table (m) */
    double table_l0;      /* range of table row 0 (m) */
    int z_transform_fft;  /* 1: z inverse transform is an FFT, 0: DFT */
    int launches_per_execute;
    size_t workspace_bytes;
    double updates_per_execute;  /* n_chan * nx * ny * nz * n_f */
    int block_config;            /* back-projection kernel in use (1..4) */
    int tile_u;                  /* its k_z bins per block (block_config 4: all
                                    n_pad, rounded up to 16, in the planar layout) */
    int bp_launches;             /* launches of the back-projection per execution:
                                    2 when its full waves and its last partial wave
                                    are separate launches (block_config 4, the
                                    z-IFFT of the pixels the full waves finished
                                    running beside the last wave), else 1 */
    /* The range table b of Eq. (8a)/(19a) (workspace PL_STAGE_RANGE_TABLE): row
     * i holds, for every k_z bin u, the type-1 NUFFT coefficients at range
     * l_i = table_l0 + i table_h,
     *   b_i(u) = table_h sum_m S_um k_m e^{j kappa''_um l_i} / phihat(kappa''_um),
     * kappa'' = kappa - kappa_c with kappa_c the centre of the band (live
     * kappa values) of the bin's group of band_group consecutive bins, and
     * phihat the Fourier transform of the ES kernel
     * ES(t) = exp(es_beta (sqrt(1 - (2t / nufft_w)^2) - 1)), |t| < nufft_w / 2.
     * The back-projection's interpolation sum_i ES((l - l_i) / table_h) b_i(u)
     * then approximates sum_m S_um k_m e^{j kappa''_um l}. */
    double es_beta;
    int band_group;
    int table_layout;     /* 0: float32 rows of bin pairs {re_u, re_u+1, im_u, im_u+1},
                             [n_chan][L][ceil(n_pad/2)]; 1: the same in bfloat16;
                             2: bfloat16 [n_chan][hi, lo][L][table_cols], column
                             2u + (re, im); 3: the same planar, column u = Re b_u,
                             column table_cols/2 + u = Im b_u (value = hi + lo) */
    int table_cols;       /* layouts 2 and 3: columns of a row */
    int table_exact;      /* 1: b evaluated as exact sums over the frequencies
                             (tensor cores); 0: type-1 NUFFT (spread, FFT,
                             deconvolution) */
    int precision;        /* pl_options.precision in use */
    int sparse_products;  /* 1: the tensor-core back-projection takes 2:4-sparse
                             products (see pl_options.dense_products) */
} pl_info;

/* Stage identifiers for timing and workspace access. */
enum {
    PL_STAGE_ZFFT = 0,        /* Eq. (2): transform over the scan axis */
    PL_STAGE_RANGE_TABLE = 1, /* Eq. (8a)/(19a): compensation + NUFFT spread + fine FFT */
    PL_STAGE_BACKPROJECT = 2, /* Eq. (8b)/(19b): interpolation + carrier + channel sum */
    PL_STAGE_ZIFFT = 3,       /* Eq. (9): inverse transform over k_z */
    PL_NUM_STAGES = 4
};
/* Further workspace identifiers for pl_plan_workspace (inspection only) of a
 * plan whose range table is evaluated as exact sums on the tensor cores
 * (pl_info.table_exact = 1), with Kp = n_f rounded up to 64 and Lp =
 * table_len rounded up to 16, all bfloat16:
 *  PL_WS_RT_OPERAND_A -> the spectrum operand [n_pad][re hi, re lo, im hi,
 *                        im lo][n_chan][Kp], S split as hi = BF16(S),
 *                        lo = BF16(S - hi) (lo planes unused with precision 2)
 *  PL_WS_RT_OPERAND_E -> the plan-time factor [n_pad][re hi, re lo, im hi,
 *                        im lo][Lp][Kp], E[u][i][m] = alpha_um
 *                        e^{j theta_um (i - L/2)}, b[c][i][u] = sum_m S E */
enum { PL_WS_RT_OPERAND_A = 16, PL_WS_RT_OPERAND_E = 17 };

/* Create a plan: validates the inputs, allocates device workspace on the
 * current device and precomputes the per-(k_z, f) tables on the GPU.
 * opt may be NULL for defaults. On success *out is a new plan. */
pl_status pl_plan_create(pl_plan **out, const pl_geometry *geom, const pl_scan *scan,
                         const pl_freqs *freqs, const pl_grid *grid, const pl_options *opt);

/* Reconstruct one scan. echo_dev: device complex64 [n_chan][n_scan][n_f]
 * (channel-major, frequency fastest); image_dev: device complex64
 * [nz][ny][nx]. Asynchronous on `stream`; the buffers must stay valid until
 * the stream reaches the end of this call's work. When the tensor-core
 * back-projection has a partial last wave (pl_info.bp_launches == 2), part of
 * the inverse z transform runs on a plan-owned stream beside it, forked from
 * and joined back into `stream` by events: the call's work stays ordered on
 * `stream` (also under stream capture). */
pl_status pl_execute(pl_plan *plan, const void *echo_dev, void *image_dev, void *stream);

/* Same reconstruction from HOST buffers: copies the echo to the device,
 * reconstructs, copies the image back and synchronises `stream` before
 * returning. Pinned host memory gives the fastest copies. */
pl_status pl_execute_host(pl_plan *plan, const void *echo_host, void *image_host,
                          void *stream);

/* A sequence of scans from HOST buffers, pipelined: echo_host[i] (complex64
 * [n_chan][n_scan][n_f]) -> image_host[i] (complex64 [nz][ny][nx]) for
 * i < n_scans, with the upload of scan i+1 and the download of scan i-1 on the
 * copy engines (two internal streams) while scan i is reconstructed on
 * `stream`. Each image is the one pl_execute gives for its echo. The first
 * call allocates a second pair of device staging buffers (workspace grows by
 * the echo and image sizes); the first call with two or more scans also
 * builds a second plan from the same inputs (its own workspace, so the
 * plan's device memory roughly doubles) that takes every other scan on an
 * internal stream, so that consecutive scans' kernels share the device.
 * Call it with the plan's device current. Synchronises `stream` before
 * returning; the host buffers should be pinned (pageable memory gives correct
 * results without the overlap). n_scans = 0 is a no-op; a NULL array or entry
 * is PL_ERR_ARG. */
pl_status pl_execute_host_stream(pl_plan *plan, int n_scans, const void *const *echo_host,
                                 void *const *image_host, void *stream);

/* Sampling and resolution design figures of Sec. II-C/D for an array, scan
 * and band (host computation, no device work):
 *   max_rx_spacing   = lambda_min sqrt((L_R + D)^2/4 + R_0^2) / (L_R + D), the
 *                      multistatic receive spacing limit; max_elem_spacing is
 *                      that (multistatic) or half of it (monostatic);
 *   max_scan_step    = lambda_min / (4 sin(theta_z/2));
 *   res_x = lambda_c / (4 sin(theta_h/2)), res_y = c / (2 B),
 *   res_z = lambda_c / (4 sin(theta_z/2)).
 * L_R = chord_len, R_0 = radius cos(half the chord angle) (chord to scene
 * centre), D = target_dim (largest target dimension, m), theta_h = the arc of
 * all chords, theta_z = the smaller of the angle the scan length subtends at
 * the radius and beamwidth_z_deg (0: no beam limit). elem_spacing is the
 * largest gap between neighbouring (receive) elements of a section;
 * spacing_ok / scan_step_ok compare the actual values with the limits. */
typedef struct {
    double lambda_min, lambda_c, bandwidth;
    double theta_h_deg, theta_z_deg;
    double max_rx_spacing, max_elem_spacing, max_scan_step;
    double res_x, res_y, res_z;
    double elem_spacing, scan_step;
    int spacing_ok, scan_step_ok;
} pl_design_info;
pl_status pl_design(const pl_geometry *geom, const pl_scan *scan, const pl_freqs *freqs,
                    double target_dim, double beamwidth_z_deg, pl_design_info *out);

/* The two comparison algorithms of Sec. III (Table II), on the plan's
 * geometry, scan, band and voxel grid; same buffers as pl_execute, asynchronous
 * on `stream`. They exist to time and check the method against; their first
 * call builds small per-plan tables (synchronously).
 *
 * pl_execute_exact: the hybrid method with exact nonuniform sums instead of
 * the NUFFT ("omega-K-BP" of Sec. III): z-FFT (Eq. 2), then per k_z bin and
 * pixel G = sum_c sum_m S k_m e^{+j kappa a_c} (Eq. 7 / 19, evanescent terms
 * dropped), then the inverse transform over k_z (Eq. 9). FP32 with
 * float-float phases; cost C x M x N_p per pixel.
 *
 * pl_execute_bp_direct: direct back-projection (the "BP" of Sec. III), the
 * matched filter of the echo model Eq. (1) / (10) with the k weight:
 * g(x,y,z) = sum_c sum_n sum_m s[c][n][m] k_m e^{+j k_m (R_T + R_R)},
 * R = distance from the element at scan height z'_n to the voxel. FP32 with
 * float-float ranges and phases; cost C x N x M per voxel. */
pl_status pl_execute_exact(pl_plan *plan, const void *echo_dev, void *image_dev, void *stream);
pl_status pl_execute_bp_direct(pl_plan *plan, const void *echo_dev, void *image_dev,
                               void *stream);

pl_status pl_plan_destroy(pl_plan *plan);
pl_status pl_plan_get_info(const pl_plan *plan, pl_info *info);

/* Device pointer and size of an intermediate buffer, valid until the plan is
 * destroyed (for inspection and tests):
 *  PL_STAGE_ZFFT        -> spectrum S, complex64 [n_chan][n_pad][n_f] (bfloat16 (re, im)
 *                          pairs with precision 2 on the NUFFT paths; not written by
 *                          the tensor-core path with an FFT-length scan: there the
 *                          z-FFT hands its output straight to the range table)
 *  PL_STAGE_RANGE_TABLE -> table b, [n_chan][L][ceil(n_pad/2)] rows of k_z bin pairs
 *                          {re_u, re_u+1, im_u, im_u+1} (float32, or bfloat16 when
 *                          precision >= 1); block_config 4: see pl_options
 *  PL_STAGE_BACKPROJECT -> image spectrum G, complex64 [parts][n_pad][ny][nx]: the
 *                          spectrum is the sum over parts (2 parts, one per half
 *                          of the channels, in the planar block_config 4 layout;
 *                          else 1) */
pl_status pl_plan_workspace(pl_plan *plan, int stage, void **dev_ptr, size_t *bytes);

/* Per-stage timing with CUDA events recorded on the execute stream.
 * enable != 0 starts recording (and clears the sums). pl_plan_stage_times
 * waits for the recorded events and returns, per stage, the summed
 * milliseconds and the number of executions timed since the last clear.
 * With pl_info.bp_launches == 2 the back-projection stage spans both of its
 * launches (with the inverse transform of the finished pixels beside the
 * second) and the inverse-transform stage is the part left after it. */
pl_status pl_plan_set_timing(pl_plan *plan, int enable);
pl_status pl_plan_stage_times(pl_plan *plan, double ms[PL_NUM_STAGES],
                              int launches[PL_NUM_STAGES]);

/* Scene simulation on the GPU (input synthesis, not part of the
 * reconstruction): echo of point scatterers, Eq. (1) for Tx = Rx and Eq. (10)
 * in general,
 *   echo[c][n][m] = sum_t amp_t exp(-j k_m (R_T + R_R)),  k_m = 2 pi f_m / c.
 * tx_xy, rx_xy: host [n_chan][2]; f_hz: host [n_f]; pts: host [n_pts][3];
 * amp: host [n_pts][2] (complex). echo_dev: device complex64
 * [n_chan][n_scan][n_f]. The range R_T + R_R of every (point, channel, scan
 * position) is formed in FP64 and kept as a float pair; k_m (R_T + R_R) is a
 * float-float product reduced modulo 2 pi before an FP32 sin/cos, so each
 * phase carries ~1e-6 rad of error (accumulation over points in FP32).
 * Synchronises `stream` before returning. */
pl_status pl_synth_echo(int n_chan, const double *tx_xy, const double *rx_xy,
                        double z0, double dz, int n_scan, const double *f_hz, int n_f,
                        int n_pts, const double *pts, const double *amp,
                        void *echo_dev, void *stream);

/* ---- Batches of uneven scans (one persistent launch) --------------------
 * A batch reconstructs n_scenes independent scans whose geometry, scan,
 * band and grid may all differ. pl_execute_batch replays one CUDA graph.
 *
 * Tensor cores (block_config 4, the default): each scene's chain -- transform
 * over z (Eq. 2), range table (Eq. 8a/19a), back-projection (Eq. 8b/19b),
 * inverse transform (Eq. 9) -- with the scenes spread over parallel streams,
 * largest first. With tc_launch = 1 the back-projections are ONE persistent
 * launch instead: the scenes' transforms and range tables on the parallel
 * streams, then one block per SM pulling every scene's back-projection blocks
 * from a device queue (largest scenes first; each scene in the
 * one-block-per-SM layout, K steps and planar or interleaved rows per scene),
 * then the inverse transforms on the parallel streams.
 *
 * FP32 kernels (block_config 1-3): the per-scene transforms over z, then ONE
 * persistent kernel that pulls work items from a device queue -- every
 * scene's range-table blocks first, then every scene's back-projection tiles,
 * largest scenes first -- and finally the per-scene inverse transforms. A
 * back-projection item waits for its scene's range table through a per-scene
 * counter.
 *
 * Every device-side wait is bounded (wait_timeout_ms) and gives up with
 * PL_ERR_TIMEOUT instead of hanging.
 *
 * Block shape: with autotune = 1 (and tile_u = block_config = 0)
 * pl_batch_create times the candidates on this batch -- the persistent
 * tensor-core back-projection, the per-scene tensor-core launches, and the
 * FP32 persistent kernel with tile_u 8, 16 and 20 -- and keeps the fastest;
 * the choice is cached per batch signature for the life of the process. The
 * persistent paths need nufft_w = 6 in every scene (FP32: and a fine grid
 * <= 512 points; tensor cores: at most 96 scenes, one precision); otherwise
 * the batch falls back to per-scene launches inside the same graph (see
 * pl_batch_info.persistent). */
typedef struct pl_batch pl_batch;

typedef struct {
    int tile_u;              /* 0 = default 16 (or autotuned) */
    int block_config;        /* 0 = default 1 (or autotuned) */
    int autotune;            /* 1: choose tile_u / block_config by timing */
    double wait_timeout_ms;  /* bound of a device-side wait (0 = 2000 ms) */
    int debug_unsatisfiable; /* test hook: scene 0's tiles wait for one more range-table
                              * block than exists, so the bounded wait must expire (FP32
                              * persistent kernel; for the tensor-core kernels see
                              * pl_options.debug_unsatisfiable) */
    int tc_launch;           /* block_config 4: 1 = one persistent back-projection for every
                              * scene (PL_ERR_UNSUPPORTED if a scene does not allow it);
                              * 0 or 2 = each scene's own launches on the parallel streams
                              * (default); with autotune both are timed */
    int reserved[6];
} pl_batch_options;

typedef struct {
    int n_scenes;
    int tile_u, block_config;
    int autotuned;             /* 1 if the shape came from timing (or its cache) */
    int persistent;            /* 1: one persistent launch (block_config 4: of the
                                  back-projection); 0: per-scene launches */
    int persistent_blocks;     /* resident blocks of the persistent launch */
    int work_items;            /* range-table + back-projection items */
    int launches_per_execute;  /* kernel launches in the graph */
    double tune_best_ms, tune_default_ms;  /* batch time of the chosen / default shape */
    double updates_per_execute;            /* sum of n_chan * nx * ny * nz * n_f */
    size_t workspace_bytes;
} pl_batch_info;

/* geoms, scans, freqs, grids: arrays of n_scenes host descriptors; opts may
 * be NULL or an array of n_scenes (precision, NUFFT, wait and check_nonfinite
 * fields are used; the block shape comes from bopt). bopt may be NULL. */
pl_status pl_batch_create(pl_batch **out, int n_scenes, const pl_geometry *geoms,
                          const pl_scan *scans, const pl_freqs *freqs, const pl_grid *grids,
                          const pl_options *opts, const pl_batch_options *bopt);
/* echo_dev[i], image_dev[i]: device buffers of scene i (layouts as in
 * pl_execute). The pointer arrays are host memory. Runs on `stream` and
 * synchronises it before returning (the status is read back: PL_ERR_TIMEOUT
 * for an expired wait, PL_ERR_NONFINITE when a scene built with
 * check_nonfinite had NaN or Inf in its echo). */
pl_status pl_execute_batch(pl_batch *batch, const void *const *echo_dev,
                           void *const *image_dev, void *stream);
pl_status pl_batch_get_info(const pl_batch *batch, pl_batch_info *info);
pl_status pl_batch_destroy(pl_batch *batch);

/* ---- Learned fast path (the paper has no learned component) --------------
 * Kernels of the 3-D convolutional encoder-decoder that maps a cheap
 * reconstruction (half the frequencies, low NUFFT oversampling) to the full
 * one; the network and its training loop are driven from
 * paper_2109_02842_gb300/learned.py. All volumes are channels-last device
 * arrays x[v][c], v = (z H + y) W + x. BF16 tensors are bfloat16, others FP32.
 * All calls are asynchronous on `stream`.
 *
 * pl_nn_conv3d: out[v][co] = act(bias[co] + sum_{tap,ci} w[co][tap Cin + ci]
 *   x[v + off(tap)][ci]); 3x3x3 taps tap = (dz 3 + dy) 3 + dx at offset
 *   (dz-1, dy-1, dx-1), zero padding; x BF16 [V][Cin]; w BF16
 *   [Cout][pl_nn_padded_k(Cin)] (row tail zero); bias FP32 [Cout] or NULL;
 *   relu != 0 applies max(., 0); out BF16 (out_bf16 != 0) or FP32 [V][Cout].
 *   BF16 tensor-core MMA with FP32 accumulation.
 * pl_nn_conv3d_wgrad: gw[co][tap Cin + ci] += sum_v gy[v][co] x[v+off][ci] and
 *   gb[co] += sum_v gy[v][co] (gb may be NULL); x, gy BF16; gw, gb FP32;
 *   Cout <= 32, 49-64 or 113-128. `work` is caller-owned device scratch of at
 *   least pl_nn_wgrad_workspace(...) bytes for per-chunk partial sums, which
 *   are added in a fixed order (bitwise reproducible gradients).
 * pl_nn_weight_flip: wt[ci][(26 - tap) Cout + co] = w[co][tap Cin + ci], the
 *   weights of the transposed convolution (input gradient = pl_nn_conv3d of
 *   the output gradient with wt, Cin and Cout swapped).
 * pl_nn_elementwise op: 0 out(BF16) = a(FP32) where b(BF16) > 0 else 0 (ReLU
 *   backward); 1 out(BF16) = a(FP32); 2 out(BF16) = a + b (BF16); 3 out(FP32) += a(FP32).
 * pl_nn_resample op (D, H, W = the fine size for 0/1, the coarse size for 2/3):
 *   0 BF16 2x2x2 mean pool; 1 its adjoint, FP32 accumulate into the fine
 *   gradient; 2 BF16 nearest x2 upsampling; 3 its adjoint (FP32 sum of the 8
 *   children).
 * pl_nn_features: feat BF16 [V][3] = (Re g / s, Im g / s, |g| / s) of a
 *   complex64 volume, s = max |g| written to *scale (device FP32).
 * pl_nn_loss: sums[0] = sum |t/s|^2, sums[1] = sum |pred - t/s|^2 (device
 *   FP32[2], fixed-order reduction; the relative L2 loss is sums[1]/sums[0]);
 *   grad (FP32 [V][2], may be NULL) = 2 (pred - t/s) / sums[0]; pred FP32
 *   [V][2], target complex64.
 * pl_nn_residual: pred[v] += gain (Re img[v], Im img[v]) / s.
 * pl_nn_check: the acceptance check of a learned correction corr (FP32
 *   [V][2], the network's output before pl_nn_residual): out (device FP32[3])
 *   = (number of non-finite entries of corr, sum of corr^2 over the finite
 *   ones, sum |gain img / s|^2); fixed-order reduction through a partial-sum
 *   array inside the library, so two checks must not run at the same time on
 *   different streams. The caller falls back to the plain reconstruction when
 *   out[0] > 0 or the correction is too large against the scaled cheap image.
 * pl_nn_to_complex: img[v] = s (pred[v][0] + j pred[v][1]).
 * pl_nn_adam: one bias-corrected Adam step (Kingma & Ba 2015) on FP32
 *   parameters p with gradient g and moments m, v; refreshes the BF16 copy
 *   p_bf16 when not NULL. */
int pl_nn_padded_k(int cin);
pl_status pl_nn_conv3d(const void *x, const void *w, const float *bias, void *out, int D, int H,
                       int W, int Cin, int Cout, int relu, int out_bf16, void *stream);
size_t pl_nn_wgrad_workspace(int D, int H, int W, int Cin, int Cout);
pl_status pl_nn_conv3d_wgrad(const void *x, const void *gy, float *gw, float *gb, void *work,
                             size_t work_bytes, int D, int H, int W, int Cin, int Cout,
                             void *stream);
pl_status pl_nn_weight_flip(const void *w, void *wt, int Cin, int Cout, void *stream);
pl_status pl_nn_elementwise(int op, const void *a, const void *b, void *out, size_t n,
                            void *stream);
pl_status pl_nn_resample(int op, const void *x, void *y, int D, int H, int W, int C,
                         void *stream);
pl_status pl_nn_features(const void *img, void *feat, float *scale, size_t n, void *stream);
pl_status pl_nn_loss(const float *pred, const void *target, const float *scale, float *sums,
                     float *grad, size_t n, void *stream);
pl_status pl_nn_residual(float *pred, const void *img, const float *scale, float gain, size_t n,
                         void *stream);
pl_status pl_nn_check(const float *corr, const void *img, const float *scale, float gain,
                      size_t n, float *out, void *stream);
pl_status pl_nn_to_complex(const float *pred, const float *scale, void *img, size_t n,
                           void *stream);
pl_status pl_nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, size_t n,
                     float lr, float b1, float b2, float eps, int step, void *stream);

/* Allocation-free variant of pl_synth_echo (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory, e.g. code running
 * while another component owns the device allocator, or services that must
 * not touch the allocator after start-up).
 *
 * Same arguments and same result as pl_synth_echo, but the device-side copies
 * of the inputs live in a fixed scratch array inside the library (a static
 * __device__ variable of about 0.8 MB that every device loading the library
 * holds until exit) instead of buffers allocated per call: this call never
 * calls cudaMalloc or cudaFree. Limits: n_chan <= PL_STATIC_MAX_CHANNELS,
 * n_f <= PL_STATIC_MAX_FREQS, n_pts <= PL_STATIC_MAX_POINTS; larger sizes
 * return PL_ERR_ARG with a message in pl_last_error().
 *  - The first call on a device looks up the scratch address for that device
 *    (with it current) and caches it; make that first call before any stream
 *    capture.
 *  - All calls share the one scratch array, which keeps the last call's
 *    contents. Calls whose GPU work overlaps (e.g. on two streams) race on it:
 *    issue them on one stream or order them.
 *  - The call does not synchronise: the inputs are copied to the scratch with
 *    cudaMemcpyAsync on `stream`, and the echo is complete when `stream`
 *    reaches the end of this call's work. From pageable host memory the copies
 *    are staged before the call returns; from page-locked (pinned) host
 *    memory, or under stream capture, they run later, so keep the host arrays
 *    valid and unchanged until `stream` has reached the end of the call. */
#define PL_STATIC_MAX_CHANNELS 4096
#define PL_STATIC_MAX_FREQS 512
#define PL_STATIC_MAX_POINTS 16384
pl_status pl_synth_echo_static(int n_chan, const double *tx_xy, const double *rx_xy,
                               double z0, double dz, int n_scan, const double *f_hz, int n_f,
                               int n_pts, const double *pts, const double *amp,
                               void *echo_dev, void *stream);

/* Measured peak of one unit that bounds the FP32 back-projection, for its
 * roofline (a device micro-benchmark on `stream`, ~0.1 s; synchronises it;
 * changes no device setting):
 *   which 0: FP32 FMA pipe, *value in TFLOP/s (2 flop per FMA);
 *   which 1: MUFU sine, *value in G sin/s;
 *   which 2: shared-memory load bandwidth (conflict-free 16-byte loads),
 *            *value in GB/s.
 * Every SM is filled with independent dependency chains; the best of three
 * timed launches after a warm-up launch is kept. */
pl_status pl_measure_peak(int which, void *stream, double *value);

const char *pl_status_string(pl_status s);
const char *pl_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int pl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POLYLINE_H */
