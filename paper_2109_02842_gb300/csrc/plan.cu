// Host side of libpolyline: argument validation, plan construction (sizes,
// device workspace, plan-time tables) and the C ABI of include/polyline.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polyline.h"
#include "common.cuh"
#include "kernels.h"
#include "plan_internal.h"
#include "tc05.cuh"
#include "wave_split.h"

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor-core back-projection layout. TMEM columns of a block: the
// accumulators (Re G, Im G: 2 UT planar; P, Q: 4 UT interleaved) and one A
// buffer (npl planes x ks steps x 8) for each of npar channel classes; 2
// classes in 256 columns (2 blocks per SM) or 3 in 512 (1 block per SM).
int tc_cols(int ut, int npar, int npl, int ks, bool planar) {
    return (planar ? 2 : 4) * ut + npar * npl * ks * 8;
}
// (force3: the one-block-per-SM layout of three classes whatever fits)
int tc_npar(int ut, int npl, int ks, bool planar, bool force3 = false) {
    if (planar && ut > 256) return 0;          // the MMA's N is at most 256
    if (!force3 && tc_cols(ut, 2, npl, ks, planar) <= 256) return 2;
    if (tc_cols(ut, 3, npl, ks, planar) <= 512) return 3;
    return 0;
}
// The layout fits: tensor memory, and two slot groups of table windows in
// shared memory (npl 4: hi/lo planes).
bool tc_fits(int ut, int npl, int ks, bool planar, bool force3 = false) {
    const int npar = tc_npar(ut, npl, ks, planar, force3);
    if (npar == 0) return false;
    const int N = planar ? ut : 2 * ut;
    const size_t cb = (size_t)(npl == 4 ? 2 : 1) * 16 * ks * 128;
    const size_t slot = (size_t)(planar ? 2 : 1) * ((N + 63) / 64) * cb;
    return 1024 + 2 * npar * slot + 512 <= 227 * 1024;
}
// The 2:4-sparse products (planar layout, 16-row windows): TMEM columns of
// the accumulators, each class's compressed A matrices (nmat x 8 columns) and
// its metadata column (8 apart); classes: 2 in 256 columns (two blocks per
// SM), else 3, else 2 in 512.
int tc_cols_sp(int ut, int npar, int nmat) { return 2 * ut + npar * nmat * 8 + npar * 8; }
int tc_npar_sp(int ut, int nmat) {
    if (ut > 256) return 0;
    if (tc_cols_sp(ut, 2, nmat) <= 256) return 2;
    if (tc_cols_sp(ut, 3, nmat) <= 512) return 3;
    if (tc_cols_sp(ut, 2, nmat) <= 512) return 2;
    return 0;
}

// Bins per block of the interleaved layout (used where the planar one does
// not fit): the fewest blocks that the largest 1-block-per-SM tile allows,
// split evenly (multiple of 8), e.g. N_p = 200 -> 2 x 104, 128 -> 2 x 64.
int tc_auto_tile(int np, int npl, int ks) {
    const int ut_max = (512 - 3 * npl * ks * 8) / 4 / 8 * 8;
    const int n = (np + ut_max - 1) / ut_max;
    const int ut = ((np + n - 1) / n + 7) / 8 * 8;
    return std::max(ut, 16);
}

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiledFn encode_tiled_fn();

// TMA map of the planar table [c][hi/lo][row][Re | Im columns] (BF16, `part`
// columns per half) for the sparse products with windows of rw = 4 NG rows
// (NG = 4 or 3 residue classes): a box is 64 columns x 4 row groups (NG rows
// apart) x NG rows in a group x (Re, Im) x `planes` (hi[, lo]), so that a box
// at (group i / NG, row-in-group i % NG) holds rows i + j + NG e in the order
// [plane][Re / Im][j][e]. The row-in-group dimension has 2 NG - 1 entries
// over overlapping rows, so any first row i is reachable; the last group
// ends inside the channel's plane (rows NG (ng - 1) + 2 NG - 2 < L).
// The interleaved table [c][hi/lo][row][tc_cols columns of (re, im) pairs]
// (planar = false, `part` = tc_cols, rw = 16 or 32): no Re / Im dimension
// (extent 1), rw / 4 row groups of 4 rows, a box holding rows i + j + 4 e in
// the order [plane][j][e] (j < 4, e < rw / 4).
bool encode_sparse_map(CUtensorMap *m, void *table, int part, int L, int C, int planes,
                       int rw, bool planar) {
    EncodeTiledFn enc = encode_tiled_fn();
    const int NG = rw == 12 ? 3 : 4;
    if (!enc || (rw != 16 && rw != 12 && rw != 32) || L < 2 * NG) return false;
    const cuuint64_t pitch = (cuuint64_t)part * 2 * (planar ? 2 : 1);
    const cuuint64_t ng = (cuuint64_t)((L - (2 * NG - 1)) / NG + 1);
    const cuuint64_t dims[5] = {(cuuint64_t)part, ng, (cuuint64_t)(2 * NG - 1),
                                (cuuint64_t)(planar ? 2 : 1), 2 * (cuuint64_t)C};
    const cuuint64_t strides[4] = {(cuuint64_t)NG * pitch, pitch,
                                   planar ? (cuuint64_t)part * 2 : pitch, (cuuint64_t)L * pitch};
    const cuuint32_t box[5] = {64, (cuuint32_t)(rw / NG), (cuuint32_t)NG,
                               (cuuint32_t)(planar ? 2 : 1), (cuuint32_t)planes};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, table, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

EncodeTiledFn encode_tiled_fn() {
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

thread_local std::string g_err;

pl_status fail(pl_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

pl_status cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PL_ERR_OOM : PL_ERR_CUDA;
}

#define PL_CUDA(call, where)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);    \
    } while (0)

bool finite(double v) { return std::isfinite(v); }

// Gauss-Legendre nodes and weights on [0, 1] by Newton's method on the
// Legendre polynomial P_n (three-term recurrence); textbook construction.
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (z + 1.0);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // = (2 / ((1-z^2) P'^2)) / 2
    }
}

// Chebyshev interpolation of ES tap t on s in [-1, 1] at D+1 nodes, returned
// as monomial coefficients in s (textbook construction, double precision).
void es_tap_polynomial(int W, double beta, int t, int D, float *mono) {
    const int n = D + 1;
    auto es = [&](double x) {
        const double z = 2.0 * x / W;
        const double q = 1.0 - z * z;
        return q > 0.0 ? std::exp(beta * (std::sqrt(q) - 1.0)) : 0.0;
    };
    std::vector<double> fx(n), c(n, 0.0);
    for (int j = 0; j < n; ++j) {
        const double s = std::cos(M_PI * (j + 0.5) / n);
        fx[j] = es(0.5 * (s + 1.0) + 0.5 * W - 1.0 - t);
    }
    for (int k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += fx[j] * std::cos(M_PI * k * (j + 0.5) / n);
        c[k] = 2.0 * acc / n;
    }
    c[0] *= 0.5;
    std::vector<std::vector<double>> T(n, std::vector<double>(n, 0.0));
    T[0][0] = 1.0;
    if (n > 1) T[1][1] = 1.0;
    for (int k = 1; k + 1 < n; ++k)
        for (int i = 0; i < n; ++i)
            T[k + 1][i] = (i > 0 ? 2.0 * T[k][i - 1] : 0.0) - T[k - 1][i];
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += c[k] * T[k][i];
        mono[i] = (float)acc;
    }
}

// Radix sequence of a 2^a 3^b 5^c length. Radix 8 (fewer passes) pays off
// in the column-pair z transforms; the fine-grid transform of the range table
// keeps radices up to 5.
bool smooth_plan(int n, FftPlan &p, bool radix8) {
    p.n = n;
    p.n_stages = 0;
    int r = n;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int oi = radix8 ? 0 : 1; oi < 5; ++oi) {
        while (r % order[oi] == 0) {
            if (p.n_stages == 16) return false;
            p.radix[p.n_stages++] = order[oi];
            r /= order[oi];
        }
    }
    return r == 1 && n > 1;
}

// min / max distance from (px, py) to the rectangle [x0,x1] x [y0,y1]
void rect_dist(double px, double py, double x0, double x1, double y0, double y1, double &dmin,
               double &dmax) {
    const double cx = std::min(std::max(px, x0), x1);
    const double cy = std::min(std::max(py, y0), y1);
    dmin = std::hypot(px - cx, py - cy);
    dmax = 0.0;
    const double xs[2] = {x0, x1}, ys[2] = {y0, y1};
    for (double xx : xs)
        for (double yy : ys) dmax = std::max(dmax, std::hypot(px - xx, py - yy));
}

// SM clock cycles of a bounded device-side wait: about 2 s by default, else
// the requested microseconds at the device's clock rate.
long long wait_budget_cycles(int us) {
    if (us <= 0) return 4ll << 30;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0)
        khz = 2000000;
    return (long long)us * khz / 1000;
}

// Plan-time device allocations go through here: pl_options.debug_fail_alloc
// = n makes the n-th one of the plan being built fail as if the device were
// out of memory (a test hook for the PL_ERR_OOM path; nothing is allocated).
thread_local int g_fail_alloc_countdown = 0;

cudaError_t plan_malloc(void **p, size_t bytes) {
    if (g_fail_alloc_countdown > 0 && --g_fail_alloc_countdown == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dalloc(T **p, size_t count, size_t &total) {
    total += count * sizeof(T);
    return plan_malloc((void **)p, std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace


namespace {

pl_status validate(const pl_geometry *g, const pl_scan *s, const pl_freqs *f, const pl_grid *gr) {
    if (!g || !s || !f || !gr) return fail(PL_ERR_ARG, "NULL descriptor");
    if (g->mode != 0 && g->mode != 1) return fail(PL_ERR_ARG, "geometry.mode must be 0 or 1");
    if (g->n_elem <= 0 || !g->elem_xy) return fail(PL_ERR_GEOMETRY, "no elements");
    for (int i = 0; i < 2 * g->n_elem; ++i)
        if (!finite(g->elem_xy[i])) return fail(PL_ERR_NONFINITE, "element position not finite");
    if (g->mode == 1) {
        if (g->n_pairs <= 0 || !g->pair_tx || !g->pair_rx)
            return fail(PL_ERR_GEOMETRY, "multistatic geometry needs pairs");
        for (int i = 0; i < g->n_pairs; ++i)
            if (g->pair_tx[i] < 0 || g->pair_tx[i] >= g->n_elem || g->pair_rx[i] < 0 ||
                g->pair_rx[i] >= g->n_elem)
                return fail(PL_ERR_GEOMETRY, "pair index out of range");
    }
    if (s->n <= 0) return fail(PL_ERR_ARG, "scan.n must be positive");
    if (!finite(s->z0) || !finite(s->dz)) return fail(PL_ERR_NONFINITE, "scan not finite");
    if (!(s->dz > 0)) return fail(PL_ERR_ARG, "scan.dz must be positive");
    if (s->n_pad != 0 && s->n_pad < s->n) return fail(PL_ERR_ARG, "scan.n_pad < scan.n");
    if (f->n <= 0 || !f->f_hz) return fail(PL_ERR_FREQ, "no frequencies");
    for (int m = 0; m < f->n; ++m) {
        if (!finite(f->f_hz[m])) return fail(PL_ERR_NONFINITE, "frequency not finite");
        if (!(f->f_hz[m] > 0)) return fail(PL_ERR_FREQ, "frequency must be positive");
        if (m > 0 && !(f->f_hz[m] > f->f_hz[m - 1]))
            return fail(PL_ERR_FREQ, "frequencies must be strictly ascending");
    }
    const double gv[6] = {gr->x0, gr->dx, gr->y0, gr->dy, gr->z0, gr->dz};
    for (double v : gv)
        if (!finite(v)) return fail(PL_ERR_NONFINITE, "grid not finite");
    if (gr->nx <= 0 || gr->ny <= 0 || gr->nz <= 0) return fail(PL_ERR_ARG, "empty image grid");
    if (!(gr->dx > 0) || !(gr->dy > 0)) return fail(PL_ERR_ARG, "grid.dx, grid.dy must be positive");
    if (gr->nz > 1 && !(gr->dz > 0)) return fail(PL_ERR_ARG, "grid.dz must be positive");
    return PL_OK;
}

BpDesc make_bp(const pl_plan *P) {
    const NufftDesc &d = P->nd;
    BpDesc bp{};
    bp.mode = P->mode;
    bp.n_chan = P->C;
    bp.n_pad = P->Np;
    bp.L = d.L;
    bp.R = P->R;
    bp.nx = P->grid.nx;
    bp.ny = P->grid.ny;
    bp.x0 = P->grid.x0;
    bp.dx = P->grid.dx;
    bp.y0 = P->grid.y0;
    bp.dy = P->grid.dy;
    bp.h = d.h;
    bp.l0 = d.l0;
    bp.inv_h = (float)(1.0 / d.h);
    bp.dxf = (float)P->grid.dx;
    bp.dyf = (float)P->grid.dy;
    bp.beta = d.beta;
    bp.two_over_w = 2.0f / d.w;
    bp.w = d.w;
    bp.tile_u = P->tile_u;
    bp.block_config = P->block_config;
    bp.tile_px = P->block_config == 4 ? backproject_tc_tile_x() : backproject_tile_x(P->block_config);
    bp.tile_py = P->block_config == 4 ? backproject_tc_tile_y() : backproject_tile_y();
    bp.bf16 = P->precision >= 1;
    return bp;
}

pl_status build_plan(pl_plan *P, const pl_geometry *g, const pl_scan *s, const pl_freqs *f,
                     const pl_grid *gr, const pl_options *opt) {
    pl_options o{};
    if (opt) o = *opt;
    if (o.nufft_sigma == 0) o.nufft_sigma = 2.0;
    if (o.nufft_w == 0) o.nufft_w = 6;

    if (!(o.nufft_sigma >= 1.2 && o.nufft_sigma <= 8.0))
        return fail(PL_ERR_ARG, "nufft_sigma must be in [1.2, 8]");
    if (o.nufft_w < 4 || o.nufft_w > 12 || (o.nufft_w & 1))
        return fail(PL_ERR_ARG, "nufft_w must be even, 4..12");
    if (o.block_config == 4) {
        if (o.tile_u != 0 && (o.tile_u % 8 != 0 || o.tile_u < 16 || o.tile_u > 112))
            return fail(PL_ERR_ARG, "with block_config 4, tile_u must be 0 or a multiple of 8 in 16..112");
    } else if (o.tile_u != 0 && o.tile_u != 8 && o.tile_u != 16 && o.tile_u != 20 && o.tile_u != 24) {
        return fail(PL_ERR_ARG, "tile_u must be 0, 8, 16, 20 or 24");
    }
    if (o.precision < 0 || o.precision > 2) return fail(PL_ERR_ARG, "precision must be 0, 1 or 2");
    if (o.debug_unsatisfiable < 0 || o.debug_unsatisfiable > 3 || o.wait_timeout_us < 0)
        return fail(PL_ERR_ARG, "debug_unsatisfiable must be 0..3, wait_timeout_us >= 0");
    if (o.check_nonfinite < 0 || o.check_nonfinite > 1 || o.debug_fail_alloc < 0 ||
        o.dense_products < 0 || o.dense_products > 1 ||
        (o.sparse_window_rows != 0 && o.sparse_window_rows != 12))
        return fail(PL_ERR_ARG, "check_nonfinite and dense_products must be 0 or 1, "
                                "sparse_window_rows 0 or 12, debug_fail_alloc >= 0");
    g_fail_alloc_countdown = o.debug_fail_alloc;
    P->check_nonfinite = o.check_nonfinite != 0;
    // the device-side status word (mapped host memory): expired waits of the
    // tensor-core kernels, non-finite echo values
    PL_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&P->h_err), sizeof(int), cudaHostAllocMapped),
            "cudaHostAlloc");
    *P->h_err = 0;
    PL_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&P->d_err), P->h_err, 0),
            "cudaHostGetDevicePointer");

    PL_CUDA(cudaGetDevice(&P->device), "cudaGetDevice");
    P->mode = g->mode;
    P->C = g->mode == 0 ? g->n_elem : g->n_pairs;
    P->N = s->n;
    P->Np = s->n_pad ? s->n_pad : s->n;
    P->M = f->n;
    P->z0s = s->z0;
    P->dzs = s->dz;
    P->grid = *gr;
    P->precision = o.precision;
    P->tile_u = o.tile_u;
    if (o.block_config < 0 || o.block_config > 4)
        return fail(PL_ERR_ARG, "block_config must be 0..4");
    P->block_config = o.block_config;
    if (P->block_config == 4 && o.nufft_w != 4 && o.nufft_w != 6 && o.nufft_w != 8)
        return fail(PL_ERR_UNSUPPORTED, "block_config 4 needs nufft_w 4, 6 or 8");
    {
        const int n = s->n_pad ? s->n_pad : s->n;
        if (P->block_config == 4) {
            // default: the planar layout with every bin in one block (N = N_p
            // rounded up to 16); an explicit tile_u asks for interleaved blocks
            if (P->tile_u == 0) {
                P->tile_u = (n + 15) / 16 * 16;
                P->tc.planar = 1;
            }
        } else if (P->tile_u == 0) {    // fewest padded bins; 20 only when it wastes less than 16
            const int w16 = (n + 15) / 16 * 16 - n, w20 = (n + 19) / 20 * 20 - n;
            P->tile_u = w20 < w16 ? 20 : 16;
        }
    }
    P->sigma = o.nufft_sigma;

    // channel positions (xT, yT, xR, yR)
    std::vector<double> chxy(4 * (size_t)P->C);
    for (int c = 0; c < P->C; ++c) {
        const int et = g->mode == 0 ? c : g->pair_tx[c];
        const int er = g->mode == 0 ? c : g->pair_rx[c];
        chxy[4 * c + 0] = g->elem_xy[2 * et];
        chxy[4 * c + 1] = g->elem_xy[2 * et + 1];
        chxy[4 * c + 2] = g->elem_xy[2 * er];
        chxy[4 * c + 3] = g->elem_xy[2 * er + 1];
    }
    std::vector<double> k(P->M);
    for (int m = 0; m < P->M; ++m) k[m] = PL_TWO_PI * f->f_hz[m] / PL_C0;
    P->h_chxy = chxy;
    P->h_k = k;

    size_t &ws = P->workspace;
    PL_CUDA(dalloc(&P->d_chxy, chxy.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_k, k.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kc, P->Np, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kchl, P->Np, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kspan, P->Np, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kband, 2 * (size_t)P->Np, ws), "cudaMalloc");
    PL_CUDA(cudaMemcpy(P->d_chxy, chxy.data(), chxy.size() * 8, cudaMemcpyHostToDevice), "copy");
    PL_CUDA(cudaMemcpy(P->d_k, k.data(), k.size() * 8, cudaMemcpyHostToDevice), "copy");

    cudaStream_t st = 0;
    // band centre and span of every k_z bin (the tensor-core back-projection
    // shares one centre per block of `group` bins); kmax = the widest span
    double kmax = 0.0;
    auto band = [&](int group) -> pl_status {
        PL_CUDA(launch_setup_kz(P->mode, P->Np, P->dzs, P->M, P->d_k, group, P->d_kband,
                                P->d_kc, P->d_kchl, P->d_kspan, st), "setup_kz");
        std::vector<double> kspan(P->Np);
        PL_CUDA(cudaMemcpy(kspan.data(), P->d_kspan, P->Np * 8, cudaMemcpyDeviceToHost), "copy");
        kmax = 0.0;
        for (double v : kspan) kmax = std::max(kmax, v);
        if (!(kmax > 0.0)) {
            // a single frequency (or all bins evanescent but one): use a nominal band
            bool alive = false;
            std::vector<double> kc(P->Np);
            PL_CUDA(cudaMemcpy(kc.data(), P->d_kc, P->Np * 8, cudaMemcpyDeviceToHost), "copy");
            for (double v : kc) alive = alive || v > 0.0;
            if (!alive) return fail(PL_ERR_EVANESCENT, "every (k_z, f) term is evanescent");
            kmax = 1.0;   // every live bin has one source at kappa'' = 0
        }
        return PL_OK;
    };
    {
        // one band centre per block of tile_u bins, for every kernel: the
        // carrier is then one sin/cos per (pixel, channel), not per bin
        const pl_status bs = band(P->tile_u);
        if (bs != PL_OK) return bs;
    }

    // NUFFT geometry
    const int W = o.nufft_w;
    double h = PL_TWO_PI / (o.nufft_sigma * kmax);
    // two pixels per thread when x-neighbours are less than one table row
    // apart in range (then their tap windows differ by at most one row)
    const double da_step = (P->mode == 0 ? 1.0 : 2.0) * gr->dx;
    const bool px2_ok = da_step < 0.999 * h && W <= 8;
    if (P->block_config == 3 && !px2_ok)
        return fail(PL_ERR_UNSUPPORTED, "block_config 3 needs an x step below the table step");
    if (P->block_config == 0) P->block_config = px2_ok ? 3 : 1;
    const int TX = P->block_config == 4 ? backproject_tc_tile_x() : backproject_tile_x(P->block_config);
    const int TY = P->block_config == 4 ? backproject_tc_tile_y() : backproject_tile_y();
    const double hs_pix = 0.5 * std::hypot((TX - 1) * gr->dx, (TY - 1) * gr->dy);
    const double hs = P->mode == 0 ? hs_pix : 2.0 * hs_pix;
    P->R = (int)std::ceil(2.0 * hs / h) + W + (P->block_config == 3 ? 1 : 0) + 5;
    const int ntx = (gr->nx + TX - 1) / TX, nty = (gr->ny + TY - 1) / TY;
    const double rx0 = gr->x0, rx1 = gr->x0 + (ntx * TX - 1) * gr->dx;
    const double ry0 = gr->y0, ry1 = gr->y0 + (nty * TY - 1) * gr->dy;
    double amin = 1e300, amax = -1e300;
    for (int c = 0; c < P->C; ++c) {
        double lo, hi, lo2 = 0, hi2 = 0;
        rect_dist(chxy[4 * c], chxy[4 * c + 1], rx0, rx1, ry0, ry1, lo, hi);
        if (P->mode == 1) rect_dist(chxy[4 * c + 2], chxy[4 * c + 3], rx0, rx1, ry0, ry1, lo2, hi2);
        amin = std::min(amin, lo + lo2);
        amax = std::max(amax, hi + hi2);
    }
    NufftDesc &d = P->nd;
    d.mode = P->mode;
    d.n_chan = P->C;
    d.n_pad = P->Np;
    d.n_f = P->M;
    d.w = W;
    d.w1 = 7;
    d.beta = (float)(0.97 * M_PI * (1.0 - 0.5 / o.nufft_sigma) * W);
    d.beta1 = (float)(2.30 * d.w1);
    d.h = h;
    int L;
    if (P->block_config == 4) {
        // tensor-core windows: 16 ks rows from the lowest first tap of each
        // (16 x 8 tile, channel), found by a pass over the tile's pixels;
        // l0 leaves w/2 + 2 rows below the nearest range
        const int npl = P->precision >= 1 ? 2 : 4;
        PL_CUDA(dalloc(&P->d_tgeo, (size_t)ntx * nty * P->C, ws), "cudaMalloc");
        int stats[2] = {0, 0}, ks = 0;
        const bool sp_allowed = !o.dense_products && (W == 4 || W == 6 || W == 8);
        // a sparse table map of this layout encodes (the encoder only checks
        // the layout: the address is not read)
        auto trial_map = [&](int part, int rows, int rw, bool planar) {
            CUtensorMap trial{};
            alignas(64) static unsigned char probe_buf[64];
            const uintptr_t fake = (reinterpret_cast<uintptr_t>(probe_buf) + 63) & ~(uintptr_t)63;
            return encode_sparse_map(&trial, reinterpret_cast<void *>(fake), part, rows, P->C,
                                     P->precision >= 1 ? 1 : 2, rw, planar);
        };
        // the planar layout with two K steps takes the sparse products with
        // 32-row windows: two channel classes of 1.5 npl compressed A
        // matrices (Re A, Im A and -Im A) beside the accumulators, and two
        // slot groups of two windows (a 64-column block of a window: Re and
        // Im rows of each plane, 32 rows each) within 200 KB
        auto sp32_fits = [&](int ut, int rows) {
            if (!sp_allowed || o.one_block_per_sm || ut > 256) return false;
            const size_t cb = (size_t)(npl == 4 ? 2 : 1) * 2 * 32 * 128;
            return tc_cols_sp(ut, 2, npl + npl / 2) <= 512 &&
                   2 * 2 * (size_t)((ut + 63) / 64) * cb <= 200 * 1024 &&
                   trial_map(ut * ((P->Np + ut - 1) / ut), rows, 32, true);
        };
        // table rows of the sparse map over windows of 16 ks rows
        auto sp_rows = [&](int ks_) {
            int r = stats[1] + 16 * ks_;
            return r + (r & 1) + 4;
        };
        for (int attempt = 0;; ++attempt) {
            d.h = h;
            d.l0 = amin - h * (0.5 * W + 2.0);
            d.L = 0;
            BpDesc gb = make_bp(P);
            int *d_stats = nullptr;
            PL_CUDA(plan_malloc(reinterpret_cast<void **>(&d_stats), 2 * sizeof(int)), "cudaMalloc");
            cudaError_t e = cudaMemset(d_stats, 0, 2 * sizeof(int));
            if (e == cudaSuccess) e = launch_setup_tile_geo_tc(gb, P->d_chxy, P->d_tgeo, d_stats, st);
            if (e == cudaSuccess) e = cudaMemcpy(stats, d_stats, sizeof(stats), cudaMemcpyDeviceToHost);
            cudaFree(d_stats);
            PL_CUDA(e, "setup_tile_geo_tc");
            ks = stats[0] <= 16 ? 1 : (stats[0] <= 32 ? 2 : 0);
            if (ks == 0)
                return fail(PL_ERR_UNSUPPORTED,
                            "a 16 x 8 pixel tile spans more than 32 table rows (grid too coarse for block_config 4)");
            if (P->tc.planar && ks == 2 && sp32_fits(P->tile_u, sp_rows(2))) break;
            if (tc_fits(P->tile_u, npl, ks, P->tc.planar != 0, o.one_block_per_sm != 0)) break;
            if (attempt > 3 || o.tile_u != 0)
                return fail(PL_ERR_UNSUPPORTED, "tile_u too large for tensor memory");
            // the planar layout with every bin in one block does not fit (too
            // many bins, or two K steps, for tensor or shared memory): planar
            // blocks of at most 208 bins where one K step does (with 16-row
            // windows; half the blocks of bins of the interleaved layout, and
            // fewer products per bin), or of at most 192 bins where two K
            // steps take the sparse products (32-row windows), else
            // interleaved blocks of bins, sized for ks, and their band
            const int nb_pl = (P->Np + 207) / 208;
            const int ut_pl = ((P->Np + nb_pl - 1) / nb_pl + 15) / 16 * 16;
            const int nb_32 = (P->Np + 191) / 192;
            const int ut_32 = ((P->Np + nb_32 - 1) / nb_32 + 15) / 16 * 16;
            if (P->tc.planar && ks == 1 && nb_pl > 1 && P->tile_u != ut_pl) {
                P->tile_u = ut_pl;
            } else if (P->tc.planar && ks == 2 && sp_allowed && !o.one_block_per_sm &&
                       P->tile_u != ut_32) {
                P->tile_u = ut_32;
            } else {
                P->tc.planar = 0;
                P->tile_u = tc_auto_tile(P->Np, npl, ks);
            }
            const pl_status bs = band(P->tile_u);
            if (bs != PL_OK) return bs;
            h = PL_TWO_PI / (o.nufft_sigma * kmax);
        }
        // rows up to the end of the highest window
        L = stats[1] + 16 * ks;
        L += L & 1;
        P->R = 16 * ks;
        P->tc.ks = ks;
        // 2:4-sparse products where the layout allows them (four more table
        // rows: the last row quad of the sparse map must hold every window)
        // (on request, windows of 12 rows, residues mod 3, where every
        // tile's taps span at most 12 rows and w <= 6: a quarter fewer bytes
        // per copy)
        // The interleaved layout with 32-row windows takes them too (one
        // sparse product per real product covers the whole window).
        P->tc.sparse = 0;
        P->tc.rw = 16;
        // (interleaved 16-row windows only with the hi/lo split: the K = 32
        // operand is the window's hi rows and lo rows)
        // (one_block_per_sm: the layout of three channel classes, so that a
        // batch's persistent back-projection can run the scene)
        auto sp_fits = [&](int n) {
            return o.one_block_per_sm ? tc_cols_sp(n, 3, npl) <= 512 : tc_npar_sp(n, npl) > 0;
        };
        const bool sp_planar = P->tc.planar && ((ks == 1 && sp_fits(P->tile_u)) ||
                                                (ks == 2 && sp32_fits(P->tile_u, L + 4)));
        const bool sp_inter = !P->tc.planar && sp_fits(2 * P->tile_u) &&
                              (ks == 2 || P->precision == 0);
        if (sp_allowed && (sp_planar || sp_inter)) {
            const int rw = sp_inter || ks == 2 ? 16 * ks
                           : (stats[0] <= 12 && W <= 6 && o.sparse_window_rows == 12) ? 12
                                                                                      : 16;
            const int n_ut = (P->Np + P->tile_u - 1) / P->tile_u;
            const int part = sp_inter ? 2 * P->tile_u * n_ut : P->tile_u * n_ut;
            if (trial_map(part, L + 4, rw, !sp_inter)) {
                P->tc.sparse = 1;
                P->tc.rw = rw;
                P->R = rw;
                L += 4;
            }
        }
        // (a planar layout with two K steps chosen for the sparse products
        // and not taking them has no dense kernel)
        if (P->tc.planar && !P->tc.sparse &&
            !tc_fits(P->tile_u, npl, ks, true, o.one_block_per_sm != 0))
            return fail(PL_ERR_UNSUPPORTED, "tensor-core layout without a kernel");
    } else {
        // every tile's R-row window [i_lo, i_lo + R), centred on its range, fits:
        // l0 = amin - ((R+1)/2 + 2) h, L = (amax - amin)/h + R + 6
        L = (int)std::ceil((amax - amin) / h) + P->R + 6;
        L += L & 1;
        d.l0 = amin - h * (0.5 * (P->R + 1) + 2.0);
    }
    if (L > 4096) return fail(PL_ERR_UNSUPPORTED, "range-profile table too long (grid too large for the band)");
    // fine grid: the smallest 2^a 3^b 5^c >= max(2 L, 64) (twice the output rows)
    int fine = std::max(2 * L, 64);
    auto smooth5 = [](int n) {
        for (int r : {2, 3, 5})
            while (n % r == 0) n /= r;
        return n == 1;
    };
    while (!smooth5(fine)) ++fine;
    int lg = 0;
    while ((1 << (lg + 1)) <= fine) ++lg;
    d.L = L;
    d.fine = fine;
    d.log2_fine = lg;
    if (range_table_smem_bytes(d) > 200 * 1024)
        return fail(PL_ERR_UNSUPPORTED, "range-profile table too long for shared memory");
    if (P->C > 8192) return fail(PL_ERR_UNSUPPORTED, "more than 8192 channels");
    if (P->block_config == 4) {
        TcArgs &ta = P->tc;
        ta.UT = P->tile_u;
        const int N = ta.planar ? ta.UT : 2 * ta.UT;
        ta.ncb = (N + 63) / 64;
        ta.n_utiles = (P->Np + ta.UT - 1) / ta.UT;
        // planar rows: [Re of every bin | Im of every bin], blocks of UT bins
        ta.split = P->precision >= 1 ? 1 : 3;
        const int planes = ta.split == 3 ? 2 : 1, npl = ta.split == 3 ? 4 : 2;
        ta.cb_bytes = (unsigned)(planes * 16 * ta.ks * 128);
        ta.im_off = ta.planar ? (unsigned)ta.ncb * ta.cb_bytes : 0u;
        ta.im_col = ta.planar ? ta.n_utiles * ta.UT : 0;
        ta.slot_bytes = (unsigned)(ta.planar ? 2 : 1) * ta.ncb * ta.cb_bytes;
        ta.npar = tc_npar(ta.UT, npl, ta.ks, ta.planar != 0, o.one_block_per_sm != 0);
        ta.tmem_cols = ta.npar == 2 ? 256 : 512;
        ta.acol = 2 * N;
        if (ta.sparse) {
            // per 64-column block: planar [hi: Re rows, Im rows][lo: Re rows,
            // Im rows] (rw rows each; 12-row windows end in a 1 KB zero pad),
            // interleaved [hi rows][lo rows] (rw each)
            ta.cb_bytes = (unsigned)(planes * (ta.planar ? 2 : 1) * ta.rw * 128);
            ta.im_off = 0;
            ta.slot_bytes = (unsigned)ta.ncb * ta.cb_bytes + (ta.rw == 12 ? 1024u : 0u);
            // (planar 32-row windows: two classes of Re A, Im A, -Im A)
            const bool p32 = ta.planar && ta.rw == 32;
            const int nmat = p32 ? npl + npl / 2 : npl;
            ta.npar = p32 ? 2 : o.one_block_per_sm ? 3 : tc_npar_sp(N, npl);
            ta.tmem_cols = tc_cols_sp(N, ta.npar, nmat) <= 256 ? 256 : 512;
            ta.mcol = ta.acol + ta.npar * nmat * 8;
        }
        // two channels per class round (twice the products per A wait and
        // release) where three classes of two-channel A buffers fit next to
        // the accumulators and two slot groups of six windows fit in shared
        // memory
        ta.cpr = 1;
        if (!ta.sparse && !o.one_block_per_sm && ta.npar == 3 && 2 * N + 3 * 2 * npl * ta.ks * 8 <= 512 &&
            1024 + 2 * (size_t)3 * 2 * ta.slot_bytes + 512 <= 227 * 1024)
            ta.cpr = 2;
        // window slots: whole slot groups of npar x cpr (at least 2 groups),
        // within ~190 KB (one block per SM) or ~100 KB (two)
        // (the sparse products consume a window twice as fast: one more slot
        // group where it fits keeps the copies ahead of them)
        const size_t pool = ta.tmem_cols > 256 ? (ta.sparse ? 200 : 190) * 1024 : 100 * 1024;
        const size_t group_bytes = (size_t)ta.slot_bytes * ta.npar * ta.cpr;
        const int nsg = (int)std::max<size_t>(2, std::min<size_t>(16, pool / group_bytes));
        ta.nst = nsg * ta.npar * ta.cpr;
        if (backproject_tc_smem_bytes(ta) > 227 * 1024)
            return fail(PL_ERR_UNSUPPORTED, "table window slots exceed shared memory");
        ta.idesc = tc05::idesc_bf16(128, N, 1);
        ta.budget = wait_budget_cycles(o.wait_timeout_us);
        ta.dbg_wait = o.debug_unsatisfiable == 1 ? 1 : 0;
        d.tc_cols = 2 * ta.n_utiles * ta.UT;
        d.tc_planar = ta.planar;
        // planar: two channel parts per tile. Each accumulator then takes as
        // many products as an interleaved P or Q accumulator over all channels
        // (the planar one takes twice as many per channel, and the
        // accumulation error measured on the tensor cores grows in
        // proportion to that count); the parts also fill the SMs' last wave
        // better than one block per tile.
        ta.nsplit = ta.planar && P->C >= 2 * ta.npar ? 2 : 1;
        // the parts add into one spectrum (zeroed first), so the inverse
        // transform reads one spectrum instead of two; the batch's
        // persistent kernel (one_block_per_sm) keeps one spectrum per part
        ta.g_atomic = (ta.nsplit == 2 && !o.one_block_per_sm) ? 1 : 0;
    } else if (backproject_smem_bytes(P->R, P->tile_u, P->C, P->precision >= 1, P->block_config) > 200 * 1024)
        return fail(PL_ERR_UNSUPPORTED, "table window too tall for shared memory (grid too coarse)");
    for (int tp = 0; tp < W; ++tp) es_tap_polynomial(W, (double)d.beta, tp, W + 1, P->coef.c[tp]);

    // plan-time tables
    std::vector<double> glx, glw;
    P->n_gl = 48;
    gauss_legendre01(P->n_gl, glx, glw);
    PL_CUDA(dalloc(&P->d_glx, glx.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_glw, glw.size(), ws), "cudaMalloc");
    PL_CUDA(cudaMemcpy(P->d_glx, glx.data(), glx.size() * 8, cudaMemcpyHostToDevice), "copy");
    PL_CUDA(cudaMemcpy(P->d_glw, glw.data(), glw.size() * 8, cudaMemcpyHostToDevice), "copy");
    PL_CUDA(dalloc(&P->d_xg, (size_t)P->Np * P->M, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_alpha, (size_t)P->Np * P->M, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_dec, (size_t)L, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_twfine, (size_t)fine, ws), "cudaMalloc");
    PL_CUDA(launch_setup_sources(d, P->dzs, P->d_k, P->d_kc, P->d_glx, P->d_glw, P->n_gl,
                                 P->d_xg, P->d_alpha, st), "setup_sources");
    PL_CUDA(launch_setup_deconv(d, P->d_glx, P->d_glw, P->n_gl, P->d_dec, st), "setup_deconv");
    PL_CUDA(launch_twiddles(fine, fine, -1, P->d_twfine, st), "twiddles");
    if (!smooth_plan(fine, P->fineplan, false)) return fail(PL_ERR_UNSUPPORTED, "fine grid length");

    // transforms over z
    const bool smooth = smooth_plan(P->Np, P->zplan, true) && P->Np <= 512;
    P->fwd_fft = smooth;
    if (smooth) {
        PL_CUDA(dalloc(&P->d_twz, (size_t)P->Np, ws), "cudaMalloc");
        PL_CUDA(launch_twiddles(P->Np, P->Np, -1, P->d_twz, st), "twiddles");
    } else {
        PL_CUDA(dalloc(&P->d_Tfwd, (size_t)P->Np * P->N, ws), "cudaMalloc");
        PL_CUDA(launch_dft_matrix_fwd(P->Np, P->N, P->d_Tfwd, st), "dft_matrix_fwd");
    }
    const double q = (gr->z0 - s->z0) / s->dz;
    const long long qi = std::llround(q);
    const bool on_grid = (gr->nz == 1 || std::fabs(gr->dz - s->dz) <= 1e-9 * s->dz) &&
                         std::fabs(q - (double)qi) <= 1e-6 && qi >= 0 && qi + gr->nz <= P->Np;
    P->inv_fft = smooth && on_grid;
    P->inv_off = (int)qi;
    if (!P->inv_fft) {
        PL_CUDA(dalloc(&P->d_Tinv, (size_t)gr->nz * P->Np, ws), "cudaMalloc");
        PL_CUDA(launch_dft_matrix_inv(P->Np, P->dzs, P->z0s, gr->nz, gr->z0, gr->dz, P->d_Tinv, st),
                "dft_matrix_inv");
        if (P->block_config == 4 && encode_tiled_fn()) {
            // tensor-core plans: the transform's products on the tensor cores
            // too (BF16 hi/lo table of T / N_p)
            ZidftTcArgs &zt = P->zt;
            zt = zidft_tc_shape(P->Np, gr->nx * gr->ny, gr->nz);
            zt.budget = wait_budget_cycles(o.wait_timeout_us);
            zt.dbg_wait = o.debug_unsatisfiable == 3 ? 1 : 0;
            const size_t nb = zidft_tc_table_elems(zt) * 2;
            PL_CUDA(plan_malloc(&P->d_TinvB, nb), "cudaMalloc");
            ws += nb;
            PL_CUDA(launch_zidft_tc_table(zt, P->d_Tinv, (float)(1.0 / P->Np),
                                          (__nv_bfloat16 *)P->d_TinvB, st),
                    "zidft_tc_table");
            if (!zidft_tc_make_map(zt, (const __nv_bfloat16 *)P->d_TinvB, &P->tmapZ,
                                   encode_tiled_fn()))
                return fail(PL_ERR_CUDA, "cuTensorMapEncodeTiled failed (z transform table)");
            P->zidft_tc = true;
        }
    }

    // per (pixel tile, channel) geometry of the back-projection
    P->bp = make_bp(P);
    if (P->block_config != 4) {
        const int tpx = P->bp.tile_px, tpy = P->bp.tile_py;
        const size_t ntiles = (size_t)((gr->nx + tpx - 1) / tpx) * ((gr->ny + tpy - 1) / tpy);
        PL_CUDA(dalloc(&P->d_tgeo, ntiles * P->C, ws), "cudaMalloc");
        PL_CUDA(launch_setup_tile_geo(P->bp, P->d_chxy, P->d_tgeo, st), "setup_tile_geo");
    }

    // data workspace
    PL_CUDA(dalloc(&P->d_S, (size_t)P->C * P->Np * P->M, ws), "cudaMalloc");
    // table rows: k_z bins in planar pairs, N_p rounded up to even; or the
    // tensor-core layout [c][hi/lo][column][row] BF16 (zero beyond what the
    // range table writes)
    if (P->block_config == 4)
        P->table_bytes = (size_t)P->C * 2 * L * d.tc_cols * 2;
    else
        P->table_bytes = (size_t)P->C * L * ((P->Np + 1) / 2) * (P->precision >= 1 ? 8 : 16);
    ws += P->table_bytes;
    PL_CUDA(plan_malloc(&P->d_table, P->table_bytes), "cudaMalloc");
    if (P->block_config == 4) {
        PL_CUDA(cudaMemset(P->d_table, 0, P->table_bytes), "cudaMemset");
        // TMA map of the table [c][hi/lo][row][column] (BF16): a box is 64
        // columns x 16 ks rows (x hi/lo), 128-byte swizzled in shared memory
        EncodeTiledFn enc = encode_tiled_fn();
        if (!enc) return fail(PL_ERR_CUDA, "cuTensorMapEncodeTiled not available");
        const TcArgs &ta = P->tc;
        if (ta.sparse) {
            if (!encode_sparse_map(&P->tmap, P->d_table, ta.planar ? d.tc_cols / 2 : d.tc_cols, L, P->C,
                                   ta.split == 3 ? 2 : 1, ta.rw, ta.planar != 0))
                return fail(PL_ERR_CUDA, "cuTensorMapEncodeTiled failed (sparse table map)");
        } else {
            const cuuint64_t dims[3] = {(cuuint64_t)d.tc_cols, (cuuint64_t)L, 2 * (cuuint64_t)P->C};
            const cuuint64_t strides[2] = {(cuuint64_t)d.tc_cols * 2, (cuuint64_t)L * d.tc_cols * 2};
            const cuuint32_t box[3] = {64, (cuuint32_t)(16 * ta.ks), (cuuint32_t)(ta.split == 3 ? 2 : 1)};
            const cuuint32_t es[3] = {1, 1, 1};
            const CUresult r = enc(&P->tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, P->d_table, dims,
                                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(PL_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        }
        // the range table as exact sums on the tensor cores (one or two
        // 64-frequency atoms: up to 128 frequencies; table rows up to 256),
        // else the NUFFT
        RtTcArgs &ra = P->rt;
        ra.C = P->C;
        ra.Np = P->Np;
        ra.M = P->M;
        ra.Kp = (P->M + 63) / 64 * 64;
        ra.natoms = ra.Kp / 64;
        ra.L = L;
        ra.Lp = (L + 15) / 16 * 16;
        // the fewest row parts whose two operand buffers (the persistent
        // kernel's double buffering) fit in shared memory, and whose two
        // accumulator pairs fit in TMEM
        for (ra.nh = 1;; ++ra.nh) {
            ra.Lh = ((ra.Lp + ra.nh - 1) / ra.nh + 15) / 16 * 16;
            if ((range_table_tc_smem_bytes(ra) <= 227 * 1024 && 4 * ra.Lh <= 512) || ra.Lh <= 16)
                break;
        }
        ra.idesc = tc05::idesc_bf16(128, ra.Lh, 0);
        ra.budget = wait_budget_cycles(o.wait_timeout_us);
        ra.dbg_wait = o.debug_unsatisfiable == 2 ? 1 : 0;
        ra.a_hi_only = P->precision == 2 ? 1 : 0;
        {
            int dev = 0, sms = 0;
            PL_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
            PL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                    "cudaDeviceGetAttribute");
            ra.grid = sms;
        }
        P->rt_tc = ra.natoms <= 2 && ra.Lp <= 256 && 4 * ra.Lh <= 512 &&
                   range_table_tc_smem_bytes(ra) <= 227 * 1024;
        if (P->rt_tc) {
            const size_t nE = (size_t)P->Np * 4 * ra.Lp * ra.Kp;
            const size_t nA = (size_t)P->Np * 4 * P->C * ra.Kp;
            const size_t nprod = (size_t)P->Np * 2 * ra.nh * ra.Lh * ((P->C + 127) / 128 * 128);
            PL_CUDA(plan_malloc(&P->d_rtE, nE * 2), "cudaMalloc");
            PL_CUDA(plan_malloc(&P->d_rtA, nA * 2), "cudaMalloc");
            PL_CUDA(cudaMemset(P->d_rtA, 0, nA * 2), "cudaMemset");   // frequencies >= M stay 0
            PL_CUDA(plan_malloc(&P->d_rtprod, nprod * 4), "cudaMalloc");
            ws += nE * 2 + nA * 2 + nprod * 4;
            PL_CUDA(launch_setup_rt_E(d, P->dzs, P->d_k, P->d_kc, P->d_alpha, ra.Lp, ra.Kp,
                                      P->d_rtE, st),
                    "setup_rt_E");
            const cuuint64_t da[3] = {(cuuint64_t)ra.Kp, (cuuint64_t)P->C, 4 * (cuuint64_t)P->Np};
            const cuuint64_t sa[2] = {(cuuint64_t)ra.Kp * 2, (cuuint64_t)P->C * ra.Kp * 2};
            const cuuint32_t ba[3] = {64, 128, 1};
            const cuuint64_t db[3] = {(cuuint64_t)ra.Kp, (cuuint64_t)ra.Lp, 4 * (cuuint64_t)P->Np};
            const cuuint64_t sb[2] = {(cuuint64_t)ra.Kp * 2, (cuuint64_t)ra.Lp * ra.Kp * 2};
            const cuuint32_t bb[3] = {64, (cuuint32_t)ra.Lh, 1};
            const cuuint32_t e3[3] = {1, 1, 1};
            CUresult r1 = enc(&P->tmapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, P->d_rtA, da, sa, ba,
                              e3, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            CUresult r2 = enc(&P->tmapE, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, P->d_rtE, db, sb, bb,
                              e3, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
                return fail(PL_ERR_CUDA, "cuTensorMapEncodeTiled failed (range table)");
        }
    }
    // the spectrum G[part][u][y][x]: two parts when the tensor-core
    // back-projection splits each tile's channels
    const int g_parts = P->block_config == 4 ? P->tc.nsplit : 1;
    PL_CUDA(dalloc(&P->d_G, (size_t)g_parts * P->Np * gr->nx * gr->ny, ws), "cudaMalloc");
    // blocks of the back-projection's full waves, and the pixels whose every
    // channel part they cover: with one bin block, tile t's last part is
    // block (nsplit - 1) T + t, so the first bp_full - (nsplit - 1) T tiles
    // (whole rows of tiles of them) are done when the full waves are
    if (P->block_config == 4 && P->tc.planar && P->tc.n_utiles == 1 && P->inv_fft) {
        int dev = 0, sms = 0;
        PL_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
        PL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                "cudaDeviceGetAttribute");
        const size_t smem = backproject_tc_smem_bytes(P->tc) + 1024;
        const int per_sm = std::max(1, std::min(512 / P->tc.tmem_cols, (int)((228 * 1024) / smem)));
        const int nbx = (gr->nx + backproject_tc_tile_x() - 1) / backproject_tc_tile_x();
        const WaveSplit wsplit =
            bp_wave_split(backproject_tc_blocks(P->bp, P->tc), sms * per_sm, P->tc.nsplit, nbx,
                          backproject_tc_tile_y(), gr->nx, gr->ny);
        if (wsplit.full > 0) {
            PL_CUDA(cudaStreamCreateWithFlags(&P->s_bp, cudaStreamNonBlocking),
                    "cudaStreamCreateWithFlags");
            PL_CUDA(cudaEventCreateWithFlags(&P->ev_bpA, cudaEventDisableTiming), "cudaEventCreate");
            PL_CUDA(cudaEventCreateWithFlags(&P->ev_bpB, cudaEventDisableTiming), "cudaEventCreate");
            PL_CUDA(cudaEventCreateWithFlags(&P->ev_z0, cudaEventDisableTiming), "cudaEventCreate");
            PL_CUDA(cudaEventCreateWithFlags(&P->ev_z1, cudaEventDisableTiming), "cudaEventCreate");
            P->bp_full = wsplit.full;
            P->zi_cols = wsplit.cols;
        }
    }
    // precision 2: the spectrum S is stored in BF16 (the NUFFT paths read
    // bfloat16 (re, im) pairs; the tensor-core exact-sum table takes the hi
    // planes of its operand only)
    d.s_bf16 = (P->precision == 2 && !(P->block_config == 4 && P->rt_tc)) ? 1 : 0;
    PL_CUDA(cudaDeviceSynchronize(), "plan setup");
    return PL_OK;
}

}  // namespace

// split: straight into the tensor-core range table's operand; s_bf16: S as
// bfloat16 (re, im) rows (precision 2 on the NUFFT paths)
static pl_status stage_zfft(pl_plan *P, const float2 *echo, cudaStream_t st, bool split,
                            int s_bf16) {
    // precision 2: a BF16 spectrum (the hi planes of the split operand only)
    const int bf16 = P->precision == 2 ? 1 : 0;
    if (P->fwd_fft && split)      // straight into the tensor-core range table's operand
        PL_CUDA(launch_fft_strided(echo, P->d_S, P->C, P->N, P->M, P->zplan, P->d_twz, -1, 1.0f,
                                   P->Np, 0, st, P->d_rtA, P->rt.Kp, nullptr, 0, bf16), "zfft");
    else if (P->fwd_fft)
        PL_CUDA(launch_fft_strided(echo, P->d_S, P->C, P->N, P->M, P->zplan, P->d_twz, -1, 1.0f,
                                   P->Np, 0, st, nullptr, 0, nullptr, 0, s_bf16), "zfft");
    else   // the tensor-core table's operand is split from an FP32 S (k_rt_prep)
        PL_CUDA(launch_dft_strided(echo, P->d_S, P->C, P->N, P->M, P->Np, P->d_Tfwd, 1.0f, st,
                                   nullptr, s_bf16), "zdft");
    return PL_OK;
}

pl_status pl_stage_zfft(pl_plan *P, const float2 *echo, cudaStream_t st) {
    if (P->check_nonfinite)
        PL_CUDA(launch_check_finite(echo, (size_t)P->C * P->N * P->M, P->d_err, st),
                "check_finite");
    return stage_zfft(P, echo, st, P->block_config == 4 && P->rt_tc, P->nd.s_bf16);
}

pl_status pl_stage_range_table(pl_plan *P, cudaStream_t st) {
    if (P->block_config == 4 && P->rt_tc) {
        PL_CUDA(launch_range_table_tc(P->rt, P->tmapA, P->tmapE, P->d_S, P->d_rtA,
                                      P->d_rtprod, P->d_table, P->nd.tc_cols / 2,
                                      P->nd.tc_planar, P->d_err, P->fwd_fft, st),
                "range_table_tc");
        return PL_OK;
    }
    const int fmt = P->block_config == 4 ? 4 : (P->precision >= 1 ? 1 : 0);
    PL_CUDA(launch_range_table(P->nd, P->fineplan, P->d_S, P->d_alpha, P->d_xg, P->d_dec,
                               P->d_twfine, P->d_table, fmt, st), "range_table");
    return PL_OK;
}

// Spectra of the back-projection's output: one per channel part, or one that
// all parts add into.
static int g_parts(const pl_plan *P) {
    return (P->block_config == 4 && !P->tc.g_atomic) ? P->tc.nsplit : 1;
}
static size_t g_bytes(const pl_plan *P) {
    return (size_t)P->Np * P->grid.nx * P->grid.ny * sizeof(float2);
}

pl_status pl_stage_backproject(pl_plan *P, cudaStream_t st) {
    if (P->block_config == 4) {
        if (P->tc.g_atomic) PL_CUDA(cudaMemsetAsync(P->d_G, 0, g_bytes(P), st), "zero G");
        PL_CUDA(launch_backproject_tc(P->bp, P->coef, P->tc, P->tmap, P->d_tgeo, P->d_kchl,
                                      P->d_G, P->d_err, st),
                "backproject_tc");
        return PL_OK;
    }
    PL_CUDA(launch_backproject(P->bp, P->coef, P->d_table, P->d_tgeo, P->d_kchl, P->d_G, st),
            "backproject");
    return PL_OK;
}

// The inverse z transform of G; `parts` = 2 adds the second channel part's
// spectrum as it loads the first.
static pl_status stage_zifft(pl_plan *P, float2 *image, cudaStream_t st, int parts) {
    const int P2 = P->grid.nx * P->grid.ny;
    const float2 *G2 = parts > 1 ? P->d_G + (size_t)P->Np * P2 : nullptr;
    if (P->inv_fft)
        PL_CUDA(launch_fft_strided(P->d_G, image, 1, P->Np, P2, P->zplan, P->d_twz, +1,
                                   1.0f / P->Np, P->grid.nz, P->inv_off, st, nullptr, 0, G2),
                "zifft");
    else if (P->zidft_tc)
        PL_CUDA(launch_zidft_tc(P->zt, &P->tmapZ, P->d_G, G2, image, P->d_err, st), "zidft_tc");
    else
        PL_CUDA(launch_dft_strided(P->d_G, image, 1, P->Np, P2, P->grid.nz, P->d_Tinv,
                                   1.0f / P->Np, st, G2), "zidft");
    return PL_OK;
}

pl_status pl_stage_zifft(pl_plan *P, float2 *image, cudaStream_t st) {
    return stage_zifft(P, image, st, g_parts(P));
}

// a5 + a6 with the back-projection's last partial wave beside the z-IFFT of
// the pixels the full waves finished (P->bp_full > 0). The last wave follows
// the full waves on the caller's stream, so its blocks are dispatched as soon
// as SMs free up; the transform of the finished pixels waits on an event on
// s_bp and takes the SMs the last wave leaves idle. Timing events (may be
// null): t[0], t[1] around the back-projection, t[2], t[3] around the z-IFFT
// left after it (the rest of the pixels, and the join).
static pl_status stage_bp_zifft_overlapped(pl_plan *P, float2 *image, cudaStream_t st,
                                           const cudaEvent_t (&t)[4]) {
    const int P2 = P->grid.nx * P->grid.ny;
    const int parts = g_parts(P);
    const float2 *G2 = parts > 1 ? P->d_G + (size_t)P->Np * P2 : nullptr;
    TcArgs a = P->tc;
    if (P->tc.g_atomic) {
        // G zeroed on the side stream, beside the caller's stream's z-FFT and
        // range table, after the previous execution's readers of G
        PL_CUDA(cudaStreamWaitEvent(st, P->ev_z1, 0), "cudaStreamWaitEvent");
    }
    if (t[0]) PL_CUDA(cudaEventRecord(t[0], st), "event");
    a.blk0 = 0;
    a.nblk = P->bp_full;
    PL_CUDA(launch_backproject_tc(P->bp, P->coef, a, P->tmap, P->d_tgeo, P->d_kchl, P->d_G,
                                  P->d_err, st), "backproject_tc (full waves)");
    PL_CUDA(cudaEventRecord(P->ev_bpA, st), "event");
    // Eq. (9) on the finished pixels [0, zi_cols), beside the last wave
    PL_CUDA(cudaStreamWaitEvent(P->s_bp, P->ev_bpA, 0), "cudaStreamWaitEvent");
    PL_CUDA(launch_fft_strided(P->d_G, image, 1, P->Np, P->zi_cols, P->zplan, P->d_twz, +1,
                               1.0f / P->Np, P->grid.nz, P->inv_off, P->s_bp, nullptr, 0, G2, P2),
            "zifft (finished pixels)");
    PL_CUDA(cudaEventRecord(P->ev_bpB, P->s_bp), "event");
    a.blk0 = P->bp_full;
    a.nblk = 0;
    PL_CUDA(launch_backproject_tc(P->bp, P->coef, a, P->tmap, P->d_tgeo, P->d_kchl, P->d_G,
                                  P->d_err, st), "backproject_tc (last wave)");
    if (t[1]) PL_CUDA(cudaEventRecord(t[1], st), "event");
    if (t[2]) PL_CUDA(cudaEventRecord(t[2], st), "event");
    const size_t c0 = (size_t)P->zi_cols;
    PL_CUDA(launch_fft_strided(P->d_G + c0, image + c0, 1, P->Np, P2 - P->zi_cols, P->zplan,
                               P->d_twz, +1, 1.0f / P->Np, P->grid.nz, P->inv_off, st, nullptr, 0,
                               G2 ? G2 + c0 : nullptr, P2),
            "zifft (rest)");
    PL_CUDA(cudaStreamWaitEvent(st, P->ev_bpB, 0), "cudaStreamWaitEvent");
    if (t[3]) PL_CUDA(cudaEventRecord(t[3], st), "event");
    return PL_OK;
}

namespace {

pl_status run(pl_plan *P, const float2 *echo, float2 *image, cudaStream_t st) {
    cudaEvent_t ev[PL_NUM_STAGES][2] = {};
    if (P->timing) {
        for (int sidx = 0; sidx < PL_NUM_STAGES; ++sidx) {
            ev[sidx][0] = P->next_event();
            ev[sidx][1] = P->next_event();
            if (!ev[sidx][0] || !ev[sidx][1]) return fail(PL_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    auto mark = [&](int sidx, int which) -> cudaError_t {
        if (!P->timing) return cudaSuccess;
        return cudaEventRecord(ev[sidx][which], st);
    };
    pl_status s;
    if (P->tc.g_atomic && P->bp_full > 0) {
        // the channel parts add into one spectrum: zero it on the side
        // stream, beside a1-a4 (the back-projection waits for it)
        PL_CUDA(cudaEventRecord(P->ev_z0, st), "event");
        PL_CUDA(cudaStreamWaitEvent(P->s_bp, P->ev_z0, 0), "cudaStreamWaitEvent");
        PL_CUDA(cudaMemsetAsync(P->d_G, 0, g_bytes(P), P->s_bp), "zero G");
        PL_CUDA(cudaEventRecord(P->ev_z1, P->s_bp), "event");
    }
    // a1: transform over the scan axis, Eq. (2)
    PL_CUDA(mark(0, 0), "event");
    if ((s = pl_stage_zfft(P, echo, st)) != PL_OK) return s;
    PL_CUDA(mark(0, 1), "event");
    // a2-a4: compensation + NUFFT spread + fine FFT + deconvolution, Eq. (8a)
    PL_CUDA(mark(1, 0), "event");
    if ((s = pl_stage_range_table(P, st)) != PL_OK) return s;
    PL_CUDA(mark(1, 1), "event");
    if (P->bp_full > 0) {
        // a5 + a6, the back-projection's last wave beside part of the z-IFFT
        const cudaEvent_t t[4] = {P->timing ? ev[2][0] : nullptr, P->timing ? ev[2][1] : nullptr,
                                  P->timing ? ev[3][0] : nullptr, P->timing ? ev[3][1] : nullptr};
        if ((s = stage_bp_zifft_overlapped(P, image, st, t)) != PL_OK) return s;
    } else {
        // a5: back-projection with the coherent channel sum, Eq. (8b)
        PL_CUDA(mark(2, 0), "event");
        if ((s = pl_stage_backproject(P, st)) != PL_OK) return s;
        PL_CUDA(mark(2, 1), "event");
        // a6: inverse transform over k_z, Eq. (9)
        PL_CUDA(mark(3, 0), "event");
        if ((s = pl_stage_zifft(P, image, st)) != PL_OK) return s;
        PL_CUDA(mark(3, 1), "event");
    }
    if (P->timing)
        for (int sidx = 0; sidx < PL_NUM_STAGES; ++sidx)
            P->recorded.push_back({sidx, {ev[sidx][0], ev[sidx][1]}});
    return PL_OK;
}

}  // namespace

pl_status pl_internal_fail(pl_status s, const char *msg) { return fail(s, msg); }
pl_status pl_internal_cuda_fail(cudaError_t e, const char *where) { return cuda_fail(e, where); }

// Tables of the comparison algorithms (first use only): kappa and k weights
// per (k_z, f), positions, scan heights and wavenumbers as float pairs.
static pl_status prepare_comparison(pl_plan *P) {
    if (P->cmp_ready) return PL_OK;
    auto pair = [](double v) {
        const float h = (float)v;
        return std::make_pair(h, (float)(v - (double)h));
    };
    std::vector<float4> chff(2 * (size_t)P->C);
    for (int c = 0; c < P->C; ++c) {
        const double *q = &P->h_chxy[4 * (size_t)c];
        auto xt = pair(q[0]), yt = pair(q[1]), xr = pair(q[2]), yr = pair(q[3]);
        chff[2 * c] = make_float4(xt.first, xt.second, yt.first, yt.second);
        chff[2 * c + 1] = make_float4(xr.first, xr.second, yr.first, yr.second);
    }
    std::vector<float2> zs(P->N), kff(P->M);
    for (int n = 0; n < P->N; ++n) {
        auto z = pair(P->z0s + n * P->dzs);
        zs[n] = make_float2(z.first, z.second);
    }
    bool uniform = P->M >= 2;
    const double dk = P->M >= 2 ? (P->h_k[P->M - 1] - P->h_k[0]) / (P->M - 1) : 0.0;
    for (int m = 0; m < P->M; ++m) {
        auto kv = pair(P->h_k[m]);
        kff[m] = make_float2(kv.first, kv.second);
        if (std::fabs(P->h_k[m] - (P->h_k[0] + m * dk)) > 1e-9 * P->h_k[m]) uniform = false;
    }
    size_t ws = 0;
    PL_CUDA(dalloc(&P->d_chff, chff.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_zs, zs.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kff, kff.size(), ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_kap, (size_t)P->Np * P->M, ws), "cudaMalloc");
    PL_CUDA(dalloc(&P->d_wum, (size_t)P->Np * P->M, ws), "cudaMalloc");
    PL_CUDA(cudaMemcpy(P->d_chff, chff.data(), chff.size() * sizeof(float4), cudaMemcpyHostToDevice),
            "copy");
    PL_CUDA(cudaMemcpy(P->d_zs, zs.data(), zs.size() * sizeof(float2), cudaMemcpyHostToDevice),
            "copy");
    PL_CUDA(cudaMemcpy(P->d_kff, kff.data(), kff.size() * sizeof(float2), cudaMemcpyHostToDevice),
            "copy");
    PL_CUDA(launch_setup_exact(P->mode, P->Np, P->dzs, P->M, P->d_k, P->d_kap, P->d_wum, 0),
            "setup_exact");
    PL_CUDA(cudaDeviceSynchronize(), "setup_exact");
    P->workspace += ws;
    ExactDesc &e = P->exact;
    e.mode = P->mode;
    e.n_chan = P->C;
    e.n_pad = P->Np;
    e.n_f = P->M;
    e.nx = P->grid.nx;
    e.ny = P->grid.ny;
    e.x0 = P->grid.x0;
    e.dx = P->grid.dx;
    e.y0 = P->grid.y0;
    e.dy = P->grid.dy;
    DirectDesc &d = P->direct;
    d.mode = P->mode;
    d.n_chan = P->C;
    d.n_scan = P->N;
    d.n_f = P->M;
    d.nx = P->grid.nx;
    d.ny = P->grid.ny;
    d.nz = P->grid.nz;
    d.uniform = uniform ? 1 : 0;
    d.x0 = P->grid.x0;
    d.dx = P->grid.dx;
    d.y0 = P->grid.y0;
    d.dy = P->grid.dy;
    d.z0 = P->grid.z0;
    d.dz = P->grid.dz;
    auto k0 = pair(P->h_k[0]), dkp = pair(dk);
    d.k0_hi = k0.first;
    d.k0_lo = k0.second;
    d.dk_hi = dkp.first;
    d.dk_lo = dkp.second;
    P->cmp_ready = true;
    return PL_OK;
}

// Deep copy of the creation inputs into P->inputs.
static void store_inputs(pl_plan *P, const pl_geometry *g, const pl_scan *s, const pl_freqs *f,
                         const pl_grid *gr, const pl_options *opt) {
    PlanInputs &in = P->inputs;
    in.g = *g;
    in.s = *s;
    in.f = *f;
    in.gr = *gr;
    in.has_opts = opt != nullptr;
    if (opt) in.o = *opt;
    in.elem_xy.assign(g->elem_xy, g->elem_xy + 2 * (size_t)g->n_elem);
    in.g.elem_xy = in.elem_xy.data();
    if (g->elem_section) {
        in.elem_section.assign(g->elem_section, g->elem_section + g->n_elem);
        in.g.elem_section = in.elem_section.data();
    }
    if (g->mode == 1 && g->n_pairs > 0) {
        in.pair_tx.assign(g->pair_tx, g->pair_tx + g->n_pairs);
        in.pair_rx.assign(g->pair_rx, g->pair_rx + g->n_pairs);
        in.g.pair_tx = in.pair_tx.data();
        in.g.pair_rx = in.pair_rx.data();
    }
    in.f_hz.assign(f->f_hz, f->f_hz + f->n);
    in.f.f_hz = in.f_hz.data();
}

extern "C" {

const char *pl_status_string(pl_status s) {
    switch (s) {
        case PL_OK: return "ok";
        case PL_ERR_ARG: return "invalid argument";
        case PL_ERR_GEOMETRY: return "invalid geometry";
        case PL_ERR_FREQ: return "invalid frequencies";
        case PL_ERR_EVANESCENT: return "all terms evanescent";
        case PL_ERR_NONFINITE: return "non-finite input";
        case PL_ERR_CUDA: return "CUDA error";
        case PL_ERR_OOM: return "out of device memory";
        case PL_ERR_TIMEOUT: return "device wait timed out";
        case PL_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *pl_last_error(void) { return g_err.c_str(); }

int pl_version(void) { return 200; }

pl_status pl_plan_create(pl_plan **out, const pl_geometry *geom, const pl_scan *scan,
                         const pl_freqs *freqs, const pl_grid *grid, const pl_options *opt) {
    if (!out) return fail(PL_ERR_ARG, "out is NULL");
    *out = nullptr;
    pl_status s = validate(geom, scan, freqs, grid);
    if (s != PL_OK) return s;
    pl_options o{};
    if (opt) o = *opt;
    // default kernel: the tensor-core back-projection where it applies, else
    // the FP32 kernels (a grid too coarse for its 32-row windows, other w)
    const int w = o.nufft_w ? o.nufft_w : 6;
    if (o.block_config == 0 && o.tile_u == 0 && (w == 4 || w == 6 || w == 8)) {
        pl_options ot = o;
        ot.block_config = 4;
        pl_plan *P = new (std::nothrow) pl_plan();
        if (!P) return fail(PL_ERR_OOM, "host allocation failed");
        s = build_plan(P, geom, scan, freqs, grid, &ot);
        g_fail_alloc_countdown = 0;
        if (s == PL_OK) {
            store_inputs(P, geom, scan, freqs, grid, opt);
            *out = P;
            return PL_OK;
        }
        delete P;
        if (s != PL_ERR_UNSUPPORTED) return s;
    }
    pl_plan *P = new (std::nothrow) pl_plan();
    if (!P) return fail(PL_ERR_OOM, "host allocation failed");
    s = build_plan(P, geom, scan, freqs, grid, &o);
    g_fail_alloc_countdown = 0;
    if (s != PL_OK) {
        delete P;
        return s;
    }
    store_inputs(P, geom, scan, freqs, grid, opt);
    *out = P;
    return PL_OK;
}

pl_status pl_plan_destroy(pl_plan *plan) {
    if (!plan) return fail(PL_ERR_ARG, "plan is NULL");
    delete plan;
    return PL_OK;
}

// A bounded wait of the tensor-core back-projection that ran out in an
// earlier execution (flags in mapped host memory: no synchronisation).
static pl_status take_device_timeout(pl_plan *plan) {
    if (!plan->h_err || *(volatile int *)plan->h_err == 0) return PL_OK;
    const int bits = *(volatile int *)plan->h_err;
    *(volatile int *)plan->h_err = 0;
    if (bits & PL_FLAG_NONFINITE)
        return fail(PL_ERR_NONFINITE, "the echo held NaN or Inf values (check_nonfinite)");
    char msg[96];
    std::snprintf(msg, sizeof msg,
                  "a bounded wait of the tensor-core kernels timed out (flags 0x%x)", bits);
    return fail(PL_ERR_TIMEOUT, msg);
}

pl_status pl_execute(pl_plan *plan, const void *echo_dev, void *image_dev, void *stream) {
    if (!plan || !echo_dev || !image_dev) return fail(PL_ERR_ARG, "NULL argument");
    pl_status s = take_device_timeout(plan);
    if (s != PL_OK) return s;
    return run(plan, (const float2 *)echo_dev, (float2 *)image_dev, (cudaStream_t)stream);
}

pl_status pl_execute_exact(pl_plan *plan, const void *echo_dev, void *image_dev, void *stream) {
    if (!plan || !echo_dev || !image_dev) return fail(PL_ERR_ARG, "NULL argument");
    pl_status s = prepare_comparison(plan);
    if (s != PL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the exact sum reads an FP32 spectrum whatever the plan's precision
    if ((s = stage_zfft(plan, (const float2 *)echo_dev, st, false, 0)) != PL_OK) return s;
    PL_CUDA(launch_exact_sum(plan->exact, plan->d_S, plan->d_kap, plan->d_wum, plan->d_chff,
                             plan->d_G, st),
            "exact_sum");
    return stage_zifft(plan, (float2 *)image_dev, st, 1);     // one whole spectrum
}

pl_status pl_execute_bp_direct(pl_plan *plan, const void *echo_dev, void *image_dev,
                               void *stream) {
    if (!plan || !echo_dev || !image_dev) return fail(PL_ERR_ARG, "NULL argument");
    pl_status s = prepare_comparison(plan);
    if (s != PL_OK) return s;
    PL_CUDA(launch_bp_direct(plan->direct, (const float2 *)echo_dev, plan->d_chff, plan->d_zs,
                             plan->d_kff, (float2 *)image_dev, (cudaStream_t)stream),
            "bp_direct");
    return PL_OK;
}

pl_status pl_execute_host(pl_plan *plan, const void *echo_host, void *image_host, void *stream) {
    if (!plan || !echo_host || !image_host) return fail(PL_ERR_ARG, "NULL argument");
    pl_status s0 = take_device_timeout(plan);
    if (s0 != PL_OK) return s0;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t in_bytes = (size_t)plan->C * plan->N * plan->M * sizeof(float2);
    const size_t out_bytes =
        (size_t)plan->grid.nx * plan->grid.ny * plan->grid.nz * sizeof(float2);
    if (!plan->d_echo_in) {
        PL_CUDA(cudaMalloc(&plan->d_echo_in, in_bytes), "cudaMalloc");
        PL_CUDA(cudaMalloc(&plan->d_img_out, out_bytes), "cudaMalloc");
        plan->workspace += in_bytes + out_bytes;
    }
    PL_CUDA(cudaMemcpyAsync(plan->d_echo_in, echo_host, in_bytes, cudaMemcpyHostToDevice, st),
            "copy echo");
    pl_status s = run(plan, plan->d_echo_in, plan->d_img_out, st);
    if (s != PL_OK) return s;
    PL_CUDA(cudaMemcpyAsync(image_host, plan->d_img_out, out_bytes, cudaMemcpyDeviceToHost, st),
            "copy image");
    PL_CUDA(cudaStreamSynchronize(st), "execute_host");
    return take_device_timeout(plan);
}

pl_status pl_execute_host_stream(pl_plan *plan, int n_scans, const void *const *echo_host,
                                 void *const *image_host, void *stream) {
    if (!plan || n_scans < 0 || (n_scans > 0 && (!echo_host || !image_host)))
        return fail(PL_ERR_ARG, "bad pl_execute_host_stream arguments");
    for (int i = 0; i < n_scans; ++i)
        if (!echo_host[i] || !image_host[i]) return fail(PL_ERR_ARG, "NULL scan buffer");
    pl_status s0 = take_device_timeout(plan);
    if (s0 != PL_OK) return s0;
    if (n_scans == 0) return PL_OK;
    const size_t in_bytes = (size_t)plan->C * plan->N * plan->M * sizeof(float2);
    const size_t out_bytes =
        (size_t)plan->grid.nx * plan->grid.ny * plan->grid.nz * sizeof(float2);
    if (!plan->d_echo_in) {
        PL_CUDA(cudaMalloc(&plan->d_echo_in, in_bytes), "cudaMalloc");
        PL_CUDA(cudaMalloc(&plan->d_img_out, out_bytes), "cudaMalloc");
        plan->workspace += in_bytes + out_bytes;
    }
    if (!plan->d_echo_in2) {
        PL_CUDA(cudaMalloc(&plan->d_echo_in2, in_bytes), "cudaMalloc");
        PL_CUDA(cudaMalloc(&plan->d_img_out2, out_bytes), "cudaMalloc");
        plan->workspace += in_bytes + out_bytes;
        PL_CUDA(cudaStreamCreateWithFlags(&plan->s_h2d, cudaStreamNonBlocking), "stream");
        PL_CUDA(cudaStreamCreateWithFlags(&plan->s_d2h, cudaStreamNonBlocking), "stream");
        for (int b = 0; b < 2; ++b) {
            PL_CUDA(cudaEventCreateWithFlags(&plan->ev_in[b], cudaEventDisableTiming), "event");
            PL_CUDA(cudaEventCreateWithFlags(&plan->ev_done[b], cudaEventDisableTiming), "event");
            PL_CUDA(cudaEventCreateWithFlags(&plan->ev_out[b], cudaEventDisableTiming), "event");
        }
        PL_CUDA(cudaEventCreateWithFlags(&plan->ev_start, cudaEventDisableTiming), "event");
    }
    cudaStream_t st = (cudaStream_t)stream;
    float2 *din[2] = {plan->d_echo_in, plan->d_echo_in2};
    float2 *dout[2] = {plan->d_img_out, plan->d_img_out2};
    // odd scans go to the twin plan on its own stream, so that consecutive
    // scans' kernels can share the device (one scan's back-projection leaves
    // SMs idle in its last wave; the other stages leave the tensor cores idle)
    pl_plan *pp[2] = {plan, plan};
    cudaStream_t sc[2] = {st, st};
    if (n_scans >= 2) {
        if (!plan->twin) {
            const PlanInputs &in = plan->inputs;
            pl_options to = in.o;
            to.debug_fail_alloc = 0;            // the test hook covers the caller's plan only
            pl_plan *T = nullptr;
            const pl_status s = pl_plan_create(&T, &in.g, &in.s, &in.f, &in.gr,
                                               in.has_opts ? &to : nullptr);
            if (s != PL_OK) return s;
            plan->twin = T;
            plan->workspace += T->workspace;
            PL_CUDA(cudaStreamCreateWithFlags(&plan->s_twin, cudaStreamNonBlocking), "stream");
        }
        if ((s0 = take_device_timeout(plan->twin)) != PL_OK) return s0;
        pp[1] = plan->twin;
        sc[1] = plan->s_twin;
    }
    // the copies and the twin's stream start after the caller's earlier work
    PL_CUDA(cudaEventRecord(plan->ev_start, st), "event");
    PL_CUDA(cudaStreamWaitEvent(plan->s_h2d, plan->ev_start, 0), "wait");
    PL_CUDA(cudaStreamWaitEvent(plan->s_d2h, plan->ev_start, 0), "wait");
    if (sc[1] != st) PL_CUDA(cudaStreamWaitEvent(sc[1], plan->ev_start, 0), "wait");
    // two-deep pipeline: the upload of scan i+1 and the download of scan i-1
    // run on the copy engines while scan i is reconstructed (on the stream of
    // its parity); scans i and i + 2 share a plan, a stream and the staging
    // pair, so each waits for the other's copies through events
    for (int i = 0; i < n_scans; ++i) {
        const int b = i & 1;
        cudaStream_t sb = sc[b];
        if (i >= 2) PL_CUDA(cudaStreamWaitEvent(plan->s_h2d, plan->ev_done[b], 0), "wait");
        PL_CUDA(cudaMemcpyAsync(din[b], echo_host[i], in_bytes, cudaMemcpyHostToDevice,
                                plan->s_h2d),
                "copy echo");
        PL_CUDA(cudaEventRecord(plan->ev_in[b], plan->s_h2d), "event");
        PL_CUDA(cudaStreamWaitEvent(sb, plan->ev_in[b], 0), "wait");
        if (i >= 2) PL_CUDA(cudaStreamWaitEvent(sb, plan->ev_out[b], 0), "wait");
        pl_status s = run(pp[b], din[b], dout[b], sb);
        if (s != PL_OK) return s;
        PL_CUDA(cudaEventRecord(plan->ev_done[b], sb), "event");
        PL_CUDA(cudaStreamWaitEvent(plan->s_d2h, plan->ev_done[b], 0), "wait");
        PL_CUDA(cudaMemcpyAsync(image_host[i], dout[b], out_bytes, cudaMemcpyDeviceToHost,
                                plan->s_d2h),
                "copy image");
        PL_CUDA(cudaEventRecord(plan->ev_out[b], plan->s_d2h), "event");
    }
    PL_CUDA(cudaStreamWaitEvent(st, plan->ev_out[(n_scans - 1) & 1], 0), "wait");
    PL_CUDA(cudaStreamSynchronize(st), "execute_host_stream");
    if (plan->twin && (s0 = take_device_timeout(plan->twin)) != PL_OK) {
        take_device_timeout(plan);                  // both plans' flags are taken
        return s0;
    }
    return take_device_timeout(plan);
}

pl_status pl_plan_get_info(const pl_plan *P, pl_info *info) {
    if (!P || !info) return fail(PL_ERR_ARG, "NULL argument");
    pl_info i{};
    i.mode = P->mode;
    i.n_chan = P->C;
    i.n_scan = P->N;
    i.n_pad = P->Np;
    i.n_f = P->M;
    i.nx = P->grid.nx;
    i.ny = P->grid.ny;
    i.nz = P->grid.nz;
    i.table_len = P->nd.L;
    i.fine_len = P->nd.fine;
    i.slab_rows = P->R;
    i.nufft_w = P->nd.w;
    i.nufft_sigma = P->sigma;
    i.table_h = P->nd.h;
    i.table_l0 = P->nd.l0;
    i.z_transform_fft = P->inv_fft ? 1 : 0;
    // z transform, range table (tensor cores: the products and the transpose,
    // plus the operand's preparation when the z transform is a DFT), the
    // back-projection, the inverse z transform
    i.launches_per_execute = (P->block_config == 4 && P->rt_tc) ? (P->fwd_fft ? 5 : 6) : 4;
    if (P->bp_full > 0) i.launches_per_execute += 2;   // a second back-projection and z-IFFT launch
    i.bp_launches = P->bp_full > 0 ? 2 : 1;
    i.workspace_bytes = P->workspace;
    i.updates_per_execute = (double)P->C * P->grid.nx * P->grid.ny * P->grid.nz * P->M;
    i.block_config = P->block_config;
    i.tile_u = P->tile_u;
    i.es_beta = (double)P->nd.beta;
    i.band_group = P->tile_u;
    if (P->block_config == 4) {
        i.table_layout = P->nd.tc_planar ? 3 : 2;
        i.table_cols = P->nd.tc_cols;
    } else {
        i.table_layout = P->precision >= 1 ? 1 : 0;
        i.table_cols = 0;
    }
    i.table_exact = (P->block_config == 4 && P->rt_tc) ? 1 : 0;
    i.precision = P->precision;
    i.sparse_products = (P->block_config == 4 && P->tc.sparse) ? 1 : 0;
    *info = i;
    return PL_OK;
}

pl_status pl_plan_workspace(pl_plan *P, int stage, void **dev_ptr, size_t *bytes) {
    if (!P || !dev_ptr || !bytes) return fail(PL_ERR_ARG, "NULL argument");
    switch (stage) {
        case PL_STAGE_ZFFT:
            *dev_ptr = P->d_S;
            *bytes = (size_t)P->C * P->Np * P->M * (P->nd.s_bf16 ? 4 : sizeof(float2));
            return PL_OK;
        case PL_STAGE_RANGE_TABLE:
            *dev_ptr = P->d_table;
            *bytes = P->table_bytes;
            return PL_OK;
        case PL_WS_RT_OPERAND_A:
        case PL_WS_RT_OPERAND_E:
            if (!(P->block_config == 4 && P->rt_tc)) break;
            if (stage == PL_WS_RT_OPERAND_A) {
                *dev_ptr = P->d_rtA;
                *bytes = (size_t)P->Np * 4 * P->C * P->rt.Kp * 2;
            } else {
                *dev_ptr = P->d_rtE;
                *bytes = (size_t)P->Np * 4 * P->rt.Lp * P->rt.Kp * 2;
            }
            return PL_OK;
        case PL_STAGE_BACKPROJECT:
            *dev_ptr = P->d_G;
            *bytes = (size_t)g_parts(P) * g_bytes(P);
            return PL_OK;
    }
    return fail(PL_ERR_ARG, "no workspace for this stage");
}

pl_status pl_plan_set_timing(pl_plan *P, int enable) {
    if (!P) return fail(PL_ERR_ARG, "plan is NULL");
    P->timing = enable != 0;
    P->recorded.clear();
    P->ev_next = 0;
    return PL_OK;
}

pl_status pl_plan_stage_times(pl_plan *P, double ms[PL_NUM_STAGES], int launches[PL_NUM_STAGES]) {
    if (!P || !ms || !launches) return fail(PL_ERR_ARG, "NULL argument");
    for (int s = 0; s < PL_NUM_STAGES; ++s) {
        ms[s] = 0.0;
        launches[s] = 0;
    }
    for (auto &r : P->recorded) {
        PL_CUDA(cudaEventSynchronize(r.second.second), "cudaEventSynchronize");
        float t = 0.f;
        PL_CUDA(cudaEventElapsedTime(&t, r.second.first, r.second.second), "cudaEventElapsedTime");
        ms[r.first] += t;
        launches[r.first] += 1;
    }
    P->recorded.clear();
    P->ev_next = 0;
    return PL_OK;
}

pl_status pl_synth_echo(int n_chan, const double *tx_xy, const double *rx_xy, double z0, double dz,
                        int n_scan, const double *f_hz, int n_f, int n_pts, const double *pts,
                        const double *amp, void *echo_dev, void *stream) {
    if (n_chan <= 0 || n_scan <= 0 || n_f <= 0 || n_pts < 0 || !tx_xy || !rx_xy || !f_hz ||
        !echo_dev || (n_pts > 0 && (!pts || !amp)))
        return fail(PL_ERR_ARG, "bad pl_synth_echo arguments");
    cudaStream_t st = (cudaStream_t)stream;
    // device copies of the caller's FP64 arrays (the kernel forms the ranges
    // in FP64)
    const size_t b_ch = sizeof(double) * 2 * n_chan, b_f = sizeof(double) * n_f;
    const size_t b_p = sizeof(double) * 3 * std::max(n_pts, 1);
    const size_t b_a = sizeof(double) * 2 * std::max(n_pts, 1);
    double *d_tx = nullptr, *d_rx = nullptr, *d_f = nullptr, *d_p = nullptr, *d_a = nullptr;
    cudaError_t e = cudaMalloc(&d_tx, b_ch);
    if (e == cudaSuccess) e = cudaMalloc(&d_rx, b_ch);
    if (e == cudaSuccess) e = cudaMalloc(&d_f, b_f);
    if (e == cudaSuccess) e = cudaMalloc(&d_p, b_p);
    if (e == cudaSuccess) e = cudaMalloc(&d_a, b_a);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tx, tx_xy, b_ch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rx, rx_xy, b_ch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_f, f_hz, b_f, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pts > 0)
        e = cudaMemcpyAsync(d_p, pts, sizeof(double) * 3 * n_pts, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pts > 0)
        e = cudaMemcpyAsync(d_a, amp, sizeof(double) * 2 * n_pts, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_synth_echo(n_chan, d_tx, d_rx, n_scan, z0, dz, n_f, d_f, n_pts, d_p, d_a,
                              (float2 *)echo_dev, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (double *q : {d_tx, d_rx, d_f, d_p, d_a})
        if (q) cudaFree(q);
    if (e != cudaSuccess) return cuda_fail(e, "pl_synth_echo");
    return PL_OK;
}

}  // extern "C"

pl_status pl_plan_take_timeout(pl_plan *plan) { return take_device_timeout(plan); }
