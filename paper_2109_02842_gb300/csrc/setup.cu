// Plan-time tables: everything that depends only on the geometry, the scan
// and the band, computed once per plan on the GPU in double precision.
//
// For bin u (k_z,u) and frequency m (k_m), Sec. II-A/B:
//   kappa_um = sqrt(4 k_m^2 - k_z,u^2)      monostatic, Eq. (5)
//   kappa_um = sqrt(k_m^2 - k_z,u^2 / 4)    multistatic, Eq. (18)
// terms with kappa^2 <= 0 are evanescent and dropped.
//
// Step (8a) is an inverse transform from the nonuniform kappa' to range l.
// It is evaluated as a type-3 nonuniform FFT (Lee & Greengard, SIAM Rev. 47
// (2005); Barnett et al., SIAM J. Sci. Comput. 41 (2019)) on a range grid
// l_i = l0 + i h, i < L, h = 2 pi / (sigma K):
//   q(l) e^{j kappa_c l} = sum_m c_m e^{j kappa_m l}
//   ~= h e^{j kappa_c l} sum_i phi(l - l_i) b_i,
//   b_i = sum_m (c_m / phihat(kappa''_m)) e^{j kappa''_m l_i},
// with kappa''= kappa - kappa_c centred on the band of bin u, phi the ES
// kernel of width w cells and phihat its Fourier transform. The carrier
// e^{j kappa_c l} plays the role of e^{j kappa_0 rho} in Eq. (8b): the paper's
// split kappa = kappa_0 + kappa' with the reference moved to the band centre,
// which halves the band the interpolation has to resolve.
// b_i itself is a type-1 transform (nonuniform sources -> uniform rows),
// computed by spreading onto a fine periodic grid, an FFT, and division by
// the spreading kernel's transform (range_table.cu).
#include <climits>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace {

__device__ __forceinline__ double kz_of(int u, int n_pad, double dz) {
    const int ut = (2 * u < n_pad) ? u : u - n_pad;
    return PL_TWO_PI * (double)ut / ((double)n_pad * dz);
}

__device__ __forceinline__ double kappa_sq(int mode, double k, double kz) {
    return mode == 0 ? 4.0 * k * k - kz * kz : k * k - 0.25 * kz * kz;
}

// Pass 1: the live kappa band [lo, hi] of every bin (lo < 0: no live term).
__global__ void k_setup_kz_bins(int mode, int n_pad, double dz, int n_f, const double *k,
                                double *band) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_pad) return;
    const double kz = kz_of(u, n_pad, dz);
    double lo = -1.0, hi = -1.0;
    for (int m = 0; m < n_f; ++m) {
        const double q = kappa_sq(mode, k[m], kz);
        if (q <= 0.0) continue;
        const double kap = sqrt(q);
        if (lo < 0.0) { lo = hi = kap; }
        lo = fmin(lo, kap);
        hi = fmax(hi, kap);
    }
    band[2 * u] = lo;
    band[2 * u + 1] = hi;
}

// Pass 2: centre and span of the band of every bin's group of `group` bins.
__global__ void k_setup_kz(int n_pad, int group, const double *band, double *kc, float2 *kc_hl,
                           double *kspan) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_pad) return;
    const int g0 = u / group * group, g1 = min(g0 + group, n_pad);
    double lo = 0.0, hi = 0.0;
    bool any = false;
    for (int v = g0; v < g1; ++v) {
        if (band[2 * v] < 0.0) continue;
        if (!any) { lo = band[2 * v]; hi = band[2 * v + 1]; any = true; }
        lo = fmin(lo, band[2 * v]);
        hi = fmax(hi, band[2 * v + 1]);
    }
    kc[u] = any ? 0.5 * (lo + hi) : 0.0;
    const float kh = (float)kc[u];
    kc_hl[u] = make_float2(kh, (float)(kc[u] - (double)kh));
    kspan[u] = any ? hi - lo : 0.0;
}

// phihat(kappa) / h = 2 * int_0^{w/2} ES(t) cos(kappa h t) dt by Gauss-Legendre
// nodes gl_x (on [0,1]) and weights gl_w.
__device__ double es_transform(double omega, int w, double beta, const double *gl_x,
                               const double *gl_w, int n_gl) {
    const double half = 0.5 * w;
    double s = 0.0;
    for (int i = 0; i < n_gl; ++i) {
        const double t = half * gl_x[i];
        s += gl_w[i] * es_kernel_d(t, 2.0 / w, beta) * cos(omega * t);
    }
    return 2.0 * half * s;
}

__global__ void k_setup_sources(NufftDesc d, double dz, const double *k, const double *kc,
                                const double *gl_x, const double *gl_w, int n_gl, float *xg,
                                float2 *alpha) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= d.n_pad * d.n_f) return;
    const int u = idx / d.n_f;
    const int m = idx - u * d.n_f;
    const double kz = kz_of(u, d.n_pad, dz);
    const double q = kappa_sq(d.mode, k[m], kz);
    if (q <= 0.0) {            // evanescent: no source
        xg[idx] = 0.0f;
        alpha[idx] = make_float2(0.f, 0.f);
        return;
    }
    const double kpp = sqrt(q) - kc[u];                // kappa'' in [-K/2, K/2]
    const double theta = kpp * d.h;                    // radians per table row
    xg[idx] = (float)(theta * d.fine / PL_TWO_PI);     // position on the fine grid
    const double phihat = d.h * es_transform(theta, d.w, d.beta, gl_x, gl_w, n_gl);
    // c_m = S k_m (the k dk weight of Eq. 7); centre the type-1 output index
    // at row L/2 and put row 0 at l0.
    const double ph = kpp * (d.l0 + d.h * (double)(d.L / 2));
    const double red = ph - PL_TWO_PI * rint(ph / PL_TWO_PI);
    // the interpolation's factor h is folded in here as well
    const double mag = d.h * k[m] / phihat;
    alpha[idx] = make_float2((float)(mag * cos(red)), (float)(mag * sin(red)));
}

__global__ void k_setup_deconv(NufftDesc d, const double *gl_x, const double *gl_w, int n_gl,
                               float *dec) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.L) return;
    const int j = i - d.L / 2;
    const double omega = PL_TWO_PI * (double)j / (double)d.fine;
    dec[i] = (float)(1.0 / es_transform(omega, d.w1, d.beta1, gl_x, gl_w, n_gl));
}

__global__ void k_twiddles(int n, int count, int sgn, float2 *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    out[k] = make_float2((float)c, (float)(sgn * s));
}

__global__ void k_dft_matrix_fwd(int n_pad, int n_scan, float2 *T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pad * n_scan) return;
    const int u = idx / n_scan;
    const int n = idx - u * n_scan;
    const long long r = ((long long)u * n) % n_pad;
    double s, c;
    sincospi(2.0 * (double)r / (double)n_pad, &s, &c);
    T[idx] = make_float2((float)c, (float)(-s));
}

__global__ void k_dft_matrix_inv(int n_pad, double dz, double z0_scan, int nz, double zv0,
                                 double dzv, float2 *T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nz * n_pad) return;
    const int p = idx / n_pad;
    const int u = idx - p * n_pad;
    const double ph = kz_of(u, n_pad, dz) * (zv0 + p * dzv - z0_scan);
    const double red = ph - PL_TWO_PI * rint(ph / PL_TWO_PI);
    T[idx] = make_float2((float)cos(red), (float)sin(red));
}

// Geometry of every (tile_px x 16 pixel tile, channel) for the back-projection.
__global__ void k_setup_tile_geo(BpDesc p, int ntx, int nty, const double *ch_xy, TileGeo *out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ntx * nty * p.n_chan) return;
    const int c = (int)(idx % p.n_chan);
    const int tile = (int)(idx / p.n_chan);
    const int tx = tile % ntx, ty = tile / ntx;
    const int TX = p.tile_px, TY = p.tile_py;
    const double xc = p.x0 + (tx * TX + 0.5 * (TX - 1)) * p.dx;
    const double yc = p.y0 + (ty * TY + 0.5 * (TY - 1)) * p.dy;
    const double dxt = xc - ch_xy[4 * c + 0], dyt = yc - ch_xy[4 * c + 1];
    const double rt = sqrt(dxt * dxt + dyt * dyt);
    double a = rt;
    TileGeo g;
    g.dxt = (float)dxt; g.dyt = (float)dyt; g.rt = (float)rt;
    g.dxr = g.dyr = g.rr = 0.f;
    if (p.mode == 1) {
        const double dxr = xc - ch_xy[4 * c + 2], dyr = yc - ch_xy[4 * c + 3];
        const double rr = sqrt(dxr * dxr + dyr * dyr);
        a += rr;
        g.dxr = (float)dxr; g.dyr = (float)dyr; g.rr = (float)rr;
    }
    int ilo = (int)floor((a - p.l0) / p.h - 0.5 * (p.R - 1));
    ilo = max(0, min(ilo, p.L - p.R));
    g.ilo = ilo;
    g.off = (float)(a - (p.l0 + ilo * p.h));
    g.a_hi = (float)a;
    g.a_lo = (float)(a - (double)g.a_hi);
    g.pad0 = g.pad1 = 0.f;
    out[idx] = g;
}

// Window of every (16 x 8 tile, channel) for the tensor-core back-projection:
// i_lo = the lowest first tap ceil(pos - w/2) over the tile's pixels (pos in
// table rows, FP64, with a 1e-3-row margin against the kernel's FP32
// rounding); stats[0] collects the rows the window must span, stats[1] the
// largest i_lo.
__global__ void k_setup_tile_geo_tc(BpDesc p, int ntx, int nty, const double *ch_xy, TileGeo *out,
                                    int *stats) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ntx * nty * p.n_chan) return;
    const int c = (int)(idx % p.n_chan);
    const int tile = (int)(idx / p.n_chan);
    const int tx = tile % ntx, ty = tile / ntx;
    const int TX = p.tile_px, TY = p.tile_py;
    const double xT = ch_xy[4 * c + 0], yT = ch_xy[4 * c + 1];
    const double xR = ch_xy[4 * c + 2], yR = ch_xy[4 * c + 3];
    auto range = [&](double x, double y) {
        double a = sqrt((x - xT) * (x - xT) + (y - yT) * (y - yT));
        if (p.mode == 1) a += sqrt((x - xR) * (x - xR) + (y - yR) * (y - yR));
        return a;
    };
    const double xc = p.x0 + (tx * TX + 0.5 * (TX - 1)) * p.dx;
    const double yc = p.y0 + (ty * TY + 0.5 * (TY - 1)) * p.dy;
    const double half = 0.5 * p.w;
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int j = 0; j < TY; ++j)
        for (int i = 0; i < TX; ++i) {
            const double pos = (range(p.x0 + (tx * TX + i) * p.dx, p.y0 + (ty * TY + j) * p.dy) -
                                p.l0) / p.h;
            lo = min(lo, (long long)ceil(pos - half - 1e-3));
            hi = max(hi, (long long)ceil(pos - half + 1e-3) + p.w);
        }
    const int ilo = (int)max(lo, 0ll);
    TileGeo g;
    const double dxt = xc - xT, dyt = yc - yT, rt = sqrt(dxt * dxt + dyt * dyt);
    double a = rt;
    g.dxt = (float)dxt; g.dyt = (float)dyt; g.rt = (float)rt;
    g.dxr = g.dyr = g.rr = 0.f;
    if (p.mode == 1) {
        const double dxr = xc - xR, dyr = yc - yR, rr = sqrt(dxr * dxr + dyr * dyr);
        a += rr;
        g.dxr = (float)dxr; g.dyr = (float)dyr; g.rr = (float)rr;
    }
    g.ilo = ilo;
    g.off = (float)(a - (p.l0 + ilo * p.h));
    g.a_hi = (float)a;
    g.a_lo = (float)(a - (double)g.a_hi);
    g.pad0 = g.pad1 = 0.f;
    out[idx] = g;
    atomicMax(&stats[0], (int)(hi - ilo));
    atomicMax(&stats[1], ilo);
}

// kappa (float pair) and the k weight of every (k_z bin, frequency) for the
// exact sum; both zero where the term is evanescent.
__global__ void k_setup_exact(int mode, int n_pad, double dz, int n_f, const double *k,
                              float2 *kap, float *wum) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_pad * n_f) return;
    const int u = idx / n_f, m = idx - u * n_f;
    const double q = kappa_sq(mode, k[m], kz_of(u, n_pad, dz));
    if (q <= 0.0) {
        kap[idx] = make_float2(0.f, 0.f);
        wum[idx] = 0.f;
        return;
    }
    const double kp = sqrt(q);
    const float h = (float)kp;
    kap[idx] = make_float2(h, (float)(kp - (double)h));
    wum[idx] = (float)k[m];
}

inline int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_setup_tile_geo_tc(const BpDesc &p, const double *ch_xy, TileGeo *tgeo,
                                     int *stats, cudaStream_t st) {
    const int ntx = (p.nx + p.tile_px - 1) / p.tile_px, nty = (p.ny + p.tile_py - 1) / p.tile_py;
    k_setup_tile_geo_tc<<<blocks((long long)ntx * nty * p.n_chan, 128), 128, 0, st>>>(
        p, ntx, nty, ch_xy, tgeo, stats);
    return cudaGetLastError();
}

cudaError_t launch_setup_exact(int mode, int n_pad, double dz, int n_f, const double *k,
                               float2 *kap, float *wum, cudaStream_t st) {
    k_setup_exact<<<blocks((long long)n_pad * n_f, 128), 128, 0, st>>>(mode, n_pad, dz, n_f, k,
                                                                      kap, wum);
    return cudaGetLastError();
}

cudaError_t launch_setup_kz(int mode, int n_pad, double dz, int n_f, const double *k, int group,
                            double *band, double *kc, float2 *kc_hl, double *kspan,
                            cudaStream_t st) {
    k_setup_kz_bins<<<blocks(n_pad, 128), 128, 0, st>>>(mode, n_pad, dz, n_f, k, band);
    k_setup_kz<<<blocks(n_pad, 128), 128, 0, st>>>(n_pad, group < 1 ? 1 : group, band, kc, kc_hl,
                                                   kspan);
    return cudaGetLastError();
}

cudaError_t launch_setup_sources(const NufftDesc &d, double dz, const double *k,
                                 const double *kc, const double *gl_x, const double *gl_w,
                                 int n_gl, float *xg, float2 *alpha, cudaStream_t st) {
    k_setup_sources<<<blocks((long long)d.n_pad * d.n_f, 128), 128, 0, st>>>(
        d, dz, k, kc, gl_x, gl_w, n_gl, xg, alpha);
    return cudaGetLastError();
}

cudaError_t launch_setup_deconv(const NufftDesc &d, const double *gl_x, const double *gl_w,
                                int n_gl, float *dec, cudaStream_t st) {
    k_setup_deconv<<<blocks(d.L, 128), 128, 0, st>>>(d, gl_x, gl_w, n_gl, dec);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(int n, int count, int sgn, float2 *out, cudaStream_t st) {
    k_twiddles<<<blocks(count, 128), 128, 0, st>>>(n, count, sgn, out);
    return cudaGetLastError();
}

cudaError_t launch_dft_matrix_fwd(int n_pad, int n_scan, float2 *T, cudaStream_t st) {
    k_dft_matrix_fwd<<<blocks((long long)n_pad * n_scan, 128), 128, 0, st>>>(n_pad, n_scan, T);
    return cudaGetLastError();
}

cudaError_t launch_dft_matrix_inv(int n_pad, double dz, double z0_scan, int nz, double zv0,
                                  double dzv, float2 *T, cudaStream_t st) {
    k_dft_matrix_inv<<<blocks((long long)nz * n_pad, 128), 128, 0, st>>>(n_pad, dz, z0_scan, nz,
                                                                       zv0, dzv, T);
    return cudaGetLastError();
}

cudaError_t launch_setup_tile_geo(const BpDesc &p, const double *ch_xy, TileGeo *tgeo,
                                  cudaStream_t st) {
    const int ntx = (p.nx + p.tile_px - 1) / p.tile_px, nty = (p.ny + p.tile_py - 1) / p.tile_py;
    k_setup_tile_geo<<<blocks((long long)ntx * nty * p.n_chan, 128), 128, 0, st>>>(p, ntx, nty,
                                                                                   ch_xy, tgeo);
    return cudaGetLastError();
}
