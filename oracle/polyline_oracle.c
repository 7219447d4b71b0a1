/*
 * FP64 CPU oracle for polyline-array hybrid reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark use it. It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Every routine here is the plain definition written out with nested loops,
 * in double precision, in the order of the paper:
 *   Wang, Li, Zhao, Sun, "Near-Field Millimeter-Wave Imaging via Arrays in the
 *   Shape of Polyline" (arXiv 2109.02842).
 * Equation numbers follow the printed numbering of that paper (Sec. II):
 *   (1) monostatic echo, (3) spectrum of the Green's function, (5) monostatic
 *   dispersion, (6)/(7) reduced model and its time-domain inversion,
 *   (8a)/(8b) filtered back-projection, (9) IFFT over k_z, (10) multistatic
 *   echo, (17)/(18) multistatic reduced model and dispersion, (19a)/(19b)
 *   multistatic filtered back-projection.
 *
 * Discrete conventions (the readings the paper leaves open):
 *   - scan positions z'_n, n < N; FT over z' with kernel exp(-j k_z z'),
 *     zero-padded to N_p >= N; k_z,u = 2*pi*ut/(N_p*dz) with ut = u for
 *     u < N_p/2 and u - N_p otherwise (the Nyquist bin is negative);
 *   - the k dk Jacobian of (7) is the weight k_m (dk is a constant, dropped);
 *   - evanescent terms (kappa^2 <= 0) are set to zero;
 *   - the z inverse transform is evaluated at arbitrary voxel heights z_p as
 *     (1/N_p) sum_u G_u exp(+j k_z,u (z_p - z'_0)).
 *
 * Complex arrays are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C0 299792458.0

static const double OR_TWO_PI = 6.283185307179586476925286766559;

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* wavenumber k = 2 pi f / c  (Sec. II-A, below Eq. (1)) */
static double or_wavenumber(double f_hz) { return OR_TWO_PI * f_hz / OR_C0; }

/* k_z of DFT bin u for an N_p-point transform at step dz (fftfreq order) */
double or_kz(int u, int n_pad, double dz)
{
    int ut = (2 * u < n_pad) ? u : u - n_pad;
    return OR_TWO_PI * (double)ut / ((double)n_pad * dz);
}

/*
 * Squared radial wavenumber.
 *   mode 0 (monostatic):  kappa^2 = 4 k^2 - k_z^2          Eq. (5)
 *   mode 1 (multistatic): kappa^2 = k^2 - k_z^2 / 4         Eq. (18)
 */
static double or_kappa_sq(int mode, double k, double kz)
{
    if (mode == 0) return 4.0 * k * k - kz * kz;
    return k * k - 0.25 * kz * kz;
}

/*
 * Echo synthesis, Eq. (1) (monostatic) and Eq. (10) (multistatic) for point
 * scatterers g = sum_t amp_t delta(r - r_t):
 *   s[c][n][m] = sum_t amp_t exp(-j k_m (R_T + R_R)),
 *   R_T = |r_t - (x_T, y_T, z'_n)|, R_R = |r_t - (x_R, y_R, z'_n)|.
 * A monostatic channel has its Tx and Rx at the same place, which gives
 * exp(-j 2 k R). No 1/R amplitude: the paper's model has none.
 *
 * tx_xy, rx_xy: [n_chan][2]; z_scan: [n_scan]; f_hz: [n_f];
 * pts: [n_pts][3]; amp: [n_pts][2] complex; out: [n_chan][n_scan][n_f][2].
 */
void or_synth_echo(int n_chan, const double *tx_xy, const double *rx_xy,
                   int n_scan, const double *z_scan, int n_f, const double *f_hz,
                   int n_pts, const double *pts, const double *amp, double *out)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < n_chan; ++c) {
        for (int n = 0; n < n_scan; ++n) {
            for (int m = 0; m < n_f; ++m) {
                double k = or_wavenumber(f_hz[m]);
                double acc_re = 0.0, acc_im = 0.0;
                for (int t = 0; t < n_pts; ++t) {
                    double dxt = pts[3 * t + 0] - tx_xy[2 * c + 0];
                    double dyt = pts[3 * t + 1] - tx_xy[2 * c + 1];
                    double dzz = pts[3 * t + 2] - z_scan[n];
                    double dxr = pts[3 * t + 0] - rx_xy[2 * c + 0];
                    double dyr = pts[3 * t + 1] - rx_xy[2 * c + 1];
                    double r_t = sqrt(dxt * dxt + dyt * dyt + dzz * dzz);
                    double r_r = sqrt(dxr * dxr + dyr * dyr + dzz * dzz);
                    double ph = -k * (r_t + r_r);
                    double cr = cos(ph), ci = sin(ph);
                    double ar = amp[2 * t + 0], ai = amp[2 * t + 1];
                    acc_re += ar * cr - ai * ci;
                    acc_im += ar * ci + ai * cr;
                }
                size_t o = (((size_t)c * n_scan + n) * n_f + m) * 2;
                out[o + 0] = acc_re;
                out[o + 1] = acc_im;
            }
        }
    }
}

/*
 * FT of the echo along the scan axis, Eq. (2), as a zero-padded DFT:
 *   S[c][u][m] = sum_{n<N} s[c][n][m] exp(-j 2 pi u n / N_p),  u < N_p.
 * The exponent index (u n mod N_p) is reduced exactly in integers.
 * s: [n_chan][n_scan][n_f][2]; S: [n_chan][n_pad][n_f][2].
 */
void or_zdft(int n_chan, int n_scan, int n_f, int n_pad, const double *s, double *S)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < n_chan; ++c) {
        for (int u = 0; u < n_pad; ++u) {
            for (int m = 0; m < n_f; ++m) {
                double acc_re = 0.0, acc_im = 0.0;
                for (int n = 0; n < n_scan; ++n) {
                    long long r = ((long long)u * n) % n_pad;
                    double ph = -OR_TWO_PI * (double)r / (double)n_pad;
                    double cr = cos(ph), ci = sin(ph);
                    size_t i = (((size_t)c * n_scan + n) * n_f + m) * 2;
                    double sr = s[i], si = s[i + 1];
                    acc_re += sr * cr - si * ci;
                    acc_im += sr * ci + si * cr;
                }
                size_t o = (((size_t)c * n_pad + u) * n_f + m) * 2;
                S[o] = acc_re;
                S[o + 1] = acc_im;
            }
        }
    }
}

/*
 * Time-domain inversion in the k_z domain with exact nonuniform sums.
 *   mode 0, Eq. (7):   G_u(x,y) = sum_c sum_m S[c][u][m] k_m exp(+j kappa_um rho_c)
 *   mode 1, Eq. (17)-(19): same with rho_c replaced by rho_T + rho_R and the
 *                      multistatic kappa of Eq. (18).
 * This is what the two steps (8a)/(8b) (and (19a)/(19b)) compute when the
 * range profile q(l) is evaluated exactly at l = rho (resp. rho_T + rho_R):
 * exp(j kappa' l) exp(j kappa_0 l) = exp(j kappa l). The sum over channels
 * runs over every section, which is the coherent sum over sections.
 *
 * tx_xy, rx_xy: [n_chan][2]; S: [n_chan][n_pad][n_f][2];
 * pix_xy: [n_pix][2]; G: [n_pad][n_pix][2].
 */
void or_hybrid_spectral(int mode, int n_chan, const double *tx_xy, const double *rx_xy,
                        int n_pad, double dz, int n_f, const double *f_hz,
                        const double *S, int n_pix, const double *pix_xy, double *G)
{
    #pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int u = 0; u < n_pad; ++u) {
        for (int p = 0; p < n_pix; ++p) {
            double kz = or_kz(u, n_pad, dz);
            double x = pix_xy[2 * p + 0], y = pix_xy[2 * p + 1];
            double acc_re = 0.0, acc_im = 0.0;
            for (int c = 0; c < n_chan; ++c) {
                double dxt = x - tx_xy[2 * c + 0], dyt = y - tx_xy[2 * c + 1];
                double rho_t = sqrt(dxt * dxt + dyt * dyt);
                double a;
                if (mode == 0) {
                    a = rho_t;
                } else {
                    double dxr = x - rx_xy[2 * c + 0], dyr = y - rx_xy[2 * c + 1];
                    a = rho_t + sqrt(dxr * dxr + dyr * dyr);
                }
                for (int m = 0; m < n_f; ++m) {
                    double k = or_wavenumber(f_hz[m]);
                    double ksq = or_kappa_sq(mode, k, kz);
                    if (ksq <= 0.0) continue; /* evanescent: set to zero */
                    double kappa = sqrt(ksq);
                    double ph = kappa * a;
                    double cr = cos(ph), ci = sin(ph);
                    size_t i = (((size_t)c * n_pad + u) * n_f + m) * 2;
                    double sr = S[i] * k, si = S[i + 1] * k;
                    acc_re += sr * cr - si * ci;
                    acc_im += sr * ci + si * cr;
                }
            }
            size_t o = ((size_t)u * n_pix + p) * 2;
            G[o] = acc_re;
            G[o + 1] = acc_im;
        }
    }
}

/*
 * Inverse transform over k_z, Eq. (9), evaluated at arbitrary voxel heights:
 *   g(x,y,z_p) = (1/N_p) sum_u G_u(x,y) exp(+j k_z,u (z_p - z'_0)).
 * G: [n_pad][n_pix][2]; z_vox: [n_z]; g: [n_z][n_pix][2].
 */
void or_zidft(int n_pad, double dz, double z0_scan, int n_pix, const double *G,
              int n_z, const double *z_vox, double *g)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int iz = 0; iz < n_z; ++iz) {
        for (int p = 0; p < n_pix; ++p) {
            double acc_re = 0.0, acc_im = 0.0;
            for (int u = 0; u < n_pad; ++u) {
                double ph = or_kz(u, n_pad, dz) * (z_vox[iz] - z0_scan);
                double cr = cos(ph), ci = sin(ph);
                size_t i = ((size_t)u * n_pix + p) * 2;
                acc_re += G[i] * cr - G[i + 1] * ci;
                acc_im += G[i] * ci + G[i + 1] * cr;
            }
            size_t o = ((size_t)iz * n_pix + p) * 2;
            g[o] = acc_re / (double)n_pad;
            g[o + 1] = acc_im / (double)n_pad;
        }
    }
}

/*
 * Direct back-projection (the comparison algorithm of Sec. III; the paper
 * prints no formula for it). Matched filter of Eq. (1)/(10) with the same
 * k weight as Eq. (7):
 *   g(x,y,z) = sum_c sum_n sum_m s[c][n][m] k_m exp(+j k_m (R_T + R_R)).
 * vox: [n_vox][3]; g: [n_vox][2].
 */
void or_bp_direct(int n_chan, const double *tx_xy, const double *rx_xy,
                  int n_scan, const double *z_scan, int n_f, const double *f_hz,
                  const double *s, int n_vox, const double *vox, double *g)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < n_vox; ++v) {
        double x = vox[3 * v + 0], y = vox[3 * v + 1], z = vox[3 * v + 2];
        double acc_re = 0.0, acc_im = 0.0;
        for (int c = 0; c < n_chan; ++c) {
            double dxt = x - tx_xy[2 * c + 0], dyt = y - tx_xy[2 * c + 1];
            double dxr = x - rx_xy[2 * c + 0], dyr = y - rx_xy[2 * c + 1];
            for (int n = 0; n < n_scan; ++n) {
                double dzz = z - z_scan[n];
                double r_t = sqrt(dxt * dxt + dyt * dyt + dzz * dzz);
                double r_r = sqrt(dxr * dxr + dyr * dyr + dzz * dzz);
                for (int m = 0; m < n_f; ++m) {
                    double k = or_wavenumber(f_hz[m]);
                    double ph = k * (r_t + r_r);
                    double cr = cos(ph), ci = sin(ph);
                    size_t i = (((size_t)c * n_scan + n) * n_f + m) * 2;
                    double sr = s[i] * k, si = s[i + 1] * k;
                    acc_re += sr * cr - si * ci;
                    acc_im += sr * ci + si * cr;
                }
            }
        }
        g[2 * v] = acc_re;
        g[2 * v + 1] = acc_im;
    }
}

/*
 * Range profile of step (8a) / (19a), evaluated exactly at the given ranges:
 *   q_{c,u}(l) = sum_m S[c][u][m] k_m exp(+j kappa'_um l),
 *   kappa' = kappa - kappa_0, kappa_0 = kappa(k_0, k_z), k_0 = min k.
 * Used to check the nonuniform FFT stage on its own.
 * S: [n_chan][n_pad][n_f][2]; l: [n_l]; q: [n_l][2] for one (c, u).
 */
void or_range_profile(int mode, int n_pad, double dz, int n_f, const double *f_hz,
                      const double *S, int c, int u, int n_l, const double *l, double *q)
{
    double kz = or_kz(u, n_pad, dz);
    double kmin = or_wavenumber(f_hz[0]);
    for (int m = 1; m < n_f; ++m) {
        double km = or_wavenumber(f_hz[m]);
        if (km < kmin) kmin = km;
    }
    double k0sq = or_kappa_sq(mode, kmin, kz);
    double kappa0 = k0sq > 0.0 ? sqrt(k0sq) : 0.0;
    for (int i = 0; i < n_l; ++i) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int m = 0; m < n_f; ++m) {
            double k = or_wavenumber(f_hz[m]);
            double ksq = or_kappa_sq(mode, k, kz);
            if (ksq <= 0.0) continue;
            double ph = (sqrt(ksq) - kappa0) * l[i];
            double cr = cos(ph), ci = sin(ph);
            size_t s_i = (((size_t)c * n_pad + u) * n_f + m) * 2;
            double sr = S[s_i] * k, si = S[s_i + 1] * k;
            acc_re += sr * cr - si * ci;
            acc_im += sr * ci + si * cr;
        }
        q[2 * i] = acc_re;
        q[2 * i + 1] = acc_im;
    }
}
