// Scene simulation (input synthesis for benchmarks and training data, not a
// reconstruction step): echo of point scatterers, Eq. (1) / Eq. (10),
//   echo[c][n][m] = sum_t amp_t exp(-j k_m (R_T + R_R)).
// Thread = (channel, scan position, 16 frequencies); points staged in shared
// memory in chunks.
//
// Precision: the phase k R reaches ~1.5e3 rad, so FP32 ranges (ulp ~1e-7 m)
// would already cost ~1e-4 rad. The range R_T + R_R of every (point, channel,
// scan position) is formed in FP64 from the FP64 inputs and kept as a float
// pair (hi + lo); each k_m R is a float-float product reduced modulo 2 pi with
// a two-constant 2 pi, so the FP32 sin/cos sees an argument within ~[-pi, pi]
// carrying ~1e-6 rad of error.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kMC = 16;       // frequencies per thread
constexpr int kPts = 128;     // points per shared-memory chunk
constexpr float kTwoPiHi = 6.28318548202514648f;    // float(2 pi)
constexpr float kTwoPiLo = -1.7484556e-7f;          // 2 pi - float(2 pi)
constexpr float kInvTwoPi = 0.159154943091895336f;

// -(kh + kl)(rh + rl) reduced modulo 2 pi
__device__ __forceinline__ float neg_phase(float kh, float kl, float rh, float rl) {
    const float p = kh * rh;
    float e = fmaf(kh, rh, -p);
    e = fmaf(kh, rl, e);
    e = fmaf(kl, rh, e);
    const float n = rintf(p * kInvTwoPi);
    float r = fmaf(-n, kTwoPiHi, p);
    r = fmaf(-n, kTwoPiLo, r);
    return -(r + e);
}

__global__ void __launch_bounds__(128)
k_synth_echo(int n_chan, const double *__restrict__ tx, const double *__restrict__ rx,
             int n_scan, double z0, double dz, int n_f, const double *__restrict__ f_hz,
             int n_pts, const double *__restrict__ pts, const double *__restrict__ amp,
             float2 *__restrict__ echo) {
    __shared__ double sp[kPts][3];
    __shared__ float2 sa[kPts];
    const int n_mc = (n_f + kMC - 1) / kMC;
    const long long total = (long long)n_chan * n_scan * n_mc;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = tid < total;
    int c = 0, n = 0, mc = 0;
    if (live) {
        mc = (int)(tid % n_mc);
        const long long cn = tid / n_mc;
        n = (int)(cn % n_scan);
        c = (int)(cn / n_scan);
    }
    const double xt = live ? tx[2 * c] : 0.0, yt = live ? tx[2 * c + 1] : 0.0;
    const double xr = live ? rx[2 * c] : 0.0, yr = live ? rx[2 * c + 1] : 0.0;
    const double zs = z0 + n * dz;
    float kh[kMC], kl[kMC];
    float2 acc[kMC];
#pragma unroll
    for (int q = 0; q < kMC; ++q) {
        const int m = mc * kMC + q;
        const double k = (live && m < n_f) ? PL_TWO_PI * f_hz[m] / PL_C0 : 0.0;
        kh[q] = (float)k;
        kl[q] = (float)(k - (double)kh[q]);
        acc[q] = make_float2(0.f, 0.f);
    }
    for (int t0 = 0; t0 < n_pts; t0 += kPts) {
        const int nt = min(kPts, n_pts - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            sp[i][0] = pts[3 * (size_t)(t0 + i)];
            sp[i][1] = pts[3 * (size_t)(t0 + i) + 1];
            sp[i][2] = pts[3 * (size_t)(t0 + i) + 2];
            sa[i] = make_float2((float)amp[2 * (size_t)(t0 + i)],
                                (float)amp[2 * (size_t)(t0 + i) + 1]);
        }
        __syncthreads();
        if (!live) continue;
        for (int i = 0; i < nt; ++i) {
            const double dzz = sp[i][2] - zs;
            const double dxt = sp[i][0] - xt, dyt = sp[i][1] - yt;
            const double dxr = sp[i][0] - xr, dyr = sp[i][1] - yr;
            const double rs = sqrt(dxt * dxt + dyt * dyt + dzz * dzz) +
                              sqrt(dxr * dxr + dyr * dyr + dzz * dzz);
            const float rh = (float)rs, rl = (float)(rs - (double)rh);
            const float2 a = sa[i];
#pragma unroll
            for (int qq = 0; qq < kMC; ++qq) {
                float s, co;
                __sincosf(neg_phase(kh[qq], kl[qq], rh, rl), &s, &co);
                acc[qq].x += a.x * co - a.y * s;
                acc[qq].y += a.x * s + a.y * co;
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int q = 0; q < kMC; ++q) {
        const int m = mc * kMC + q;
        if (m < n_f) echo[((size_t)c * n_scan + n) * n_f + m] = acc[q];
    }
}

}  // namespace

cudaError_t launch_synth_echo(int n_chan, const double *tx_xy, const double *rx_xy, int n_scan,
                              double z0, double dz, int n_f, const double *f_hz, int n_pts,
                              const double *pts, const double *amp, float2 *echo,
                              cudaStream_t st) {
    const long long total = (long long)n_chan * n_scan * ((n_f + kMC - 1) / kMC);
    const int blocks = (int)((total + 127) / 128);
    k_synth_echo<<<blocks, 128, 0, st>>>(n_chan, tx_xy, rx_xy, n_scan, z0, dz, n_f, f_hz, n_pts,
                                         pts, amp, echo);
    return cudaGetLastError();
}
