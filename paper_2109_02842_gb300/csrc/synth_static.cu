// Allocation-free variant of the scene-synthesis entry point.
//
// pl_synth_echo copies the caller's channel positions, frequencies and point
// list to device buffers it allocates with cudaMalloc for every call. Some
// callers cannot do that: code that runs while another component owns the
// device allocator, memory-capped or real-time services that must not touch
// the allocator after start-up, or code that only holds pre-registered memory.
// pl_synth_echo_static gives them the same result using a fixed scratch
// array that lives in this file as a static __device__ variable; the caller
// still passes the inputs (host) and the output (device).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/polyline.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kMaxChan = PL_STATIC_MAX_CHANNELS;
constexpr int kMaxFreq = PL_STATIC_MAX_FREQS;
constexpr int kMaxPts = PL_STATIC_MAX_POINTS;

// Byte offsets inside the scratch array: device copies of the caller's FP64
// arrays, in the layouts the synthesis kernel reads directly.
constexpr size_t kRawTx = 0;
constexpr size_t kRawRx = kRawTx + sizeof(double) * 2 * kMaxChan;
constexpr size_t kRawF = kRawRx + sizeof(double) * 2 * kMaxChan;
constexpr size_t kRawPts = kRawF + sizeof(double) * kMaxFreq;
constexpr size_t kRawAmp = kRawPts + sizeof(double) * 3 * kMaxPts;
constexpr size_t kScratchBytes = kRawAmp + sizeof(double) * 2 * kMaxPts;

// The scratch. Every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_synth_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[256] = {};

// Device address of the scratch for the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_synth_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pl_status pl_synth_echo_static(int n_chan, const double *tx_xy, const double *rx_xy,
                                          double z0, double dz, int n_scan, const double *f_hz,
                                          int n_f, int n_pts, const double *pts,
                                          const double *amp, void *echo_dev, void *stream) {
    if (n_chan <= 0 || n_scan <= 0 || n_f <= 0 || n_pts < 0 || !tx_xy || !rx_xy || !f_hz ||
        !echo_dev || (n_pts > 0 && (!pts || !amp)))
        return pl_internal_fail(PL_ERR_ARG, "bad pl_synth_echo_static arguments");
    if (n_chan > kMaxChan || n_f > kMaxFreq || n_pts > kMaxPts)
        return pl_internal_fail(PL_ERR_ARG,
                                "pl_synth_echo_static: sizes exceed the static scratch "
                                "(at most PL_STATIC_MAX_CHANNELS channels, "
                                "PL_STATIC_MAX_FREQS frequencies, PL_STATIC_MAX_POINTS points)");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kRawTx, tx_xy, sizeof(double) * 2 * n_chan,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kRawRx, rx_xy, sizeof(double) * 2 * n_chan,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kRawF, f_hz, sizeof(double) * n_f, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pts > 0)
        e = cudaMemcpyAsync(base + kRawPts, pts, sizeof(double) * 3 * n_pts,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_pts > 0)
        e = cudaMemcpyAsync(base + kRawAmp, amp, sizeof(double) * 2 * n_pts,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const double *sb = reinterpret_cast<const double *>(base);
        e = launch_synth_echo(n_chan, sb + kRawTx / 8, sb + kRawRx / 8, n_scan, z0, dz, n_f,
                              sb + kRawF / 8, n_pts, sb + kRawPts / 8, sb + kRawAmp / 8,
                              (float2 *)echo_dev, st);
    }
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "pl_synth_echo_static");
    return PL_OK;
}
