// Internal: the plan object and stage helpers shared by plan.cu and batch.cu.
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "../../include/polyline.h"
#include "common.cuh"
#include "kernels.h"

// The inputs a plan was created from (deep copies: the pointers of the
// structs point into the vectors), so that a second plan can be built alike.
struct PlanInputs {
    pl_geometry g{};
    pl_scan s{};
    pl_freqs f{};
    pl_grid gr{};
    pl_options o{};
    bool has_opts = false;
    std::vector<double> elem_xy, f_hz;
    std::vector<int> elem_section, pair_tx, pair_rx;
};

struct pl_plan {
    // problem
    int mode = 0, C = 0, N = 0, Np = 0, M = 0;
    double z0s = 0, dzs = 0;
    pl_grid grid{};
    int precision = 0;
    int tile_u = 16;
    int block_config = 1;
    int device = 0;
    // nufft
    NufftDesc nd{};
    double sigma = 2.0;
    int R = 0;
    TcArgs tc{};           // tensor-core variant (block_config 4)
    CUtensorMap tmap{};    // its TMA map of the range table
    // status word in mapped host memory and its device alias: expired waits of
    // the tensor-core kernels, PL_FLAG_NONFINITE from the echo scan
    int *h_err = nullptr;
    int *d_err = nullptr;
    bool check_nonfinite = false;   // scan every echo for NaN / Inf first
    // its range table as exact sums on the tensor cores (range_table_tc.cu)
    bool rt_tc = false;
    RtTcArgs rt{};
    CUtensorMap tmapA{}, tmapE{};
    void *d_rtE = nullptr, *d_rtA = nullptr, *d_rtprod = nullptr;
    CoefTable coef{};
    BpDesc bp{};
    // the tensor-core back-projection's last partial wave: an execution
    // launches the blocks of the full waves (bp_full), then the rest, on its
    // stream, and meanwhile, on s_bp, the z-IFFT of the first zi_cols pixels,
    // whose channel parts all finished in the full waves, on the SMs the last
    // wave leaves idle (bp_full 0: one launch each)
    int bp_full = 0, zi_cols = 0;
    cudaStream_t s_bp = nullptr;
    cudaEvent_t ev_bpA = nullptr, ev_bpB = nullptr;
    cudaEvent_t ev_z0 = nullptr, ev_z1 = nullptr;   // zeroing G on s_bp (atomic parts)
    // transforms
    bool fwd_fft = true, inv_fft = true;
    int inv_off = 0;
    FftPlan zplan{};
    FftPlan fineplan{};
    // device memory
    double *d_chxy = nullptr, *d_k = nullptr, *d_kc = nullptr, *d_kspan = nullptr;
    double *d_kband = nullptr;
    double *d_glx = nullptr, *d_glw = nullptr;
    float *d_xg = nullptr, *d_dec = nullptr;
    float2 *d_kchl = nullptr;
    TileGeo *d_tgeo = nullptr;
    float2 *d_alpha = nullptr, *d_twz = nullptr, *d_twfine = nullptr;
    float2 *d_Tfwd = nullptr, *d_Tinv = nullptr;
    // the inverse transform at off-grid heights on the tensor cores (tensor-core
    // plans): its shape, BF16 table and TMA map
    bool zidft_tc = false;
    ZidftTcArgs zt{};
    void *d_TinvB = nullptr;
    CUtensorMap tmapZ{};
    float2 *d_S = nullptr, *d_G = nullptr;
    void *d_table = nullptr;
    size_t table_bytes = 0;
    float2 *d_echo_in = nullptr, *d_img_out = nullptr;   // pl_execute_host staging
    // pl_execute_host_stream: a second staging pair, the copy streams and the
    // events that order them against the reconstruction
    float2 *d_echo_in2 = nullptr, *d_img_out2 = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_in[2]{}, ev_done[2]{}, ev_out[2]{}, ev_start = nullptr;
    // ... and the second plan (same inputs, own workspace) and device stream
    // that take every other scan, so that consecutive scans overlap
    PlanInputs inputs;
    pl_plan *twin = nullptr;
    cudaStream_t s_twin = nullptr;
    // comparison algorithms (exact sum, direct BP), set up on first use
    std::vector<double> h_chxy, h_k;                      // [C][4] positions, [M] k
    float2 *d_kap = nullptr, *d_zs = nullptr, *d_kff = nullptr;
    float *d_wum = nullptr;
    float4 *d_chff = nullptr;
    bool cmp_ready = false;
    ExactDesc exact{};
    DirectDesc direct{};
    size_t workspace = 0;
    int n_gl = 0;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> recorded;
    size_t ev_next = 0;

    ~pl_plan() {
        void *ptrs[] = {d_chxy, d_k,    d_kc,   d_kspan, d_kband, d_glx,  d_glw,     d_kchl, d_tgeo,
                        d_xg,   d_dec,  d_alpha, d_twz,  d_twfine, d_Tfwd, d_Tinv,
                        d_S,    d_G,    d_table, d_echo_in, d_img_out, d_kap, d_zs,
                        d_kff,  d_wum,  d_chff, d_rtE, d_rtA, d_rtprod, d_echo_in2, d_img_out2,
                        d_TinvB};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        for (cudaEvent_t e : {ev_in[0], ev_in[1], ev_done[0], ev_done[1], ev_out[0], ev_out[1],
                              ev_start})
            if (e) cudaEventDestroy(e);
        if (s_h2d) cudaStreamDestroy(s_h2d);
        if (s_d2h) cudaStreamDestroy(s_d2h);
        if (s_twin) cudaStreamDestroy(s_twin);
        if (s_bp) cudaStreamDestroy(s_bp);
        for (cudaEvent_t e : {ev_bpA, ev_bpB, ev_z0, ev_z1})
            if (e) cudaEventDestroy(e);
        delete twin;
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        if (h_err) cudaFreeHost(h_err);
    }

    cudaEvent_t next_event() {
        if (ev_next == ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev_pool.push_back(e);
        }
        return ev_pool[ev_next++];
    }
};

// Return the mapped status (and set the thread's error message) on a CUDA error.
#define PL_CUDA_RET(call)                                                   \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return pl_internal_cuda_fail(e_, #call);     \
    } while (0)

// PL_ERR_NONFINITE if the echo scan of an earlier execution of the plan found
// NaN / Inf, else PL_ERR_TIMEOUT if one of its bounded device waits ran out,
// else PL_OK; the flags are cleared.
pl_status pl_plan_take_timeout(pl_plan *plan);

// Launch one stage of a plan on `st` (no timing events, no synchronisation).
pl_status pl_stage_zfft(pl_plan *P, const float2 *echo, cudaStream_t st);
pl_status pl_stage_range_table(pl_plan *P, cudaStream_t st);
pl_status pl_stage_backproject(pl_plan *P, cudaStream_t st);
pl_status pl_stage_zifft(pl_plan *P, float2 *image, cudaStream_t st);
