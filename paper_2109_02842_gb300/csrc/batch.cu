// Batches of uneven scans: per-scene z transforms and ONE persistent kernel
// for the range tables and back-projections of every scene, replayed as a
// CUDA graph (include/polyline.h, "Batches of uneven scans").
//
// Work queue: a device counter hands out items in a fixed order -- first all
// range-table items (scene, channel, 8 k_z bins), then all back-projection
// items (scene, pixel tile, k_z tile); scenes are ordered by decreasing
// back-projection cost, so the longest tiles start first. A range-table item
// bumps its scene's completion counter after its table rows are written and
// fenced; a back-projection item waits until its scene's counter reaches the
// scene's item count. Every range-table item is handed out before any
// back-projection item and is then owned by a resident block, so a wait can
// only be for work already in progress. The wait is still bounded (a clock64
// budget): on expiry the block sets an error flag, skips the tile and carries
// on; the host maps the flag to PL_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "bp_body.cuh"
#include "plan_internal.h"
#include "rt_body.cuh"

namespace {

// k_z bins per range-table item: 8 keeps the item's shared memory (fine grids
// of 8 bins, ping-pong) at <= 70 KB for fine <= 512, so the persistent kernel
// stays at 2-3 resident blocks per SM.
constexpr int kBatchUB = 8;

struct BatchScene {
    // range table
    NufftDesc nd;
    FftPlan fp;
    const float2 *S;
    const float2 *alpha;
    const float *xg;
    const float *dec;
    const float2 *tw_fine;
    void *table;
    int nub, rt_items, rt_begin;
    // back-projection
    BpDesc bp;
    const TileGeo *tgeo;
    const float2 *kc_hl;
    float2 *G;
    int ntx, nty, nut, bp_items, bp_begin;
    int need;           // range-table items this scene's tiles wait for
};

struct BatchConst {
    CoefTable ct;
    int n_scenes;
    int total_rt;       // range-table items (they come first in the queue)
    int total;          // all items
    long long budget;   // clock64 cycles a wait may last
};

// counters[0]: next item; counters[1]: wait-expired flag;
// counters[2 + s]: completed range-table items of scene s (queue order)
template <int UT, int CC, int MINB, int PX>
__global__ void __launch_bounds__(256, MINB)
k_batch(BatchConst bc, const BatchScene *__restrict__ scenes, int *counters) {
    extern __shared__ float4 smem4[];
    __shared__ int s_item, s_scene, s_ok;
    __shared__ NufftDesc s_nd;
    __shared__ FftPlan s_fp;
    __shared__ BpDesc s_bp;
    volatile int *vc = counters;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = atomicAdd(&counters[0], 1);
            int s = 0;
            if (item < bc.total_rt) {
                s = bc.n_scenes - 1;
                while (s > 0 && scenes[s].rt_begin > item) --s;
            } else if (item < bc.total) {
                s = bc.n_scenes - 1;
                while (s > 0 && scenes[s].bp_begin > item) --s;
            }
            s_item = item;
            s_scene = s;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= bc.total) break;
        const BatchScene &sc = scenes[s_scene];
        if (item < bc.total_rt) {
            if (threadIdx.x == 0) {
                s_nd = sc.nd;
                s_fp = sc.fp;
            }
            __syncthreads();
            const int local = item - sc.rt_begin;
            rt::rt_block<kBatchUB>(s_nd, s_fp, sc.S, sc.alpha, sc.xg, sc.dec, sc.tw_fine, sc.table,
                             sc.bp.bf16, local / sc.nub, local % sc.nub,
                             reinterpret_cast<float2 *>(smem4));
            __threadfence();                   // this block's table rows, device-wide
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&counters[2 + s_scene], 1);
        } else {
            if (threadIdx.x == 0) {
                s_bp = sc.bp;
                int ok = 1;
                const long long t0 = clock64();
                while (vc[2 + s_scene] < sc.need) {
                    if (vc[1] != 0 || clock64() - t0 > bc.budget) {
                        ok = 0;
                        atomicExch(&counters[1], 1);
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                const int local = item - sc.bp_begin;
                const int ut = local % sc.nut;
                const int tl = local / sc.nut;
                bp::bp_tile<UT, 6, CC, PX>(s_bp, bc.ct, sc.table, sc.tgeo, sc.kc_hl, sc.G,
                                           tl % sc.ntx, tl / sc.ntx, ut, sc.ntx, smem4);
            }
        }
        __syncthreads();
    }
}

template <int UT, int CC, int MINB, int PX>
cudaError_t launch_batch_t(const BatchConst &bc, const BatchScene *scenes, int *counters,
                           size_t smem, int *blocks_out, bool query, cudaStream_t st) {
    auto kern = k_batch<UT, CC, MINB, PX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (query) {
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *blocks_out = std::max(1, per_sm) * sms;
        return e;
    }
    kern<<<*blocks_out, 256, smem, st>>>(bc, scenes, counters);
    return cudaGetLastError();
}

template <int UT>
cudaError_t launch_batch_u(int block_config, const BatchConst &bc, const BatchScene *scenes,
                           int *counters, size_t smem, int *blocks, bool query, cudaStream_t st) {
    if (block_config == 2)
        return launch_batch_t<UT, 16, 2, 1>(bc, scenes, counters, smem, blocks, query, st);
    if (block_config == 3)
        return launch_batch_t<UT, 8, 2, 2>(bc, scenes, counters, smem, blocks, query, st);
    return launch_batch_t<UT, 8, 3, 1>(bc, scenes, counters, smem, blocks, query, st);
}

cudaError_t launch_batch(int tile_u, int block_config, const BatchConst &bc,
                         const BatchScene *scenes, int *counters, size_t smem, int *blocks,
                         bool query, cudaStream_t st) {
    switch (tile_u) {
        case 8: return launch_batch_u<8>(block_config, bc, scenes, counters, smem, blocks, query, st);
        case 20: return launch_batch_u<20>(block_config, bc, scenes, counters, smem, blocks, query, st);
        default: return launch_batch_u<16>(block_config, bc, scenes, counters, smem, blocks, query, st);
    }
}

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;   // signature -> (tile_u, block_config)
std::map<std::string, int> g_tune_tc_cache;                // signature -> tc_launch

}  // namespace

constexpr int kAuxStreams = 8;

struct pl_batch {
    int n = 0;
    std::vector<pl_plan *> plans;
    int tile_u = 16, block_config = 1;
    bool persistent = false;
    int pblocks = 0;
    size_t smem = 0;
    BatchConst bc{};
    BatchScene *d_scenes = nullptr;
    int *d_counters = nullptr;
    int *h_flag = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    // scene-parallel streams of the non-persistent path (forked in the graph)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;
    std::vector<int> order;          // scenes, largest first
    std::vector<const void *> cap_echo;
    std::vector<void *> cap_img;
    pl_batch_info info{};
    // the persistent tensor-core back-projection: requested mode (0 auto,
    // 1 persistent, 2 per-scene launches), and when in use the scenes'
    // descriptors (device), table maps (a kernel parameter), items, launch shape
    int tc_mode = 0;
    bool tc_persistent = false;
    TcBatchMaps *h_maps = nullptr;
    TcScene *d_tcscenes = nullptr;
    int tc_total = 0, tc_split = 3, tc_grid = 0;
    size_t tc_smem = 0;

    void free_plans() {
        for (pl_plan *p : plans) pl_plan_destroy(p);
        plans.clear();
    }
    ~pl_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        for (cudaStream_t s : aux) cudaStreamDestroy(s);
        for (cudaEvent_t e : aux_ev) cudaEventDestroy(e);
        if (d_scenes) cudaFree(d_scenes);
        if (d_tcscenes) cudaFree(d_tcscenes);
        delete h_maps;
        if (d_counters) cudaFree(d_counters);
        if (h_flag) cudaFreeHost(h_flag);
        free_plans();
    }
};

namespace {

// tc_mode (block_config 4): 2 = per-scene launches in the layout each scene
// picks; otherwise every scene in the one-block-per-SM layout of the
// persistent back-projection
pl_status make_plans(pl_batch *B, int n, const pl_geometry *g, const pl_scan *s, const pl_freqs *f,
                     const pl_grid *gr, const pl_options *opts, int tile_u, int block_config,
                     int tc_mode) {
    B->free_plans();
    for (int i = 0; i < n; ++i) {
        pl_options o{};
        if (opts) o = opts[i];
        o.tile_u = block_config == 4 ? 0 : tile_u;     // the tensor-core kernel sizes its own
        o.block_config = block_config;
        o.one_block_per_sm = (block_config == 4 && tc_mode != 2) ? 1 : 0;
        pl_plan *p = nullptr;
        pl_status st = pl_plan_create(&p, &g[i], &s[i], &f[i], &gr[i], &o);
        if (st != PL_OK) return st;
        B->plans.push_back(p);
    }
    return PL_OK;
}

// Work items, queue order and device descriptors for the current plans.
pl_status build_queue(pl_batch *B, int tile_u, double timeout_ms, int debug) {
    const int n = (int)B->plans.size();
    B->tile_u = tile_u;
    B->block_config = B->plans[0]->block_config;
    B->persistent = true;
    for (pl_plan *p : B->plans)
        if (p->nd.w != 6 || p->nd.fine > 512 || p->block_config != B->block_config ||
            p->block_config == 4)
            B->persistent = false;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int i) {
        const pl_plan *p = B->plans[i];
        return (double)p->C * p->grid.nx * p->grid.ny * p->Np;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    B->order = order;
    std::vector<BatchScene> hs(n);
    int rt = 0;
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        const pl_plan *p = B->plans[order[k]];
        BatchScene &d = hs[k];
        d.nd = p->nd;
        d.fp = p->fineplan;
        d.S = p->d_S;
        d.alpha = p->d_alpha;
        d.xg = p->d_xg;
        d.dec = p->d_dec;
        d.tw_fine = p->d_twfine;
        d.table = p->d_table;
        d.nub = (p->Np + kBatchUB - 1) / kBatchUB;
        d.rt_items = p->C * d.nub;
        d.rt_begin = rt;
        rt += d.rt_items;
        d.bp = p->bp;
        d.bp.tile_u = tile_u;
        d.tgeo = p->d_tgeo;
        d.kc_hl = p->d_kchl;
        d.G = p->d_G;
        d.ntx = (p->grid.nx + d.bp.tile_px - 1) / d.bp.tile_px;
        d.nty = (p->grid.ny + 15) / 16;
        d.nut = (p->Np + tile_u - 1) / tile_u;
        d.bp_items = d.ntx * d.nty * d.nut;
        d.need = d.rt_items + ((debug && k == 0) ? 1 : 0);
        smem = std::max(smem, rt::smem_bytes(p->nd.fine, kBatchUB, p->nd.n_f));
        smem = std::max(smem, backproject_smem_bytes(p->R, tile_u, p->C, p->precision >= 1,
                                                     B->block_config));
    }
    int total = rt;
    for (int k = 0; k < n; ++k) {
        hs[k].bp_begin = total;
        total += hs[k].bp_items;
    }
    if (smem > 200 * 1024) B->persistent = false;
    B->smem = smem;
    // the tensor-core scenes' back-projections as one persistent launch: every
    // scene in the one-block-per-SM layout with 6 taps, one split, the same tap
    // polynomials, and the largest window pool within shared memory
    B->tc_persistent = false;
    if (B->block_config == 4 && B->tc_mode != 2) {
        const pl_plan *p0 = B->plans[0];
        bool ok = n <= kTcBatchMaxScenes;
        size_t tsm = 0;
        for (const pl_plan *p : B->plans) {
            ok = ok && p->block_config == 4 && p->nd.w == 6 && p->tc.npar == 3 && p->tc.cpr == 1 &&
                 p->tc.split == p0->tc.split &&
                 std::memcmp(&p->coef, &p0->coef, sizeof(CoefTable)) == 0;
            tsm = std::max(tsm, backproject_tc_batch_smem_bytes(p->tc));
        }
        ok = ok && tsm + 1024 <= 227 * 1024;      // + the kernel's static shared memory
        if (!ok && B->tc_mode == 1)
            return pl_internal_fail(PL_ERR_UNSUPPORTED,
                                    "a scene does not allow the persistent tensor-core launch");
        if (ok) {
            std::vector<TcScene> ts(n);
            if (!B->h_maps) B->h_maps = new (std::nothrow) TcBatchMaps();
            if (!B->h_maps) return pl_internal_fail(PL_ERR_OOM, "host allocation failed");
            int total_tc = 0;
            for (int k = 0; k < n; ++k) {
                const pl_plan *p = B->plans[order[k]];
                TcScene &t = ts[k];
                t.bp = p->bp;
                t.ta = p->tc;
                t.ta.blk0 = 0;
                t.ta.nblk = 0;
                t.tgeo = p->d_tgeo;
                t.kc_hl = p->d_kchl;
                t.G = p->d_G;
                t.begin = total_tc;
                t.nblk = backproject_tc_blocks(p->bp, p->tc);
                total_tc += t.nblk;
                B->h_maps->m[k] = p->tmap;
            }
            if (B->d_tcscenes) cudaFree(B->d_tcscenes);
            B->d_tcscenes = nullptr;
            PL_CUDA_RET(cudaMalloc(&B->d_tcscenes, sizeof(TcScene) * n));
            PL_CUDA_RET(cudaMemcpy(B->d_tcscenes, ts.data(), sizeof(TcScene) * n,
                                   cudaMemcpyHostToDevice));
            int dev = 0, sms = 0;
            PL_CUDA_RET(cudaGetDevice(&dev));
            PL_CUDA_RET(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            B->tc_total = total_tc;
            B->tc_split = p0->tc.split;
            B->tc_grid = sms;
            B->tc_smem = tsm;
            B->tc_persistent = true;
        }
    }
    B->bc = BatchConst{};
    B->bc.ct = B->plans[0]->coef;
    B->bc.n_scenes = n;
    B->bc.total_rt = rt;
    B->bc.total = total;
    int dev = 0, khz = 0;
    PL_CUDA_RET(cudaGetDevice(&dev));
    PL_CUDA_RET(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    B->bc.budget = (long long)(timeout_ms * (double)khz);
    if (B->d_scenes) cudaFree(B->d_scenes);
    B->d_scenes = nullptr;
    PL_CUDA_RET(cudaMalloc(&B->d_scenes, sizeof(BatchScene) * n));
    PL_CUDA_RET(cudaMemcpy(B->d_scenes, hs.data(), sizeof(BatchScene) * n, cudaMemcpyHostToDevice));
    if (B->persistent)
        PL_CUDA_RET(launch_batch(tile_u, B->block_config, B->bc, B->d_scenes, B->d_counters,
                                 B->smem, &B->pblocks, true, nullptr));
    B->info.work_items = B->tc_persistent ? B->tc_total : total;
    B->info.persistent = (B->persistent || B->tc_persistent) ? 1 : 0;
    B->info.persistent_blocks = B->persistent ? B->pblocks : (B->tc_persistent ? B->tc_grid : 0);
    if (B->persistent) {
        B->info.launches_per_execute = 2 * n + 1;
    } else if (B->tc_persistent) {
        // per scene: the z transform, its range-table launches and the
        // inverse transform; one back-projection launch for all
        int total = 1;
        for (const pl_plan *p : B->plans)
            total += 2 + ((p->block_config == 4 && p->rt_tc) ? (p->fwd_fft ? 2 : 3) : 1);
        B->info.launches_per_execute = total;
    } else {        // each scene's own kernels (pl_plan_get_info counts them)
        int total = 0;
        for (pl_plan *p : B->plans) {
            pl_info pi{};
            if (pl_plan_get_info(p, &pi) == PL_OK) total += pi.launches_per_execute;
        }
        B->info.launches_per_execute = total;
    }
    if ((!B->persistent || B->tc_persistent) && B->aux.empty()) {
        // scenes of the per-scene path run on kAuxStreams streams at once
        for (int k = 0; k < kAuxStreams; ++k) {
            cudaStream_t s = nullptr;
            cudaEvent_t e = nullptr;
            PL_CUDA_RET(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            B->aux.push_back(s);
            PL_CUDA_RET(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            B->aux_ev.push_back(e);
        }
        cudaEvent_t e = nullptr;
        PL_CUDA_RET(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        B->aux_ev.push_back(e);    // the fork event
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    return PL_OK;
}

pl_status enqueue(pl_batch *B, const void *const *echo, void *const *image, cudaStream_t st) {
    const int n = (int)B->plans.size();
    pl_status s;
    PL_CUDA_RET(cudaMemsetAsync(B->d_counters, 0, sizeof(int) * (2 + n), st));
    // the FP32 persistent kernel: the z transforms first, on `st`; the
    // tensor-core paths run each scene's z transform at the head of its chain
    // on the parallel streams
    if (B->persistent)
        for (int i = 0; i < n; ++i)
            if ((s = pl_stage_zfft(B->plans[i], (const float2 *)echo[i], st)) != PL_OK) return s;
    if (B->persistent) {
        PL_CUDA_RET(launch_batch(B->tile_u, B->block_config, B->bc, B->d_scenes, B->d_counters,
                                 B->smem, &B->pblocks, false, st));
        for (int i = 0; i < n; ++i)
            if ((s = pl_stage_zifft(B->plans[i], (float2 *)image[i], st)) != PL_OK) return s;
    } else if (B->tc_persistent) {
        // the scenes' range tables on the parallel streams, then one
        // persistent back-projection for every scene, then the inverse
        // transforms on the parallel streams again
        const int K = (int)B->aux.size();
        cudaEvent_t fork = B->aux_ev[K];
        for (int phase = 0; phase < 2; ++phase) {
            PL_CUDA_RET(cudaEventRecord(fork, st));
            for (int k = 0; k < K; ++k) PL_CUDA_RET(cudaStreamWaitEvent(B->aux[k], fork, 0));
            for (int j = 0; j < n; ++j) {
                const int i = B->order[j];
                cudaStream_t as = B->aux[j % K];
                if (phase == 0) {
                    if ((s = pl_stage_zfft(B->plans[i], (const float2 *)echo[i], as)) != PL_OK)
                        return s;
                    s = pl_stage_range_table(B->plans[i], as);
                } else {
                    s = pl_stage_zifft(B->plans[i], (float2 *)image[i], as);
                }
                if (s != PL_OK) return s;
            }
            for (int k = 0; k < K; ++k) {
                PL_CUDA_RET(cudaEventRecord(B->aux_ev[k], B->aux[k]));
                PL_CUDA_RET(cudaStreamWaitEvent(st, B->aux_ev[k], 0));
            }
            if (phase == 0)
                PL_CUDA_RET(launch_backproject_tc_batch(*B->h_maps, B->plans[0]->coef,
                                                        B->d_tcscenes, n, B->tc_total, B->tc_split,
                                                        B->d_counters, B->d_counters + 1,
                                                        B->tc_grid, B->tc_smem, st));
        }
    } else {
        // per-scene range table, back-projection and inverse transform, the
        // scenes (largest first) dealt round-robin to the streams, joined at
        // the end; the forward transforms above ran on st
        const int K = (int)B->aux.size();
        cudaEvent_t fork = B->aux_ev[K];
        PL_CUDA_RET(cudaEventRecord(fork, st));
        for (int k = 0; k < K; ++k) PL_CUDA_RET(cudaStreamWaitEvent(B->aux[k], fork, 0));
        for (int j = 0; j < n; ++j) {
            const int i = B->order[j];
            cudaStream_t as = B->aux[j % K];
            if ((s = pl_stage_zfft(B->plans[i], (const float2 *)echo[i], as)) != PL_OK) return s;
            if ((s = pl_stage_range_table(B->plans[i], as)) != PL_OK) return s;
            if ((s = pl_stage_backproject(B->plans[i], as)) != PL_OK) return s;
            if ((s = pl_stage_zifft(B->plans[i], (float2 *)image[i], as)) != PL_OK) return s;
        }
        for (int k = 0; k < K; ++k) {
            PL_CUDA_RET(cudaEventRecord(B->aux_ev[k], B->aux[k]));
            PL_CUDA_RET(cudaStreamWaitEvent(st, B->aux_ev[k], 0));
        }
    }
    PL_CUDA_RET(cudaMemcpyAsync(B->h_flag, B->d_counters + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                st));
    return PL_OK;
}

pl_status capture(pl_batch *B, const void *const *echo, void *const *image) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    cudaGraph_t g = nullptr;
    PL_CUDA_RET(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    pl_status s = enqueue(B, echo, image, B->cap);
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (s != PL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return pl_internal_cuda_fail(e, "cudaGraphInstantiate");
    B->cap_echo.assign(echo, echo + B->plans.size());
    B->cap_img.assign(image, image + B->plans.size());
    return PL_OK;
}

pl_status run_batch(pl_batch *B, const void *const *echo, void *const *image, cudaStream_t st) {
    const size_t n = B->plans.size();
    bool same = B->exec && B->cap_echo.size() == n;
    for (size_t i = 0; same && i < n; ++i)
        same = B->cap_echo[i] == echo[i] && B->cap_img[i] == image[i];
    if (!same) {
        pl_status s = capture(B, echo, image);
        if (s != PL_OK) return s;
    }
    *B->h_flag = 0;
    PL_CUDA_RET(cudaGraphLaunch(B->exec, st));
    PL_CUDA_RET(cudaStreamSynchronize(st));
    if (*B->h_flag) return pl_internal_fail(PL_ERR_TIMEOUT, "a bounded device-side wait expired");
    pl_status first = PL_OK;
    for (pl_plan *p : B->plans) {                // every plan's flags are taken
        const pl_status ps = pl_plan_take_timeout(p);
        if (first == PL_OK) first = ps;
    }
    return first;
}

// Time one batch execution (ms), best of `reps` after one warm-up.
pl_status time_batch(pl_batch *B, const void *const *echo, void *const *image, int reps,
                     double *ms) {
    pl_status s = run_batch(B, echo, image, B->cap);
    if (s != PL_OK) return s;
    cudaEvent_t a, b;
    PL_CUDA_RET(cudaEventCreate(&a));
    PL_CUDA_RET(cudaEventCreate(&b));
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, B->cap);
        s = run_batch(B, echo, image, B->cap);
        cudaEventRecord(b, B->cap);
        cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        best = std::min(best, (double)t);
        if (s != PL_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return s;
}

std::string signature(int n, const pl_geometry *g, const pl_scan *s, const pl_freqs *f,
                      const pl_grid *gr, const pl_options *opts) {
    std::string sig;
    for (int i = 0; i < n; ++i) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d:%d:%d:%d:%d:%.6g:%.6g;", g[i].mode,
                 g[i].mode == 0 ? g[i].n_elem : g[i].n_pairs, s[i].n, s[i].n_pad, f[i].n,
                 gr[i].nx, gr[i].ny, gr[i].nz, opts ? opts[i].nufft_w : 0, gr[i].dx,
                 opts ? opts[i].nufft_sigma : 0.0);
        sig += buf;
    }
    return sig;
}

}  // namespace

extern "C" {

pl_status pl_batch_create(pl_batch **out, int n, const pl_geometry *g, const pl_scan *s,
                          const pl_freqs *f, const pl_grid *gr, const pl_options *opts,
                          const pl_batch_options *bopt) {
    if (!out || n <= 0 || !g || !s || !f || !gr) return pl_internal_fail(PL_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    pl_batch_options bo{};
    if (bopt) bo = *bopt;
    if (bo.wait_timeout_ms <= 0) bo.wait_timeout_ms = 2000.0;
    if (bo.tc_launch < 0 || bo.tc_launch > 2) return pl_internal_fail(PL_ERR_ARG, "tc_launch must be 0..2");
    pl_batch *B = new (std::nothrow) pl_batch();
    if (!B) return pl_internal_fail(PL_ERR_OOM, "host allocation failed");
    B->n = n;
    // tensor cores without autotuning: each scene's own launches unless the
    // persistent launch is asked for (tc_launch 1); the autotuner times both
    B->tc_mode = bo.tc_launch == 1 ? 1 : 2;
    auto bail = [&](pl_status st) { delete B; return st; };
    cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counters, sizeof(int) * (2 + n));
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_flag, sizeof(int));
    if (e != cudaSuccess) return bail(pl_internal_cuda_fail(e, "pl_batch_create"));

    // default: the tensor-core kernel, unless an FP32 block shape is asked for
    int tile_u = bo.tile_u ? bo.tile_u : 16;
    int bcfg = bo.block_config ? bo.block_config : (bo.tile_u ? 1 : 4);
    const bool tune = bo.autotune && !bo.tile_u && !bo.block_config;
    pl_status st;
    if (tune) {
        const std::string sig = signature(n, g, s, f, gr, opts);
        bool cached = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune_cache.find(sig);
            if (it != g_tune_cache.end()) {
                tile_u = it->second.first;
                bcfg = it->second.second;
                B->tc_mode = g_tune_tc_cache[sig];
                cached = true;
            }
        }
        if (!cached) {
            // scratch echo / image buffers for timing (contents do not matter)
            std::vector<void *> ebuf(n, nullptr), ibuf(n, nullptr);
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                const int C = g[i].mode == 0 ? g[i].n_elem : g[i].n_pairs;
                e = cudaMalloc(&ebuf[i], sizeof(float2) * (size_t)C * s[i].n * f[i].n);
                if (e == cudaSuccess)
                    e = cudaMemset(ebuf[i], 0, sizeof(float2) * (size_t)C * s[i].n * f[i].n);
                if (e == cudaSuccess)
                    e = cudaMalloc(&ibuf[i], sizeof(float2) * (size_t)gr[i].nx * gr[i].ny * gr[i].nz);
            }
            double best = 1e30, dflt = 0.0;
            int best_tc = 0;
            // the tensor-core kernels (one persistent back-projection; each
            // scene's own launches, scenes on parallel streams) and the FP32
            // persistent kernel in three block shapes
            const int cfgs[4] = {4, 4, 1, 3};
            const int tcm[4] = {1, 2, 0, 0};
            const int tus[3] = {8, 16, 20};
            for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
                B->tc_mode = tcm[ci];
                if (make_plans(B, n, g, s, f, gr, opts, 16, cfgs[ci], tcm[ci]) != PL_OK) continue;
                for (int ti = 0; ti < (cfgs[ci] == 4 ? 1 : 3); ++ti) {
                    double ms = 0.0;
                    if (build_queue(B, tus[ti], bo.wait_timeout_ms, 0) != PL_OK) continue;
                    if (time_batch(B, ebuf.data(), ibuf.data(), 2, &ms) != PL_OK) continue;
                    if (cfgs[ci] == 1 && tus[ti] == 16) dflt = ms;
                    if (ms < best) {
                        best = ms;
                        tile_u = tus[ti];
                        bcfg = cfgs[ci];
                        best_tc = tcm[ci];
                    }
                }
            }
            B->tc_mode = best_tc;
            for (int i = 0; i < n; ++i) {
                if (ebuf[i]) cudaFree(ebuf[i]);
                if (ibuf[i]) cudaFree(ibuf[i]);
            }
            if (e != cudaSuccess) return bail(pl_internal_cuda_fail(e, "autotune"));
            B->info.tune_best_ms = best;
            B->info.tune_default_ms = dflt;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[sig] = {tile_u, bcfg};
            g_tune_tc_cache[sig] = best_tc;
        }
        B->info.autotuned = 1;
    }
    if ((st = make_plans(B, n, g, s, f, gr, opts, tile_u, bcfg, B->tc_mode)) != PL_OK)
        return bail(st);
    if ((st = build_queue(B, tile_u, bo.wait_timeout_ms, bo.debug_unsatisfiable)) != PL_OK)
        return bail(st);
    if (B->block_config == 4 && B->tc_mode == 0 && !B->tc_persistent) {
        // a scene rules out the persistent launch: each scene in its own layout
        B->tc_mode = 2;
        if ((st = make_plans(B, n, g, s, f, gr, opts, tile_u, bcfg, 2)) != PL_OK) return bail(st);
        if ((st = build_queue(B, tile_u, bo.wait_timeout_ms, bo.debug_unsatisfiable)) != PL_OK)
            return bail(st);
    }
    B->info.n_scenes = n;
    B->info.tile_u = tile_u;
    B->info.block_config = B->block_config;
    double upd = 0.0;
    size_t ws = 0;
    for (pl_plan *p : B->plans) {
        upd += (double)p->C * p->grid.nx * p->grid.ny * p->grid.nz * p->M;
        ws += p->workspace;
    }
    B->info.updates_per_execute = upd;
    B->info.workspace_bytes = ws;
    *out = B;
    return PL_OK;
}

pl_status pl_execute_batch(pl_batch *B, const void *const *echo, void *const *image, void *stream) {
    if (!B || !echo || !image) return pl_internal_fail(PL_ERR_ARG, "NULL argument");
    for (int i = 0; i < B->n; ++i)
        if (!echo[i] || !image[i]) return pl_internal_fail(PL_ERR_ARG, "NULL scene buffer");
    return run_batch(B, echo, image, (cudaStream_t)stream);
}

pl_status pl_batch_get_info(const pl_batch *B, pl_batch_info *info) {
    if (!B || !info) return pl_internal_fail(PL_ERR_ARG, "NULL argument");
    *info = B->info;
    return PL_OK;
}

pl_status pl_batch_destroy(pl_batch *B) {
    if (!B) return pl_internal_fail(PL_ERR_ARG, "batch is NULL");
    delete B;
    return PL_OK;
}

}  // extern "C"
