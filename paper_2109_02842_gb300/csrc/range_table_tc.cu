// Range-profile table of step (8a) / (19a) for the tensor-core back-projection,
// evaluated as exact sums on the tensor cores instead of a type-1 NUFFT (up to
// 128 frequencies):
//
//   b[c][i][u] = sum_m S[c][u][m] E[u][i][m],   E = alpha e^{+j theta_um (i - L/2)},
//
// theta_um = kappa''_um h and alpha as in setup.cu (k weight, 1/phihat of the
// interpolation kernel, range-origin phase). For one k_z bin u this is a
// complex matrix product over the frequencies: channels (M = 128 per block) x
// table rows (N = L rounded up to 16) x frequencies (K). Operands are BF16
// split hi + lo (three products per real product; with a BF16 spectrum, two:
// A hi times E hi and E lo), the complex product is
// four real ones with the imaginary-by-imaginary term negated through the
// instruction descriptor, and the two accumulators (Re, Im) live in TMEM.
//
//   k_rt_prep          S [C][N_p][M] -> A [u][re hi, re lo, im hi, im lo][C][K] BF16
//   k_range_table_tc   persistent, one block per SM, over the items (128-channel
//                      block, bin, row part): TMA (128-byte swizzled, K-major) A
//                      and E tiles, 12 MMAs per 16-frequency step (up to two
//                      64-frequency atoms per item), tcgen05.ld,
//                      BF16 hi/lo, stored straight from the registers into
//                      prod [u][hi, lo][row][Cp] of (re, im) pairs, channels
//                      innermost (full 128-byte lines). Row parts of Lh rows
//                      (a multiple of 16, at most 96 so that two items'
//                      operands fit in shared memory). Warp-specialised
//                      (a copy warp, a product warp, eight store warps) over
//                      two operand buffers and two accumulator pairs: one
//                      item's stores overlap the next item's products and
//                      the copies of the one after.
//   k_rt_transpose     prod -> table [c][hi, lo][L][column 2u + (re, im)] (or
//                      planar: Re at column u, Im at row_words + u), the layout
//                      the back-projection streams (u innermost)
//
// E [u][re hi, re lo, im hi, im lo][L'][K] = alpha_um e^{+j theta_um (i - L/2)} is a
// plan-time table (the per-(k_z, f) factor on the side of the smaller operand).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

namespace {

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16(x);
    lo = __float2bfloat16(x - __bfloat162float(hi));
}

__device__ __forceinline__ double kz_at(int u, int n_pad, double dz) {
    const int ut = (2 * u < n_pad) ? u : u - n_pad;
    return PL_TWO_PI * (double)ut / ((double)n_pad * dz);
}

__global__ void k_setup_rt_E(NufftDesc d, double dz, const double *k, const double *kc,
                             const float2 *alpha, int Lp, int Kp, __nv_bfloat16 *E) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)d.n_pad * Lp * Kp) return;
    const int m = (int)(idx % Kp);
    const int i = (int)((idx / Kp) % Lp);
    const int u = (int)(idx / ((long long)Kp * Lp));
    double re = 0.0, im = 0.0;
    if (i < d.L && m < d.n_f) {
        const double kz = kz_at(u, d.n_pad, dz);
        const double q = d.mode == 0 ? 4.0 * k[m] * k[m] - kz * kz : k[m] * k[m] - 0.25 * kz * kz;
        if (q > 0.0) {
            // the source factor alpha_um (k weight, 1 / phihat, range-origin
            // phase) rides on E, so the operand A is the plain spectrum
            const double ph = (sqrt(q) - kc[u]) * d.h * (double)(i - d.L / 2);
            const float2 al = alpha[(size_t)u * d.n_f + m];
            const double c = cos(ph), sn = sin(ph);
            re = (double)al.x * c - (double)al.y * sn;
            im = (double)al.x * sn + (double)al.y * c;
        }
    }
    __nv_bfloat16 h, l;
    const size_t plane = (size_t)Lp * Kp;
    const size_t base = (size_t)u * 4 * plane + (size_t)i * Kp + m;
    split_bf16((float)re, h, l);
    E[base] = h;
    E[base + plane] = l;
    split_bf16((float)im, h, l);
    E[base + 2 * plane] = h;
    E[base + 3 * plane] = l;
}

// A[u][plane][c][m] = split(S[c][u][m]) (zero for m >= M)
__global__ void k_rt_prep(const float2 *__restrict__ S, int C, int Np, int M, int Kp,
                          int hi_only, __nv_bfloat16 *__restrict__ A) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)C * Np * Kp) return;
    const int m = (int)(idx % Kp);
    const int u = (int)((idx / Kp) % Np);
    const int c = (int)(idx / ((long long)Kp * Np));
    float2 a = make_float2(0.f, 0.f);
    if (m < M) a = S[((size_t)c * Np + u) * M + m];
    __nv_bfloat16 h, l;
    const size_t plane = (size_t)C * Kp;
    const size_t base = (size_t)u * 4 * plane + (size_t)c * Kp + m;
    split_bf16(a.x, h, l);
    A[base] = h;
    if (!hi_only) A[base + plane] = l;
    split_bf16(a.y, h, l);
    A[base + 2 * plane] = h;
    if (!hi_only) A[base + 3 * plane] = l;
}

// One block per SM (persistent) walks the work items (128-channel block, bin,
// row part) gridDim.x apart; an item is natoms stages, one per 64-frequency
// atom, stage st's operands in buffer st & 1 and the item's products in
// accumulator pair item & 1. The block is warp-specialised so that the
// copies, the products and the stores of consecutive items overlap:
//  * warp 8 (one lane) issues a stage's copies once its buffer is free (the
//    products of stage st - 2 completed: empty[st & 1]);
//  * warp 9 (one lane) issues a stage's products once its operands landed
//    (full[st & 1]) and, at an item's first stage, once the item's
//    accumulator pair has been read out for item - 2 (acc_empty), then
//    commits them to empty[] and, at the item's last stage, to acc_full[];
//  * warps 0-7 read each item's accumulators back once its products
//    completed, release them (acc_empty) and convert and store the item.
// Every wait is bounded; one that runs out sets a bit in *err and the abort
// flag, the roles stop taking stages, and before tensor memory is released
// the copies and products issued have completed.
__global__ void __launch_bounds__(320, 1)
k_range_table_tc(RtTcArgs ra, const __grid_constant__ CUtensorMap tmA,
                 const __grid_constant__ CUtensorMap tmB, uint32_t *__restrict__ prod, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t a_full[2], a_empty[2], e_full[2], e_empty[2];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain, dbg_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    volatile int *abortp = &abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t a_tile = 128 * 128;                 // one plane x 64-frequency atom of A
    const uint32_t b_tile = (uint32_t)ra.Lh * 128;     // of E (one row part)
    const int NA = ra.natoms;
    const int ncb = (ra.C + 127) / 128;
    // pairs (128-channel block, bin) gridDim.x apart, channel blocks varying
    // fastest so that the blocks running together share each bin's E tiles
    // in L2; a block takes all row parts of its pair in turn (item k = pair
    // k / nh, row part k % nh), so that with one atom the pair's A tile is
    // copied once for all its row parts
    const int npairs = ncb * ra.Np;
    const int pmine = (npairs - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int nmine = pmine * ra.nh;
    const int nstages = nmine * NA;
    const bool share_a = NA == 1;
    const long long budget = ra.budget;
    auto coords = [&](int k, int &c0, int &u, int &h) {
        const int pr = (int)blockIdx.x + (k / ra.nh) * (int)gridDim.x;
        c0 = 128 * (pr % ncb);
        u = pr / ncb;
        h = k % ra.nh;
    };
    // stage st: its A load (the pair's with one atom, else the stage's own)
    // goes to A slot ai & 1, its E tile to E slot st & 1
    auto a_index = [&](int st) { return share_a ? st / ra.nh : st; };
    auto loads_a = [&](int st) { return !share_a || st % ra.nh == 0; };
    auto frees_a = [&](int st) { return !share_a || st % ra.nh == ra.nh - 1; };
    unsigned char *Abuf = smem, *Ebuf = smem + 2 * 4 * a_tile;
    const uint32_t a_bytes = 4 * a_tile - (ra.a_hi_only ? 2 * a_tile : 0u);

    if (threadIdx.x == 0) {
        tc05::mbar_init(&dbg_bar, 1);
        tc05::mbar_init(&drain, 1);
        for (int b = 0; b < 2; ++b) {
            tc05::mbar_init(&a_full[b], 1);
            tc05::mbar_init(&a_empty[b], 1);
            tc05::mbar_init(&e_full[b], 1);
            tc05::mbar_init(&e_empty[b], 1);
            tc05::mbar_init(&acc_full[b], 1);
            tc05::mbar_init(&acc_empty[b], 8);          // the eight store warps
        }
        tc05::fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) {
        tc05::tmem_alloc(&tmem_slot, 512);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 8) {
        // ------------------------------------------------ copies
        if (lane == 0) {
            int issued = 0, a_issued = 0;
            for (int st = 0; st < nstages && !*abortp; ++st) {
                const int at = st % NA, k = st / NA;
                int c0, u, h;
                coords(k, c0, u, h);
                if (loads_a(st)) {
                    // the A slot is free once the products of A load ai - 2 completed
                    const int ai = a_index(st), b = ai & 1;
                    if (ai >= 2 &&
                        !tc05::mbar_wait(&a_empty[b], (uint32_t)((ai >> 1) - 1) & 1u, budget)) {
                        atomicOr(err, 4);
                        *abortp = 1;
                        break;
                    }
                    unsigned char *As = Abuf + b * 4 * a_tile;
                    // with a BF16 spectrum only A's hi planes (0 and 2) are loaded
                    tc05::mbar_arrive_expect_tx(&a_full[b], a_bytes);
                    for (int p = 0; p < 4; ++p)
                        if (!ra.a_hi_only || (p & 1) == 0)
                            tc05::tma_load_3d(As + p * a_tile, &tmA, &a_full[b], 64 * at, c0,
                                              4 * u + p);
                    a_issued = ai + 1;
                }
                const int e = st & 1;
                if (st >= 2 &&
                    !tc05::mbar_wait(&e_empty[e], (uint32_t)((st >> 1) - 1) & 1u, budget)) {
                    atomicOr(err, 4);
                    *abortp = 1;
                    break;
                }
                unsigned char *Bs = Ebuf + e * 4 * b_tile;
                tc05::mbar_arrive_expect_tx(&e_full[e], 4 * b_tile);
                for (int p = 0; p < 4; ++p)
                    tc05::tma_load_3d(Bs + p * b_tile, &tmB, &e_full[e], 64 * at, h * ra.Lh,
                                      4 * u + p);
                issued = st + 1;
            }
            // the last copies issued (at most one per slot outstanding) have
            // landed before shared memory is released
            for (int ai = a_issued > 2 ? a_issued - 2 : 0; ai < a_issued; ++ai)
                if (!tc05::mbar_wait(&a_full[ai & 1], (uint32_t)(ai >> 1) & 1u, budget))
                    atomicOr(err, 16);
            for (int st = issued > 2 ? issued - 2 : 0; st < issued; ++st)
                if (!tc05::mbar_wait(&e_full[st & 1], (uint32_t)(st >> 1) & 1u, budget))
                    atomicOr(err, 16);
        }
        __syncwarp();
    } else if (warp == 9) {
        // ------------------------------------------------ products
        if (lane == 0) {
            for (int st = 0; st < nstages && !*abortp; ++st) {
                const int k = st / NA, at = st % NA;
                const int ai = a_index(st), ab = ai & 1, e = st & 1;
                // (an item's first stage) its accumulator pair read out for item k - 2
                if (at == 0 && k >= 2 &&
                    !tc05::mbar_wait(&acc_empty[k & 1], (uint32_t)((k >> 1) - 1) & 1u, budget)) {
                    atomicOr(err, 8);
                    *abortp = 1;
                    break;
                }
                // (test hook: the first stage waits on a barrier nothing completes)
                bool landed = (ra.dbg_wait && st == 0)
                                  ? tc05::mbar_wait(&dbg_bar, 0, budget)
                                  : tc05::mbar_wait(&e_full[e], (uint32_t)(st >> 1) & 1u, budget);
                if (landed && loads_a(st))
                    landed = tc05::mbar_wait(&a_full[ab], (uint32_t)(ai >> 1) & 1u, budget);
                if (!landed) {
                    atomicOr(err, 1);
                    *abortp = 1;
                    break;
                }
                tc05::fence_after_sync();
                const unsigned char *As = Abuf + ab * 4 * a_tile, *Bs = Ebuf + e * 4 * b_tile;
                const uint32_t id = ra.idesc, idn = ra.idesc | (1u << 13);   // negate A
                const uint32_t dre = tmem + (uint32_t)((k & 1) * 2 * ra.Lh), dim = dre + ra.Lh;
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = ks * 32;
                    auto da = [&](int p) {
                        return tc05::smem_desc_sw128(tc05::smem_addr(As + p * a_tile) + ko, 16, 1024);
                    };
                    auto db = [&](int p) {
                        return tc05::smem_desc_sw128(tc05::smem_addr(Bs + p * b_tile) + ko, 16, 1024);
                    };
                    const uint32_t acc = (at > 0 || ks > 0) ? 1u : 0u;
                    // planes: 0 re hi, 1 re lo, 2 im hi, 3 im lo
                    // Re += a_r b_r - a_i b_i
                    tc05::mma_ss(dre, da(0), db(0), id, acc);
                    tc05::mma_ss(dre, da(0), db(1), id, 1u);
                    if (!ra.a_hi_only) tc05::mma_ss(dre, da(1), db(0), id, 1u);
                    tc05::mma_ss(dre, da(2), db(2), idn, 1u);
                    tc05::mma_ss(dre, da(2), db(3), idn, 1u);
                    if (!ra.a_hi_only) tc05::mma_ss(dre, da(3), db(2), idn, 1u);
                    // Im += a_r b_i + a_i b_r
                    tc05::mma_ss(dim, da(0), db(2), id, acc);
                    tc05::mma_ss(dim, da(0), db(3), id, 1u);
                    if (!ra.a_hi_only) tc05::mma_ss(dim, da(1), db(2), id, 1u);
                    tc05::mma_ss(dim, da(2), db(0), id, 1u);
                    tc05::mma_ss(dim, da(2), db(1), id, 1u);
                    if (!ra.a_hi_only) tc05::mma_ss(dim, da(3), db(0), id, 1u);
                }
                tc05::mma_commit(&e_empty[e]);                  // the E slot may be refilled
                if (frees_a(st)) tc05::mma_commit(&a_empty[ab]);   // and the A slot
                if (at == NA - 1) tc05::mma_commit(&acc_full[k & 1]);   // the item is done
            }
            // every product issued has completed before tensor memory is released
            tc05::mma_commit(&drain);
            if (!tc05::mbar_wait(&drain, 0, budget)) atomicOr(err, 32);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ stores (warps 0-7)
        // each thread (one channel: its TMEM lane) converts 16 rows at a time
        // to BF16 hi/lo (re, im) pairs and stores them into prod
        // [u][hi, lo][row][Cp], channels innermost, so each store instruction
        // of a warp writes 32 consecutive channels (a full 128-byte line).
        // Warps 0-3 and 4-7 take alternate 16-row chunks of their TMEM lane
        // quarter.
        const int Cp = ncb * 128;                // channel stride of prod
        const int R = ra.nh * ra.Lh;             // rows of prod per (bin, plane)
        const int q = warp & 3;
        for (int k = 0; k < nmine; ++k) {
            bool ok = !*abortp && tc05::mbar_wait(&acc_full[k & 1], (uint32_t)(k >> 1) & 1u, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    if (!*abortp) atomicOr(err, 2);
                    *abortp = 1;
                }
                break;
            }
            tc05::fence_after_sync();
            int c0, u, h;
            coords(k, c0, u, h);
            const int rows_here = min(ra.Lh, ra.L - h * ra.Lh);     // table rows of this part
            const uint32_t lane_base =
                tmem + (uint32_t)((k & 1) * 2 * ra.Lh) + ((uint32_t)(32 * q) << 16);
            const int c = c0 + 32 * q + lane;
            uint32_t *g_hi = prod + ((size_t)(2 * u + 0) * R + h * ra.Lh) * Cp + c;
            uint32_t *g_lo = prod + ((size_t)(2 * u + 1) * R + h * ra.Lh) * Cp + c;
            for (int i0 = 16 * (warp >> 2); i0 < rows_here; i0 += 32) {
                uint32_t vr[16], vi[16];
                tc05::tmem_ld16(lane_base + i0, vr);
                tc05::tmem_ld16(lane_base + ra.Lh + i0, vi);
                tc05::tmem_wait_ld();
                const int n = min(16, rows_here - i0);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j < n) {
                        const float re = __uint_as_float(vr[j]), im = __uint_as_float(vi[j]);
                        __nv_bfloat162 hv = __floats2bfloat162_rn(re, im);
                        const float2 hf = __bfloat1622float2(hv);
                        __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
                        g_hi[(size_t)(i0 + j) * Cp] = *reinterpret_cast<uint32_t *>(&hv);
                        g_lo[(size_t)(i0 + j) * Cp] = *reinterpret_cast<uint32_t *>(&l);
                    }
                }
            }
            // the accumulator pair is free for item k + 2's products
            tc05::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&acc_empty[k & 1]);
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 512);
}

// prod [u][plane][row][Cp] (uint32 = (re, im) BF16 pair) -> table
// [c][plane][L][u], u beyond N_p written as zeros so the padding columns stay
// zero. Interleaved rows hold row_words (re, im) pairs; planar rows hold
// row_words Re entries, then row_words Im. A block covers 64 channels x 64
// bins of one (plane, row); each thread transposes a 4 x 4 block in
// registers: four independent 16-byte loads (4 channels of one bin each) and
// four row stores (4 bins of one channel), so a warp (16 channels x 32 bins)
// reads and writes 64-byte runs with no shared memory or barrier.
__device__ __forceinline__ uint32_t word_of(const uint4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

template <bool PLANAR>
__global__ void __launch_bounds__(256)
k_rt_transpose(const uint32_t *__restrict__ prod, uint32_t *__restrict__ table, int C, int Cp,
               int L, int R, int Np, int row_words) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 64 + 16 * (warp & 3) + 4 * (lane & 3);
    const int u = blockIdx.y * 64 + 32 * (warp >> 2) + 4 * (lane >> 2);
    const int p = blockIdx.z / L, i = blockIdx.z - p * L;
    if (c >= C || u >= row_words) return;      // row_words is a multiple of 4
    // channels c..c+3 are below Cp (a multiple of 128); those at C and beyond
    // are loaded but never stored
    const uint32_t *src = prod + ((size_t)p * R + i) * Cp + c;
    const size_t bin_stride = (size_t)2 * R * Cp;
    uint4 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        v[r] = u + r < Np ? *reinterpret_cast<const uint4 *>(src + (size_t)(u + r) * bin_stride)
                          : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (c + e >= C) break;
        const uint32_t w0 = word_of(v[0], e), w1 = word_of(v[1], e);
        const uint32_t w2 = word_of(v[2], e), w3 = word_of(v[3], e);
        uint32_t *row = table + (((size_t)(c + e) * 2 + p) * L + i) * row_words;
        if (PLANAR) {
            // low halves (Re) of the four bins, then the high halves (Im)
            __nv_bfloat16 *rb = reinterpret_cast<__nv_bfloat16 *>(row);
            *reinterpret_cast<uint2 *>(rb + u) =
                make_uint2(__byte_perm(w0, w1, 0x5410), __byte_perm(w2, w3, 0x5410));
            *reinterpret_cast<uint2 *>(rb + row_words + u) =
                make_uint2(__byte_perm(w0, w1, 0x7632), __byte_perm(w2, w3, 0x7632));
        } else {
            *reinterpret_cast<uint4 *>(row + u) = make_uint4(w0, w1, w2, w3);
        }
    }
}

}  // namespace

size_t range_table_tc_smem_bytes(const RtTcArgs &ra) {
    // two operand buffers of one 64-frequency atom each (whatever natoms)
    return 1024 + (size_t)2 * 4 * (128 * 128 + (size_t)ra.Lh * 128);
}

cudaError_t launch_setup_rt_E(const NufftDesc &d, double dz, const double *k, const double *kc,
                              const float2 *alpha, int Lp, int Kp, void *E, cudaStream_t st) {
    const long long n = (long long)d.n_pad * Lp * Kp;
    k_setup_rt_E<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, dz, k, kc, alpha, Lp, Kp,
                                                              (__nv_bfloat16 *)E);
    return cudaGetLastError();
}

cudaError_t launch_range_table_tc(const RtTcArgs &ra, const CUtensorMap &tmA,
                                  const CUtensorMap &tmB, const float2 *S,
                                  void *A, void *prod, void *table, int row_words, int planar,
                                  int *err, bool prepared, cudaStream_t st) {
    if (ra.natoms < 1 || ra.natoms > 2 || 4 * ra.Lh > 512 || ra.grid < 1 || row_words % 4 != 0 ||
        2 * ra.L > 65535)
        return cudaErrorInvalidValue;
    cudaError_t e;
    if (!prepared) {     // the z transform wrote S, not the split operand
        const long long n = (long long)ra.C * ra.Np * ra.Kp;
        k_rt_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, ra.C, ra.Np, ra.M, ra.Kp,
                                                               ra.a_hi_only, (__nv_bfloat16 *)A);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const size_t smem = range_table_tc_smem_bytes(ra);
    e = cudaFuncSetAttribute(k_range_table_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    // (blocks take (channel block, bin) pairs with all their row parts)
    const int pairs = (ra.C + 127) / 128 * ra.Np;
    k_range_table_tc<<<min(pairs, ra.grid), 320, smem, st>>>(ra, tmA, tmB, (uint32_t *)prod, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int Cp = (ra.C + 127) / 128 * 128, R = ra.nh * ra.Lh;
    dim3 tg((ra.C + 63) / 64, (row_words + 63) / 64, 2 * ra.L);
    if (planar)
        k_rt_transpose<true><<<tg, 256, 0, st>>>((const uint32_t *)prod, (uint32_t *)table, ra.C,
                                                 Cp, ra.L, R, ra.Np, row_words);
    else
        k_rt_transpose<false><<<tg, 256, 0, st>>>((const uint32_t *)prod, (uint32_t *)table, ra.C,
                                                  Cp, ra.L, R, ra.Np, row_words);
    return cudaGetLastError();
}
