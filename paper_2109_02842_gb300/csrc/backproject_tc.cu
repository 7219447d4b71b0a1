// Back-projection (step 8b / 19b) on the fifth-generation tensor cores.
//
// With the band centre kappa_T shared by the k_z bins of a block (the range
// table is built with that centre for every bin of the group), the carrier
// e^{j kappa_T a_c(p)} depends on the pixel and the channel only, so it goes
// into the interpolation weights and the whole channel sum becomes a chain
// of dense products accumulated in tensor memory:
//
//   G[p][u] = sum_c sum_k A_c[p][k] B_c[k][u],
//   A_c[p][k] = phi(a_c(p) - l_{i_c + k}) e^{j kappa_T a_c(p)},  B_c[k][u] = b_c[i_c + k][u],
//
// p one of the block's 128 pixels (the MMA's M), k one of the 16 KS table rows
// of the block's window for channel c (starting at i_c, chosen at plan time
// so that every pixel's w taps fall inside), u the block's UT k_z bins.
// Complex products are real ones in one of two layouts of the table rows:
//  * planar (PLANAR, the default when it fits): a row holds Re b of every
//    bin, then Im b; the accumulators are Re G and Im G (UT columns each) and
//    Re G += Re A Re B - Im A Im B, Im G += Re A Im B + Im A Re B, the minus
//    through the instruction descriptor's negate-A bit; UT covers every bin,
//    so a channel is one round of 4 (x3 with hi/lo) products of N = UT;
//  * interleaved: a row holds (re_u, im_u) pairs, P = sum Re(A) B and
//    Q = sum Im(A) B (2 UT columns each) give G = (P_re - Q_im, P_im + Q_re),
//    and the bins go in blocks of UT.
// Operands are BF16; for FP32-level accuracy each is split into hi + lo
// and the product taken as hi.hi + hi.lo + lo.hi (SPLIT = 3), relative
// error ~1e-5; SPLIT = 1 takes hi.hi only (~1e-3). In the planar layout a
// tile's channels go to two blocks (nsplit = 2), so that each accumulator
// sums as many products as an interleaved one; the two add their sums into
// one spectrum (atomic adds onto G zeroed beforehand) or, in a batch's
// persistent launch, write spectra G[0], G[1] that the inverse z transform
// adds as it loads them.
//
// By default the products are 2:4 sparse (tcgen05.mma.sp, the kernel
// k_backproject_tc_sp below): a window's rows taken in residue order put at
// most two of a pixel's w taps in every group of four K indices, so a
// product of logical K = 32 covers twice the rows of a dense one at the
// same cost (planar 16-row windows: K = [Re rows; Im rows]; planar 32-row
// windows: the Re rows and the Im rows as two operands; interleaved: the
// window's 32 rows, or its hi and lo rows). The dense kernel below
// (k_backproject_tc) serves dense_products = 1 and the layouts without a
// sparse variant.
//
// Block = 16 x 8 pixels x UT bins, 4 NPAR + 2 warps (NPAR = 2 and two blocks
// per SM when the accumulators and three A buffers fit in 256 TMEM columns,
// NPAR = 3 and one block per SM with 512):
//  * warps 0 .. 4 NPAR - 1 build A: warp w owns TMEM lanes 32 (w % 4) .. +31
//    (its pixels) for the channels c = w / 4 (mod NPAR). Per channel a thread forms
//    its pixel's range offset, the w tap weights (per-tap polynomials of the
//    ES kernel), the carrier, the BF16 hi/lo parts, shifts them to the taps'
//    position in the 16 KS-row window and writes the row to TMEM
//    (tcgen05.st); one A buffer per channel class, so NPAR - 1 classes are
//    being written while the MMAs read the other;
//  * warp 4 NPAR (one thread) issues the tcgen05.mma chain of each channel and
//    commits its completion to the barriers that free the A buffer and the
//    table slot;
//  * warp 4 NPAR + 1 (one thread) streams the table windows with TMA into a
//    ring of smem slots: per channel ceil(N / 64) boxes (twice that planar:
//    Re and Im columns) of 64 columns x 16 KS rows x hi/lo from the
//    row-major table [c][hi/lo][row][column],
//    written with 128-byte swizzling, which is the MN-major layout the MMA
//    reads (64-column atoms, rows 128 B apart); a window may start at any row.
// At the end the accumulators (2 N FP32 columns) are read back with
// tcgen05.ld and written as G[part][u][y][x].
//
// Every wait is bounded (a clock budget); a wait that runs out sets a bit in
// *err, the block skips the rest of its work and still waits (bounded) for
// its own copies and products before releasing tensor memory. (ta.dbg_wait
// makes the MMA warp wait first on a barrier nothing completes, so that
// tests can run these exit paths.)
#include <cuda_bf16.h>

#include "bp_body.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

namespace {

constexpr int TCX = 16, TCY = 8;
template <int NPAR>
struct Warps {
    static constexpr int compute = 4 * NPAR;          // A-building warps
    static constexpr int threads = (compute + 2) * 32; // + MMA warp + TMA warp
};

// Put the NT words t at word offset wo of an NW-word row, zeros elsewhere
// (a barrel shift over the bits of wo; words pushed past NW are dropped).
template <int NW, int NT>
__device__ __forceinline__ void place(const uint32_t (&t)[NT], int wo, uint32_t (&r)[NW]) {
#pragma unroll
    for (int j = 0; j < NW; ++j) r[j] = j < NT ? t[j] : 0u;
#pragma unroll
    for (int b = 1; b < NW; b <<= 1) {
        const bool on = (wo & b) != 0;
#pragma unroll
        for (int j = NW - 1; j >= 0; --j) r[j] = on ? (j >= b ? r[j - b] : 0u) : r[j];
    }
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
// BF16 pair (a, b) and the BF16 pair of its residuals
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = bf2(a, b);
    lo = bf2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}

// One (pixel, channel) of a tile: the window row o of the first of the w taps
// (0 <= o <= ROWS - w for a window of ROWS rows), the tap weights and the
// carrier e^{j kappa_T a} (sin, cos). The pixel sits (ddx, ddy) from the tile
// centre; g holds the channel's geometry relative to that centre.
template <int W, int ROWS>
__device__ __forceinline__ void channel_taps(const BpDesc &p, const CoefTable &ct, const TileGeo &g,
                                             float ddx, float ddy, float2 kT, int &o,
                                             float (&w)[W], float &sn, float &cs) {
    constexpr int ND = W + 2;                   // polynomial coefficients per tap
    // delta = a - a* from rho^2 - rho*^2 = d (2 D + d): no cancellation
    float ex = g.dxt + ddx, ey = g.dyt + ddy;
    float num = fmaf(ddx, 2.0f * g.dxt + ddx, ddy * (2.0f * g.dyt + ddy));
    float r2 = fmaf(ex, ex, ey * ey);
    float dl = num * __frcp_rn(fmaf(r2, rsqrtf(r2), g.rt));
    if (p.mode == 1) {
        ex = g.dxr + ddx;
        ey = g.dyr + ddy;
        num = fmaf(ddx, 2.0f * g.dxr + ddx, ddy * (2.0f * g.dyr + ddy));
        r2 = fmaf(ex, ex, ey * ey);
        dl += num * __frcp_rn(fmaf(r2, rsqrtf(r2), g.rr));
    }
    // taps: rows o .. o + w - 1 of the window, weights from the per-tap
    // polynomials in s = 2 (pos - o) - (w - 1)
    const float pos = (dl + g.off) * p.inv_h;
    o = min(max((int)ceilf(pos - 0.5f * W), 0), ROWS - W);
    const float s = fmaf(2.0f, pos - (float)o, -(float)(W - 1));
#pragma unroll
    for (int t = 0; t < W; ++t) {
        float acc = ct.c[t][ND - 1];
#pragma unroll
        for (int d = ND - 2; d >= 0; --d) acc = fmaf(acc, s, ct.c[t][d]);
        w[t] = acc;
    }
    // carrier e^{j kappa_T a} = e^{j (kappa_T delta + (kappa_T a* mod 2 pi))}
    const float th = fmaf(kT.x, dl, bp::phase_ff(kT.x, kT.y, g.a_hi, g.a_lo));
    __sincosf(th, &sn, &cs);
}

// Barriers of one block's item: b_full[NSG], done[NSG], a_full[NPAR],
// a_done[NPAR], acc_full (NSG = nst / (NPAR CPR) slot groups).
__host__ __device__ constexpr int tc_barriers(int nsg, int npar) { return 2 * nsg + 2 * npar + 1; }

// One block of the back-projection: 16 x 8 pixel tile, bin block and channel
// part decoded from the linear block index `lin`. The caller has allocated
// tensor memory (`tmem`, tmem_cols columns) and initialised the barriers
// `bars` (layout above: arrival counts 1, 1, 4, 1, 1); on return every copy
// and product the block issued has completed and no arrival on `bars` is
// outstanding, so the caller may re-initialise them for another item.
template <int W, int KS, int SPLIT, int NPAR, bool PLANAR, int CPR>
__device__ __forceinline__ void bp_tc_item(const BpDesc &p, const CoefTable &ct, const TcArgs &ta,
                                           const CUtensorMap *tmap, const TileGeo *__restrict__ tgeo,
                                           const float2 *__restrict__ kc_hl,
                                           float2 *__restrict__ G, int *err, int lin,
                                           unsigned char *smem, uint64_t *bars, uint32_t tmem,
                                           uint64_t *dbg_bar) {
    constexpr int NCW = Warps<NPAR>::compute;
    constexpr int NPL = SPLIT == 3 ? 4 : 2;     // A planes: (re, im) x (hi[, lo])
    constexpr int NW = 8 * KS;                  // 32-bit words of an A row (16 KS BF16)
    constexpr int NT = W / 2 + 1;               // words of the taps after the parity shift
    // Channels go in groups of NPAR (channel c = NPAR g + k, class k); the
    // slots form NSG slot groups of NPAR. b_full[s]: the windows of the group
    // in slot group s landed (TMA); done[s]: that group's products completed
    // (frees the slot group); a_full[k]: A of class k written (its 4 warps);
    // a_done[k]: the products reading class k's A buffer completed.
    const int NSG = ta.nst / (NPAR * CPR);
    uint64_t *b_full = bars;
    uint64_t *done = b_full + NSG;
    uint64_t *a_full = done + NSG;
    uint64_t *a_done = a_full + NPAR;
    uint64_t *acc_full = a_done + NPAR;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // linear block index: tile x fastest, then tile y, then bin block x
    // channel part
    const int nbx = (p.nx + TCX - 1) / TCX, nby = (p.ny + TCY - 1) / TCY;
    const int bx = lin % nbx, by = (lin / nbx) % nby, bz = lin / (nbx * nby);
    const int tile = by * nbx + bx;
    // bz = bin block x channel part: channels [cb, ce) of the tile
    const int utile = bz / ta.nsplit, part = bz - utile * ta.nsplit;
    const int u0 = utile * ta.UT;
    const int C = p.n_chan;
    const int cper = (C + ta.nsplit - 1) / ta.nsplit;
    const int cb = part * cper, ce = min(C, cb + cper);
    const TileGeo *tg = tgeo + (size_t)tile * C;
    const long long budget = ta.budget;
    const uint32_t N = PLANAR ? ta.UT : 2 * ta.UT;     // the MMA's N

    if (warp < NCW) {
        // ------------------------------------------------ A rows (weights)
        const int q = warp & 3, par = warp >> 2;
        const int pix = 32 * q + lane;
        const int px = pix % TCX, py = pix / TCX;
        const float ddx = ((float)px - 0.5f * (TCX - 1)) * p.dxf;
        const float ddy = ((float)py - 0.5f * (TCY - 1)) * p.dyf;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        // class par's round `it` takes channels cb + (it NPAR + par) CPR + j,
        // j < CPR, into its A buffer (CPR channel slots)
        const uint32_t abuf = lane_base + ta.acol + par * (CPR * NPL * KS * 8);
        const float2 kT = kc_hl[u0];
        bool ok = true;
        int it = 0, jc = 0;
        // the geometry of the class's next channel is loaded one channel ahead
        TileGeo gn;
        if (cb + par * CPR < ce) gn = tg[cb + par * CPR];
        for (int c = cb + par * CPR; c < ce;) {
            const TileGeo g = gn;
            const int cnext = jc + 1 < CPR ? c + 1 : c + 1 + (NPAR - 1) * CPR;
            if (cnext < ce) gn = tg[cnext];
            int o;
            float w[W], sn, cs;
            channel_taps<W, 16 * KS>(p, ct, g, ddx, ddy, kT, o, w, sn, cs);
            // element o of the row starts word o / 2; an odd o puts a zero first
            const bool odd = (o & 1) != 0;
            float e[W + 2];
#pragma unroll
            for (int k = 0; k < W + 2; ++k) {
                const float ev = k < W ? w[k] : 0.f;
                const float od = (k >= 1 && k <= W) ? w[k - 1] : 0.f;
                e[k] = odd ? od : ev;
            }
            uint32_t rows[NPL][NW];
            {
                uint32_t tw[NPL][NT];
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const float r0 = e[2 * j] * cs, r1 = e[2 * j + 1] * cs;
                    const float i0 = e[2 * j] * sn, i1 = e[2 * j + 1] * sn;
                    if (SPLIT == 3) {
                        split2(r0, r1, tw[0][j], tw[1][j]);
                        split2(i0, i1, tw[2][j], tw[NPL - 1][j]);
                    } else {
                        tw[0][j] = bf2(r0, r1);
                        tw[1][j] = bf2(i0, i1);
                    }
                }
#pragma unroll
                for (int pl = 0; pl < NPL; ++pl) place<NW, NT>(tw[pl], o >> 1, rows[pl]);
            }
            // before a round's first channel: the products of the class's
            // previous round must be done
            if (CPR == 1 || jc == 0) {
                if (it > 0) ok = tc05::mbar_wait(&a_done[par], (uint32_t)(it - 1) & 1u, budget);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc05::fence_after_sync();
            }
            const int jslot = CPR == 1 ? 0 : jc;
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl)
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    uint32_t v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = rows[pl][8 * ks + j];
                    tc05::tmem_st8(abuf + ((jslot * NPL + pl) * KS + ks) * 8, v);
                }
            // after the round's last channel its A is complete
            const bool round_end = CPR == 1 || jc + 1 == CPR || cnext >= ce;
            if (round_end) {
                tc05::tmem_wait_st();
                tc05::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc05::mbar_arrive(&a_full[par]);
                jc = 0;
                ++it;
            } else {
                ++jc;
            }
            c = cnext;
        }
        // the release of the class's last round has arrived (no arrival on
        // a_done outstanding when the block returns)
        if (ok && it > 0) ok = __all_sync(0xffffffffu, tc05::mbar_wait(&a_done[par], (uint32_t)(it - 1) & 1u, budget));
        if (!ok && lane == 0) atomicOr(err, 1);

        // ------------------------------------------------ epilogue
        bool done = tc05::mbar_wait(acc_full, 0, budget);
        done = __all_sync(0xffffffffu, done);
        if (done) {
            tc05::fence_after_sync();
            const int ix = bx * TCX + px, iy = by * TCY + py;
            const bool inside = ix < p.nx && iy < p.ny;
            const size_t plane = (size_t)p.nx * p.ny;
            const size_t pofs = (size_t)iy * p.nx + ix;
            // this channel part's spectrum, or the one all parts add into
            float2 *Gp = G + (size_t)(ta.g_atomic ? 0 : part) * p.n_pad * plane;
            for (int ch = par; ch < (int)(N / 16); ch += NPAR) {
                uint32_t pv[16], qv[16];
                tc05::tmem_ld16(lane_base + 16 * ch, pv);
                tc05::tmem_ld16(lane_base + N + 16 * ch, qv);
                tc05::tmem_wait_ld();
                if (!inside) continue;
                // planar: 16 bins (Re G, Im G columns); interleaved: 8 bins
                // (re, im pairs of P and Q)
                constexpr int NB = PLANAR ? 16 : 8;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int u = u0 + NB * ch + b;
                    if (u >= p.n_pad) continue;
                    const float2 v =
                        PLANAR ? make_float2(__uint_as_float(pv[b]), __uint_as_float(qv[b]))
                               : make_float2(__uint_as_float(pv[2 * b]) - __uint_as_float(qv[2 * b + 1]),
                                             __uint_as_float(pv[2 * b + 1]) + __uint_as_float(qv[2 * b]));
                    if (ta.g_atomic)
                        atomicAdd(&Gp[u * plane + pofs], v);
                    else
                        Gp[u * plane + pofs] = v;
                }
            }
        } else if (lane == 0) {
            atomicOr(err, 2);
        }
    } else if (warp == NCW) {
        // ------------------------------------------------ MMA issue
        // The whole warp runs the loop on warp-uniform counters (so addresses
        // and descriptors stay in uniform registers); one lane issues. One
        // pass per group of NPAR channels: one wait for the group's windows,
        // then per class a wait for its A, its products and a commit that
        // frees its A buffer; one commit frees the group's slots.
        const uint32_t lo16 = (16 * KS * 128) >> 4;       // lo plane, 16-byte units
        const uint64_t d0 = tc05::smem_desc_sw128(tc05::smem_addr(smem), ta.cb_bytes, 1024);
        const uint32_t slot16 = ta.slot_bytes >> 4;
        const uint32_t abase = tmem + ta.acol;
        constexpr int PG = NPAR * CPR;                       // channels per slot group
        const int n_groups = (ce - cb + PG - 1) / PG;
        const uint32_t im16 = ta.im_off >> 4;              // Im B columns (planar)
        const uint32_t idn = ta.idesc | (1u << 13);        // negated A
        bool ok = true;
        if (ta.dbg_wait) ok = __all_sync(0xffffffffu, tc05::mbar_wait(dbg_bar, 0, budget));
        int sg = 0;
        uint32_t bpar = 0;
        for (int g = 0; g < n_groups && ok; ++g) {
            const int nleft = ce - cb - g * PG;              // channels of the group
            ok = tc05::mbar_wait(&b_full[sg], bpar, budget);
#pragma unroll
            for (int k = 0; k < NPAR; ++k) {
                if (k * CPR >= nleft) break;
                ok = ok && tc05::mbar_wait(&a_full[k], (uint32_t)g & 1u, budget);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc05::fence_after_sync();
                if (lane == 0) {
#pragma unroll
                  for (int j = 0; j < CPR; ++j) {
                    if (k * CPR + j >= nleft) break;
                    const uint32_t a0 = abase + (k * CPR + j) * (NPL * KS * 8);
                    const uint64_t dk = d0 + (uint64_t)(((sg * NPAR + k) * CPR + j) * slot16);
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        const uint64_t bh = dk + (uint64_t)(ks * (2048 >> 4));
                        const uint32_t acc = (g > 0 || k > 0 || j > 0 || ks > 0) ? 1u : 0u;
                        if (PLANAR) {
                            // Re G += Re A Re B - Im A Im B, Im G += Re A Im B + Im A Re B
                            const uint64_t bi = bh + im16;
                            if (SPLIT == 3) {
                                const uint64_t bl = bh + lo16, bil = bi + lo16;
                                const uint32_t ar = a0 + (0 * KS + ks) * 8, arl = a0 + (1 * KS + ks) * 8;
                                const uint32_t ai = a0 + (2 * KS + ks) * 8, ail = a0 + (3 * KS + ks) * 8;
                                tc05::mma_ts(tmem, ar, bh, ta.idesc, acc);
                                tc05::mma_ts(tmem, ar, bl, ta.idesc, 1u);
                                tc05::mma_ts(tmem, arl, bh, ta.idesc, 1u);
                                tc05::mma_ts(tmem, ai, bi, idn, 1u);
                                tc05::mma_ts(tmem, ai, bil, idn, 1u);
                                tc05::mma_ts(tmem, ail, bi, idn, 1u);
                                tc05::mma_ts(tmem + N, ar, bi, ta.idesc, acc);
                                tc05::mma_ts(tmem + N, ar, bil, ta.idesc, 1u);
                                tc05::mma_ts(tmem + N, arl, bi, ta.idesc, 1u);
                                tc05::mma_ts(tmem + N, ai, bh, ta.idesc, 1u);
                                tc05::mma_ts(tmem + N, ai, bl, ta.idesc, 1u);
                                tc05::mma_ts(tmem + N, ail, bh, ta.idesc, 1u);
                            } else {
                                const uint32_t ar = a0 + ks * 8, ai = a0 + (KS + ks) * 8;
                                tc05::mma_ts(tmem, ar, bh, ta.idesc, acc);
                                tc05::mma_ts(tmem, ai, bi, idn, 1u);
                                tc05::mma_ts(tmem + N, ar, bi, ta.idesc, acc);
                                tc05::mma_ts(tmem + N, ai, bh, ta.idesc, 1u);
                            }
                        } else if (SPLIT == 3) {
                            const uint64_t bl = bh + lo16;
                            tc05::mma_ts(tmem, a0 + (0 * KS + ks) * 8, bh, ta.idesc, acc);
                            tc05::mma_ts(tmem, a0 + (0 * KS + ks) * 8, bl, ta.idesc, 1u);
                            tc05::mma_ts(tmem, a0 + (1 * KS + ks) * 8, bh, ta.idesc, 1u);
                            tc05::mma_ts(tmem + N, a0 + (2 * KS + ks) * 8, bh, ta.idesc, acc);
                            tc05::mma_ts(tmem + N, a0 + (2 * KS + ks) * 8, bl, ta.idesc, 1u);
                            tc05::mma_ts(tmem + N, a0 + (3 * KS + ks) * 8, bh, ta.idesc, 1u);
                        } else {
                            tc05::mma_ts(tmem, a0 + ks * 8, bh, ta.idesc, acc);
                            tc05::mma_ts(tmem + N, a0 + (KS + ks) * 8, bh, ta.idesc, acc);
                        }
                    }
                  }
                    tc05::mma_commit(&a_done[k]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) tc05::mma_commit(&done[sg]);
            __syncwarp();
            if (++sg == NSG) {
                sg = 0;
                bpar ^= 1u;
            }
        }
        if (lane == 0) {
            if (!ok) atomicOr(err, 4);
            tc05::mma_commit(acc_full);
        }
    } else {
        // ------------------------------------------------ TMA producer
        // (the whole warp runs the loop; one lane issues the copies)
        constexpr int PG = NPAR * CPR;                       // channels per slot group
        const int n_groups = (ce - cb + PG - 1) / PG;
        bool ok = true;
        int issued = 0;          // groups issued
        int sg = 0;
        uint32_t dpar = 0;
        int ilo_next[PG];        // first window rows, one group ahead
#pragma unroll
        for (int k = 0; k < PG; ++k) ilo_next[k] = cb + k < ce ? tg[cb + k].ilo : 0;
        for (int g = 0; g < n_groups; ++g) {
            const int nch = min(PG, ce - cb - g * PG);
            int ilo[PG];
#pragma unroll
            for (int k = 0; k < PG; ++k) {
                ilo[k] = ilo_next[k];
                const int cn = cb + (g + 1) * PG + k;
                if (cn < ce) ilo_next[k] = tg[cn].ilo;
            }
            // group g reuses the slot group of group g - NSG: phase g / NSG - 1
            if (g >= NSG) ok = tc05::mbar_wait(&done[sg], dpar, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (lane == 0) {
                tc05::mbar_arrive_expect_tx(&b_full[sg], (uint32_t)nch * ta.slot_bytes);
#pragma unroll
                for (int k = 0; k < PG; ++k) {
                    if (k >= nch) break;
                    unsigned char *dst = smem + (size_t)(sg * PG + k) * ta.slot_bytes;
                    const int cz = 2 * (cb + g * PG + k);
                    for (int j = 0; j < ta.ncb; ++j) {
                        // planar: the Re columns of the bins, then (im_off bytes
                        // on) their Im columns; interleaved: (re, im) pairs
                        tc05::tma_load_3d(dst + (size_t)j * ta.cb_bytes, tmap, &b_full[sg],
                                          (PLANAR ? u0 : 2 * u0) + 64 * j, ilo[k], cz);
                        if (PLANAR)
                            tc05::tma_load_3d(dst + ta.im_off + (size_t)j * ta.cb_bytes, tmap,
                                              &b_full[sg], ta.im_col + u0 + 64 * j, ilo[k], cz);
                    }
                }
            }
            issued = g + 1;
            if (++sg == NSG) {
                sg = 0;
                if (g + 1 >= 2 * NSG) dpar ^= 1u;
            }
        }
        // every issued copy has landed before the block can exit, and the
        // products of every issued group have released its slot group (no
        // arrival on b_full or done outstanding)
        if (lane == 0) {
            if (!ok) atomicOr(err, 8);
            for (int s = 0; s < NSG && s < issued; ++s) {
                const int n_s = (issued - 1 - s) / NSG + 1;   // groups loaded into slot group s
                if (!tc05::mbar_wait(&b_full[s], (n_s - 1) & 1, budget)) atomicOr(err, 16);
                if (ok && !tc05::mbar_wait(&done[s], (n_s - 1) & 1, budget)) atomicOr(err, 32);
            }
        }
    }
}

// Compressed 2:4-sparse A rows of one (pixel, channel) for a window of RW
// rows taken in residue order: NG = RW / 4 residue classes j of four rows
// each (row j + NG e at K position 4 j + e, e < 4). Taps t < NG fall in
// distinct classes j = (o + t) mod NG at e = (o + t) / NG, tap t + NG (< w)
// in the same class at e + 1, so each class holds at most two taps (w <=
// 2 NG). Kept pair of class j: positions (e, e + 1) with values (w_t, w_{t+NG}
// or 0), or (2, 3) with (0, w_t) when a lone tap sits at e = 3. The K = 32
// operand is [Re rows | Im rows] (classes 0 .. NG - 1 of each, then zero
// groups when NG = 3), so the rows are a1 = [Re A | -Im A] and a3 = [Im A |
// Re A] (BF16 hi, and lo for SPLIT 3; word k = the kept pair of K group k)
// and mA, mB the metadata of K 0..15 and 16..31.
// INTER (interleaved layout, RW = 16, SPLIT = 3): the K = 32 operand is
// instead the window's [hi rows | lo rows] and the rows are a1 = [Re A_hi |
// Re A_hi], a3 = [Im A_hi | Im A_hi] (products A_hi b_hi + A_hi b_lo) and
// a1l = [Re A_lo | 0], a3l = [Im A_lo | 0] (A_lo b_hi).
template <int W, int RW, int SPLIT, bool INTER = false>
__device__ __forceinline__ void sparse_rows(int o, const float (&w)[W], float sn, float cs,
                                            uint32_t (&a1h)[8], uint32_t (&a3h)[8],
                                            uint32_t (&a1l)[8], uint32_t (&a3l)[8],
                                            uint32_t &mA, uint32_t &mB) {
    constexpr int NG = RW / 4;
    static_assert(RW == 16 || RW == 12, "window rows");
    static_assert(W <= 2 * NG, "at most two taps per residue class");
    const int r = o % NG, ob = o / NG;
    float kv0[NG], kv1[NG];
    uint32_t nib[NG];
#pragma unroll
    for (int t = 0; t < NG; ++t) {
        const int e = ob + ((r + t) >= NG ? 1 : 0);
        const bool two = t + NG < W;
        const float first = w[t];
        const float second = two ? w[t + NG < W ? t + NG : t] : 0.f;
        const bool top = !two && e == 3;
        kv0[t] = top ? 0.f : first;
        kv1[t] = top ? first : second;
        const uint32_t i0 = top ? 2u : (uint32_t)e;
        nib[t] = i0 | ((i0 + 1u) << 2);
    }
    // rotate from tap order t to class order j = (t + r) mod NG, one step at
    // a time
#pragma unroll
    for (int step = 1; step < NG; ++step) {
        if (step <= r) {
            const float l0 = kv0[NG - 1], l1 = kv1[NG - 1];
            const uint32_t ln = nib[NG - 1];
#pragma unroll
            for (int j = NG - 1; j > 0; --j) {
                kv0[j] = kv0[j - 1];
                kv1[j] = kv1[j - 1];
                nib[j] = nib[j - 1];
            }
            kv0[0] = l0;
            kv1[0] = l1;
            nib[0] = ln;
        }
    }
    constexpr uint32_t NEG = 0x80008000u;
    constexpr uint32_t PAD = 0x4u;                  // kept positions (0, 1), values zero
#pragma unroll
    for (int k = 0; k < 8; ++k) a1h[k] = a3h[k] = a1l[k] = a3l[k] = 0u;
    uint32_t nb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) nb[k] = PAD;
#pragma unroll
    for (int j = 0; j < NG; ++j) {
        const float r0 = kv0[j] * cs, r1 = kv1[j] * cs;
        const float i0 = kv0[j] * sn, i1 = kv1[j] * sn;
        uint32_t rh, rl, ih, il;
        if (SPLIT == 3) {
            split2(r0, r1, rh, rl);
            split2(i0, i1, ih, il);
        } else {
            rh = bf2(r0, r1);
            ih = bf2(i0, i1);
            rl = il = 0u;
        }
        if (INTER) {
            a1h[j] = a1h[NG + j] = rh;
            a3h[j] = a3h[NG + j] = ih;
            a1l[j] = rl;
            a3l[j] = il;
        } else {
            a1h[j] = rh;
            a1h[NG + j] = ih ^ NEG;
            a3h[j] = ih;
            a3h[NG + j] = rh;
            a1l[j] = rl;
            a1l[NG + j] = il ^ NEG;
            a3l[j] = il;
            a3l[NG + j] = rl;
        }
        nb[j] = nb[NG + j] = nib[j];
    }
    mA = nb[0] | (nb[1] << 4) | (nb[2] << 8) | (nb[3] << 12);
    mB = nb[4] | (nb[5] << 4) | (nb[6] << 8) | (nb[7] << 12);
}

// Compressed 2:4-sparse A rows of one (pixel, channel) for a 32-row window
// (the interleaved layout, K = the window's 32 rows): residue classes j of
// the rows mod 4, row j + 4 e at K position 8 j + e (e < 8), so class j
// spans the K groups 2 j and 2 j + 1. Taps t < 4 fall in distinct classes j
// = (o + t) mod 4 at e = (o + t) / 4, tap t + 4 (< w) at e + 1: at most two
// taps per class, in one group or straddling the two (e = 3, e + 1 = 4).
// Each group keeps a pair of positions; a group without a tap keeps (0, 1)
// with zero values. Rows re = Re A, im = Im A (BF16 hi, and lo for SPLIT 3;
// word k = the kept pair of K group k); mA, mB the metadata of K 0..15 and
// 16..31.
template <int W, int SPLIT>
__device__ __forceinline__ void sparse_rows32(int o, const float (&w)[W], float sn, float cs,
                                              uint32_t (&reh)[8], uint32_t (&imh)[8],
                                              uint32_t (&rel)[8], uint32_t (&iml)[8],
                                              uint32_t &mA, uint32_t &mB) {
    static_assert(W <= 8, "at most two taps per residue class");
    constexpr uint32_t PAD = 0x4u;                  // kept positions (0, 1)
    const int r = o & 3, ob = o >> 2;
    // per tap t < 4 (its class): the kept pairs of the class's two groups
    float v0[4][2], v1[4][2];
    uint32_t nb[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int e = ob + ((r + t) >> 2);           // 0 .. 7
        const int hi = e >> 2, pos = e & 3;
        const bool two = t + 4 < W;
        const float first = w[t];
        const float second = two ? w[t + 4 < W ? t + 4 : t] : 0.f;
        const bool straddle = two && pos == 3;       // e = 3: second tap at e = 4
        // the group holding the (first) tap
        float a0, a1;
        uint32_t n;
        if (pos <= 2) {
            a0 = first;
            a1 = second;
            n = (uint32_t)pos | ((uint32_t)(pos + 1) << 2);
        } else {
            a0 = 0.f;
            a1 = first;
            n = 2u | (3u << 2);
        }
        // the other group keeps (0, 1) with zeros, except when straddling
        // (then hi = 0): group 1 keeps (0, 1) = (w_{t+4}, 0)
        const bool h1 = hi != 0;
        v0[t][0] = h1 ? 0.f : a0;
        v1[t][0] = h1 ? 0.f : a1;
        nb[t][0] = h1 ? PAD : n;
        v0[t][1] = h1 ? a0 : (straddle ? second : 0.f);
        v1[t][1] = h1 ? a1 : 0.f;
        nb[t][1] = h1 ? n : PAD;
    }
    // rotate from tap order t to class order j = (t + r) mod 4
#pragma unroll
    for (int step = 1; step < 4; ++step) {
        if (step <= r) {
            float l0[2], l1[2];
            uint32_t ln[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                l0[h] = v0[3][h];
                l1[h] = v1[3][h];
                ln[h] = nb[3][h];
            }
#pragma unroll
            for (int j = 3; j > 0; --j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    v0[j][h] = v0[j - 1][h];
                    v1[j][h] = v1[j - 1][h];
                    nb[j][h] = nb[j - 1][h];
                }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                v0[0][h] = l0[h];
                v1[0][h] = l1[h];
                nb[0][h] = ln[h];
            }
        }
    }
    uint32_t g[8];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * j + h;
            const float r0 = v0[j][h] * cs, r1 = v1[j][h] * cs;
            const float i0 = v0[j][h] * sn, i1 = v1[j][h] * sn;
            if (SPLIT == 3) {
                split2(r0, r1, reh[k], rel[k]);
                split2(i0, i1, imh[k], iml[k]);
            } else {
                reh[k] = bf2(r0, r1);
                imh[k] = bf2(i0, i1);
                rel[k] = iml[k] = 0u;
            }
            g[k] = nb[j][h];
        }
    mA = g[0] | (g[1] << 4) | (g[2] << 8) | (g[3] << 12);
    mB = g[4] | (g[5] << 4) | (g[6] << 8) | (g[7] << 12);
}

// The same block with 2:4-sparse products (planar layout, one 16-row window
// per channel, one channel per class round). The window's rows are taken in
// residue order, K index 4 j + e <-> window row j + 4 e (j, e < 4): a pixel's
// w <= 8 taps, consecutive rows o .. o + w - 1, put at most two in each
// group of four K indices, so each A row is 2:4 sparse. The B operand of one
// sparse product (K = 32) is the window's Re rows followed by its Im rows,
// S = [Re b; Im b] (a 5-D TMA box: 64 columns x 4 x 4 rows x Re / Im x hi /
// lo), and the complex product becomes
//   Re G += [Re A | -Im A] S,   Im G += [Im A | Re A] S,
// so a channel takes six sparse products (hi/lo split: A_hi S_hi, A_hi S_lo,
// A_lo S_hi for each accumulator) instead of twelve dense ones. Each class
// buffer holds the four compressed A matrices (8 columns each: 8 kept values
// per K half); the kept positions, the same in both K halves, go to the
// class's metadata column. Each class buffer is filled by NSET sets of four
// warps in turn (set s takes the class's rounds r = s mod NSET), so that one
// set computes its next channel while another's is stored and multiplied.
// A set may overwrite the buffer for round r only when round r - 1 (stored
// by another set) has been consumed. The products of round r release it on
// a_done[class][r mod NSET], so that each release barrier runs through the
// rounds of one set: a waiter never falls two phases behind the barrier it
// tests (the parity of a phase test would not tell them apart).
template <int W, int SPLIT, int NPAR, int NSET, int RW, bool PLANAR>
__device__ __forceinline__ void bp_tc_item_sp(const BpDesc &p, const CoefTable &ct,
                                              const TcArgs &ta, const CUtensorMap *tmap,
                                              const TileGeo *__restrict__ tgeo,
                                              const float2 *__restrict__ kc_hl,
                                              float2 *__restrict__ G, int *err, int lin,
                                              unsigned char *smem, uint64_t *bars, uint32_t tmem,
                                              uint64_t *dbg_bar) {
    static_assert(W == 4 || W == 6 || W == 8, "taps");
    constexpr int NCW = 4 * NPAR * NSET;         // A-building warps
    // compressed A matrices per channel: Re A, Im A (hi, lo); planar 32-row
    // windows also -Im A (the Re and Im rows are separate K = 32 operands)
    constexpr bool P32 = PLANAR && RW == 32;
    constexpr int NMAT = (SPLIT == 3 ? 4 : 2) + (P32 ? (SPLIT == 3 ? 2 : 1) : 0);
    const int NSG = ta.nst / NPAR;
    uint64_t *b_full = bars;
    uint64_t *done = b_full + NSG;
    uint64_t *a_full = done + NSG;
    uint64_t *a_done = a_full + NPAR;            // [class][set]
    uint64_t *acc_full = a_done + NPAR * NSET;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbx = (p.nx + TCX - 1) / TCX, nby = (p.ny + TCY - 1) / TCY;
    const int bx = lin % nbx, by = (lin / nbx) % nby, bz = lin / (nbx * nby);
    const int tile = by * nbx + bx;
    const int utile = bz / ta.nsplit, part = bz - utile * ta.nsplit;
    const int u0 = utile * ta.UT;
    const int C = p.n_chan;
    const int cper = (C + ta.nsplit - 1) / ta.nsplit;
    const int cb = part * cper, ce = min(C, cb + cper);
    const TileGeo *tg = tgeo + (size_t)tile * C;
    const long long budget = ta.budget;
    // the MMA's N: planar Re G, Im G (UT columns each); interleaved P, Q (2 UT)
    const uint32_t N = PLANAR ? ta.UT : 2 * ta.UT;

    if (warp < NCW) {
        // ------------------------------------------------ A rows (compressed)
        const int q = warp & 3, par = (warp >> 2) % NPAR, set = (warp >> 2) / NPAR;
        const int pix = 32 * q + lane;
        const int px = pix % TCX, py = pix / TCX;
        const float ddx = ((float)px - 0.5f * (TCX - 1)) * p.dxf;
        const float ddy = ((float)py - 0.5f * (TCY - 1)) * p.dyf;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t abuf = lane_base + ta.acol + par * (NMAT * 8);
        const uint32_t mbuf = lane_base + ta.mcol + par * 8;
        const float2 kT = kc_hl[u0];
        bool ok = true;
        const int rounds = ce - cb > par ? (ce - cb - par + NPAR - 1) / NPAR : 0;
        // round r's release: barrier a_done[par][r mod NSET], its phase r / NSET
        auto released = [&](int r) {
            return tc05::mbar_wait(&a_done[par * NSET + r % NSET], (uint32_t)(r / NSET) & 1u,
                                   budget);
        };
        constexpr int STEP = NPAR * NSET;
        TileGeo gn;
        if (cb + par + NPAR * set < ce) gn = tg[cb + par + NPAR * set];
        for (int it = set; it < rounds; it += NSET) {
            const int c = cb + par + NPAR * it;
            const TileGeo g = gn;
            if (c + STEP < ce) gn = tg[c + STEP];
            int o;
            float w[W], sn, cs;
            channel_taps<W, RW>(p, ct, g, ddx, ddy, kT, o, w, sn, cs);
            // planar: a1 = [Re A | -Im A], a3 = [Im A | Re A] over [Re rows |
            // Im rows]; interleaved (32 rows): a1 = Re A, a3 = Im A
            uint32_t a1h[8], a3h[8], a1l[8], a3l[8], mA, mB;
            if constexpr (RW == 32)
                sparse_rows32<W, SPLIT>(o, w, sn, cs, a1h, a3h, a1l, a3l, mA, mB);
            else
                sparse_rows<W, RW, SPLIT, !PLANAR>(o, w, sn, cs, a1h, a3h, a1l, a3l, mA, mB);
            // metadata word of this lane: rows (r, r + 8) of its 16-lane block,
            // K 0..15 in lanes r < 8 and K 16..31 in lanes r + 8
            const uint32_t oA = __shfl_xor_sync(0xffffffffu, mA, 8);
            const uint32_t oB = __shfl_xor_sync(0xffffffffu, mB, 8);
            const uint32_t mword = (lane & 8) ? (oB | (mB << 16)) : (mA | (oA << 16));
            // round it - 1 consumed (and with it every earlier round)
            if (it > 0) ok = released(it - 1);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc05::fence_after_sync();
            tc05::tmem_st8(abuf, a1h);                         // a1 hi
            tc05::tmem_st8(abuf + 8, a3h);                     // a3 hi
            if (SPLIT == 3) {
                tc05::tmem_st8(abuf + 16, a1l);                // a1 lo
                tc05::tmem_st8(abuf + 24, a3l);                // a3 lo
            }
            if constexpr (P32) {
                // -Im A (hi, lo) after them
                constexpr uint32_t NEG = 0x80008000u;
                uint32_t v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = a3h[j] ^ NEG;
                tc05::tmem_st8(abuf + (SPLIT == 3 ? 32 : 16), v);
                if (SPLIT == 3) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = a3l[j] ^ NEG;
                    tc05::tmem_st8(abuf + 40, v);
                }
            }
            tc05::tmem_st1(mbuf, mword);
            tc05::tmem_wait_st();
            tc05::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&a_full[par]);
        }
        // the class's last round released: every release has arrived (none
        // outstanding on exit)
        if (ok && rounds > 0) ok = released(rounds - 1);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicOr(err, 1);

        // ------------------------------------------------ epilogue
        bool fin = __all_sync(0xffffffffu, tc05::mbar_wait(acc_full, 0, budget));
        if (fin) {
            tc05::fence_after_sync();
            const int ix = bx * TCX + px, iy = by * TCY + py;
            const bool inside = ix < p.nx && iy < p.ny;
            const size_t plane = (size_t)p.nx * p.ny;
            const size_t pofs = (size_t)iy * p.nx + ix;
            float2 *Gp = G + (size_t)(ta.g_atomic ? 0 : part) * p.n_pad * plane;
            for (int ch = warp >> 2; ch < (int)(N / 16); ch += NPAR * NSET) {
                uint32_t pv[16], qv[16];
                tc05::tmem_ld16(lane_base + 16 * ch, pv);
                tc05::tmem_ld16(lane_base + N + 16 * ch, qv);
                tc05::tmem_wait_ld();
                if (!inside) continue;
                // planar: 16 bins (Re G, Im G columns); interleaved: 8 bins
                // ((re, im) pairs of P and Q: G = (P_re - Q_im, P_im + Q_re))
                constexpr int NB = PLANAR ? 16 : 8;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int u = u0 + NB * ch + b;
                    if (u >= p.n_pad) continue;
                    const float2 v =
                        PLANAR ? make_float2(__uint_as_float(pv[b]), __uint_as_float(qv[b]))
                               : make_float2(__uint_as_float(pv[2 * b]) - __uint_as_float(qv[2 * b + 1]),
                                             __uint_as_float(pv[2 * b + 1]) + __uint_as_float(qv[2 * b]));
                    if (ta.g_atomic)
                        atomicAdd(&Gp[u * plane + pofs], v);
                    else
                        Gp[u * plane + pofs] = v;
                }
            }
        } else if (lane == 0) {
            atomicOr(err, 2);
        }
    } else if (warp == NCW) {
        // ------------------------------------------------ MMA issue
        const uint64_t d0 = tc05::smem_desc_sw128(tc05::smem_addr(smem), ta.cb_bytes, 1024);
        const uint32_t slot16 = ta.slot_bytes >> 4;
        // S_lo after S_hi: planar [Re rows; Im rows], interleaved the rows
        const uint32_t lo16 = (uint32_t)(RW * (PLANAR ? 2 : 1) * 128) >> 4;
        const uint32_t idsp = ta.idesc | (1u << 2);        // 2:4 sparse A
        const int n_groups = (ce - cb + NPAR - 1) / NPAR;
        bool ok = true;
        if (ta.dbg_wait) ok = __all_sync(0xffffffffu, tc05::mbar_wait(dbg_bar, 0, budget));
        int sg = 0;
        uint32_t bpar = 0;
        for (int g = 0; g < n_groups && ok; ++g) {
            const int nleft = ce - cb - g * NPAR;
            ok = tc05::mbar_wait(&b_full[sg], bpar, budget);
#pragma unroll
            for (int k = 0; k < NPAR; ++k) {
                if (k >= nleft) break;
                ok = ok && tc05::mbar_wait(&a_full[k], (uint32_t)g & 1u, budget);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc05::fence_after_sync();
                if (lane == 0) {
                    const uint32_t a1 = tmem + ta.acol + k * (NMAT * 8);
                    const uint32_t meta = tmem + ta.mcol + k * 8;
                    const uint64_t sh = d0 + (uint64_t)((sg * NPAR + k) * slot16);
                    const uint32_t acc = (g > 0 || k > 0) ? 1u : 0u;
                    if constexpr (P32) {
                        // planar 32-row windows: K = the Re rows, then the Im
                        // rows, of the window (Re b, Im b; hi, lo planes)
                        //   Re G += Re A Re b + (-Im A) Im b
                        //   Im G += Im A Re b + Re A Im b
                        constexpr uint32_t PART16 = (32 * 128) >> 4;
                        const uint64_t rbh = sh, ibh = sh + PART16;
                        const uint32_t ar = a1, ai = a1 + 8;
                        const uint32_t ani = a1 + (SPLIT == 3 ? 32 : 16);
                        tc05::mma_sp_ts(tmem, ar, rbh, meta, idsp, acc);
                        tc05::mma_sp_ts(tmem, ani, ibh, meta, idsp, 1u);
                        tc05::mma_sp_ts(tmem + N, ai, rbh, meta, idsp, acc);
                        tc05::mma_sp_ts(tmem + N, ar, ibh, meta, idsp, 1u);
                        if (SPLIT == 3) {
                            const uint64_t rbl = sh + 2 * PART16, ibl = sh + 3 * PART16;
                            const uint32_t arl = a1 + 16, ail = a1 + 24, anil = a1 + 40;
                            tc05::mma_sp_ts(tmem, ar, rbl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem, arl, rbh, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem, ani, ibl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem, anil, ibh, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, ai, rbl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, ail, rbh, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, ar, ibl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, arl, ibh, meta, idsp, 1u);
                        }
                    } else {
                        // planar: Re G += [Re A | -Im A] S, Im G += [Im A | Re A] S;
                        // interleaved: P += Re A B, Q += Im A B
                        tc05::mma_sp_ts(tmem, a1, sh, meta, idsp, acc);
                        tc05::mma_sp_ts(tmem + N, a1 + 8, sh, meta, idsp, acc);
                        if (SPLIT == 3 && (PLANAR || RW == 32)) {
                            const uint64_t sl = sh + lo16;
                            tc05::mma_sp_ts(tmem, a1, sl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem, a1 + 16, sh, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, a1 + 8, sl, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, a1 + 24, sh, meta, idsp, 1u);
                        } else if (SPLIT == 3) {
                            // interleaved 16-row windows: S = [hi rows | lo rows],
                            // the first two products took A_hi (b_hi + b_lo)
                            tc05::mma_sp_ts(tmem, a1 + 16, sh, meta, idsp, 1u);
                            tc05::mma_sp_ts(tmem + N, a1 + 24, sh, meta, idsp, 1u);
                        }
                    }
                    tc05::mma_commit(&a_done[k * NSET + g % NSET]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (lane == 0) tc05::mma_commit(&done[sg]);
            __syncwarp();
            if (++sg == NSG) {
                sg = 0;
                bpar ^= 1u;
            }
        }
        if (lane == 0) {
            if (!ok) atomicOr(err, 4);
            tc05::mma_commit(acc_full);
        }
    } else {
        // ------------------------------------------------ TMA producer
        const int n_groups = (ce - cb + NPAR - 1) / NPAR;
        bool ok = true;
        int issued = 0;
        int sg = 0;
        uint32_t dpar = 0;
        int ilo_next[NPAR];
#pragma unroll
        for (int k = 0; k < NPAR; ++k) ilo_next[k] = cb + k < ce ? tg[cb + k].ilo : 0;
        for (int g = 0; g < n_groups; ++g) {
            const int nch = min(NPAR, ce - cb - g * NPAR);
            int ilo[NPAR];
#pragma unroll
            for (int k = 0; k < NPAR; ++k) {
                ilo[k] = ilo_next[k];
                const int cn = cb + (g + 1) * NPAR + k;
                if (cn < ce) ilo_next[k] = tg[cn].ilo;
            }
            if (g >= NSG) ok = tc05::mbar_wait(&done[sg], dpar, budget);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (lane == 0) {
                // the bytes the copies deliver (a 12-row window's pad is not copied)
                tc05::mbar_arrive_expect_tx(&b_full[sg],
                                            (uint32_t)(nch * ta.ncb) * ta.cb_bytes);
#pragma unroll
                for (int k = 0; k < NPAR; ++k) {
                    if (k >= nch) break;
                    unsigned char *dst = smem + (size_t)(sg * NPAR + k) * ta.slot_bytes;
                    const int cz = 2 * (cb + g * NPAR + k);
                    // rows ilo + j + NG e: group ilo / NG + e, row-in-group
                    // ilo % NG + j (NG = RW / 4)
                    constexpr int NG = RW == 12 ? 3 : 4;
                    const int a0 = ilo[k] / NG, g0 = ilo[k] - a0 * NG;
                    const int x0 = PLANAR ? u0 : 2 * u0;
                    for (int j = 0; j < ta.ncb; ++j)
                        tc05::tma_load_5d(dst + (size_t)j * ta.cb_bytes, tmap, &b_full[sg],
                                          x0 + 64 * j, a0, g0, 0, cz);
                }
            }
            issued = g + 1;
            if (++sg == NSG) {
                sg = 0;
                if (g + 1 >= 2 * NSG) dpar ^= 1u;
            }
        }
        if (lane == 0) {
            if (!ok) atomicOr(err, 8);
            for (int s = 0; s < NSG && s < issued; ++s) {
                const int n_s = (issued - 1 - s) / NSG + 1;
                if (!tc05::mbar_wait(&b_full[s], (n_s - 1) & 1, budget)) atomicOr(err, 16);
                if (ok && !tc05::mbar_wait(&done[s], (n_s - 1) & 1, budget)) atomicOr(err, 32);
            }
        }
    }
}

// The per-scan kernel: one block per (tile, bin block, channel part) from
// ta.blk0 on (a launch may cover a range of blocks); the barriers follow the
// window slots in shared memory.
template <int W, int KS, int SPLIT, int NPAR, bool PLANAR, int CPR>
__global__ void __launch_bounds__(Warps<NPAR>::threads, NPAR == 2 ? 2 : 1)
k_backproject_tc(BpDesc p, CoefTable ct, TcArgs ta, const __grid_constant__ CUtensorMap tmap,
                 const TileGeo *__restrict__ tgeo, const float2 *__restrict__ kc_hl,
                 float2 *__restrict__ G, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled TMA destinations and MMA operands sit on 1024-byte boundaries
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int NSG = ta.nst / (NPAR * CPR);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)ta.nst * ta.slot_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + tc_barriers(NSG, NPAR));
    __shared__ __align__(8) uint64_t dbg_bar;    // test hook: never completed
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc05::mbar_init(&dbg_bar, 1);
        for (int s = 0; s < NSG; ++s) {
            tc05::mbar_init(&bars[s], 1);
            tc05::mbar_init(&bars[NSG + s], 1);
        }
        for (int k = 0; k < NPAR; ++k) {
            tc05::mbar_init(&bars[2 * NSG + k], 4);
            tc05::mbar_init(&bars[2 * NSG + NPAR + k], 1);
        }
        tc05::mbar_init(&bars[2 * NSG + 2 * NPAR], 1);
        tc05::fence_mbar_init();
    }
    if (warp == 0) {
        tc05::tmem_alloc(tmem_slot, ta.tmem_cols);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bp_tc_item<W, KS, SPLIT, NPAR, PLANAR, CPR>(p, ct, ta, &tmap, tgeo, kc_hl, G, err,
                                               (int)blockIdx.x + ta.blk0, smem, bars, tmem,
                                               &dbg_bar);
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, ta.tmem_cols);
}

// The per-scan kernel of the sparse products (planar, 16-row windows, one
// channel per class round).
template <int NPAR, int NSET>
struct SpWarps {
    static constexpr int threads = (4 * NPAR * NSET + 2) * 32;   // + MMA warp + TMA warp
};

template <int W, int SPLIT, int NPAR, int NSET, int RW, bool PLANAR>
__global__ void __launch_bounds__(SpWarps<NPAR, NSET>::threads, 1)
k_backproject_tc_sp(BpDesc p, CoefTable ct, TcArgs ta, const __grid_constant__ CUtensorMap tmap,
                    const TileGeo *__restrict__ tgeo, const float2 *__restrict__ kc_hl,
                    float2 *__restrict__ G, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int NSG = ta.nst / NPAR;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)ta.nst * ta.slot_bytes);
    // b_full[NSG], done[NSG], a_full[NPAR], a_done[NPAR][NSET], acc_full
    const int nbars = 2 * NSG + NPAR + NPAR * NSET + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + nbars);
    __shared__ __align__(8) uint64_t dbg_bar;    // test hook: never completed
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc05::mbar_init(&dbg_bar, 1);
        for (int i = 0; i < nbars; ++i)
            tc05::mbar_init(&bars[i], (i >= 2 * NSG && i < 2 * NSG + NPAR) ? 4u : 1u);
        tc05::fence_mbar_init();
    }
    if (warp == 0) {
        tc05::tmem_alloc(tmem_slot, ta.tmem_cols);
        tc05::tmem_relinquish();
    }
    if (RW == 12) {
        // 12-row windows: the last two K groups of an operand (zero weights)
        // read 8 rows past its data, into the next column block of the same
        // window (copied with it) or the window slot's 1 KB pad, which no
        // copy writes: zero the pads so that those rows are finite, and order
        // these writes before the products
        const size_t pad0 = (size_t)ta.ncb * ta.cb_bytes;
        for (int i = threadIdx.x; i < ta.nst * 64; i += blockDim.x) {
            uint4 *z = reinterpret_cast<uint4 *>(smem + (size_t)(i >> 6) * ta.slot_bytes + pad0);
            z[i & 63] = make_uint4(0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bp_tc_item_sp<W, SPLIT, NPAR, NSET, RW, PLANAR>(p, ct, ta, &tmap, tgeo, kc_hl, G, err,
                                            (int)blockIdx.x + ta.blk0, smem, bars, tmem, &dbg_bar);
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, ta.tmem_cols);
}

// The batch: ONE persistent launch, one block per SM, over a device work
// queue of every scene's back-projection blocks (scenes in decreasing cost,
// a scene's blocks in their linear order). Per item the block copies the
// scene's descriptors into shared memory, (re-)initialises the barriers and
// runs the item in that scene's layout (K steps and planar or interleaved
// picked at run time; all scenes in the one-block-per-SM layout). Tensor
// memory is allocated once for the block's life. An expired wait anywhere
// stops every block from taking further items.
template <int W, int SPLIT>
__global__ void __launch_bounds__(Warps<3>::threads, 1)
k_backproject_tc_batch(const __grid_constant__ TcBatchMaps maps, CoefTable ct,
                       const TcScene *__restrict__ scenes, int n_scenes, int total,
                       int *counters, int *err) {
    constexpr int kMaxBars = tc_barriers(16, 3);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[kMaxBars];
    __shared__ __align__(8) uint64_t dbg_bar;     // test hook: never completed
    __shared__ uint32_t tmem_slot;
    __shared__ int s_item, s_scene;
    __shared__ int s_begin[kTcBatchMaxScenes];    // the scenes' first items
    __shared__ __align__(16) BpDesc s_bp;
    __shared__ __align__(16) TcArgs s_ta;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n_bars = 0;          // barriers initialised for the last item (thread 0)
    for (int i = threadIdx.x; i < n_scenes; i += blockDim.x) s_begin[i] = scenes[i].begin;
    if (threadIdx.x == 0) tc05::mbar_init(&dbg_bar, 1);
    if (warp == 0) {
        tc05::tmem_alloc(&tmem_slot, 512);
        tc05::tmem_relinquish();
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    for (;;) {
        // the next item and its scene (binary search over the scenes' first
        // items), then warp 0 copies the scene's descriptors
        if (threadIdx.x == 0) {
            int item = total;
            if (*(volatile int *)err == 0) item = atomicAdd(&counters[0], 1);
            int lo = 0, hi = n_scenes - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_begin[mid] <= item) lo = mid; else hi = mid - 1;
            }
            s_item = item;
            s_scene = lo;
        }
        __syncthreads();
        if (warp == 0 && s_item < total) {
            const uint32_t *src_b = reinterpret_cast<const uint32_t *>(&scenes[s_scene].bp);
            const uint32_t *src_t = reinterpret_cast<const uint32_t *>(&scenes[s_scene].ta);
            uint32_t *dst_b = reinterpret_cast<uint32_t *>(&s_bp);
            uint32_t *dst_t = reinterpret_cast<uint32_t *>(&s_ta);
            for (int i = lane; i < (int)(sizeof(BpDesc) / 4); i += 32) dst_b[i] = src_b[i];
            for (int i = lane; i < (int)(sizeof(TcArgs) / 4); i += 32) dst_t[i] = src_t[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_item < total) {
                // the previous item left every barrier with its phases
                // complete and no arrival outstanding
                for (int i = 0; i < n_bars; ++i) tc05::mbar_inval(&bars[i]);
                const int NSG = s_ta.nst / 3;
                for (int i = 0; i < 2 * NSG; ++i) tc05::mbar_init(&bars[i], 1);
                for (int k = 0; k < 3; ++k) {
                    tc05::mbar_init(&bars[2 * NSG + k], 4);
                    tc05::mbar_init(&bars[2 * NSG + 3 + k], 1);
                }
                tc05::mbar_init(&bars[2 * NSG + 6], 1);
                n_bars = tc_barriers(NSG, 3);
                tc05::fence_mbar_init();
            }
        }
        tc05::fence_before_sync();
        __syncthreads();
        tc05::fence_after_sync();
        const int item = s_item;
        if (item >= total) break;
        const TcScene &sd = scenes[s_scene];
        const CUtensorMap *tm = &maps.m[s_scene];
        const int lin = item - sd.begin;
        if (s_ta.sparse) {
            // sparse products (one warp set per class buffer; barriers laid
            // out as for the dense products)
            if (s_ta.planar)
                bp_tc_item_sp<W, SPLIT, 3, 1, 16, true>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl,
                                                        sd.G, err, lin, smem, bars, tmem,
                                                        &dbg_bar);
            else if (s_ta.rw == 32)
                bp_tc_item_sp<W, SPLIT, 3, 1, 32, false>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl,
                                                         sd.G, err, lin, smem, bars, tmem,
                                                         &dbg_bar);
            else if constexpr (SPLIT == 3)
                bp_tc_item_sp<W, SPLIT, 3, 1, 16, false>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl,
                                                         sd.G, err, lin, smem, bars, tmem,
                                                         &dbg_bar);
        } else if (s_ta.ks == 1) {
            if (s_ta.planar)
                bp_tc_item<W, 1, SPLIT, 3, true, 1>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl, sd.G,
                                                    err, lin, smem, bars, tmem, &dbg_bar);
            else
                bp_tc_item<W, 1, SPLIT, 3, false, 1>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl, sd.G,
                                                     err, lin, smem, bars, tmem, &dbg_bar);
        } else {
            if (s_ta.planar)
                bp_tc_item<W, 2, SPLIT, 3, true, 1>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl, sd.G,
                                                    err, lin, smem, bars, tmem, &dbg_bar);
            else
                bp_tc_item<W, 2, SPLIT, 3, false, 1>(s_bp, ct, s_ta, tm, sd.tgeo, sd.kc_hl, sd.G,
                                                     err, lin, smem, bars, tmem, &dbg_bar);
        }
        tc05::fence_before_sync();
        __syncthreads();
        tc05::fence_after_sync();
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, 512);
}

template <int W, int KS, int SPLIT, int NPAR, bool PLANAR, int CPR>
cudaError_t launch_t(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                     const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                     cudaStream_t st) {
    const size_t smem = backproject_tc_smem_bytes(ta);
    cudaError_t e = cudaFuncSetAttribute(k_backproject_tc<W, KS, SPLIT, NPAR, PLANAR, CPR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int total = backproject_tc_blocks(p, ta);
    const int nblk = ta.nblk > 0 ? ta.nblk : total - ta.blk0;
    if (ta.blk0 < 0 || nblk <= 0 || ta.blk0 + nblk > total) return cudaErrorInvalidValue;
    k_backproject_tc<W, KS, SPLIT, NPAR, PLANAR, CPR><<<nblk, Warps<NPAR>::threads, smem, st>>>(
        p, ct, ta, tm, tgeo, kc_hl, G, err);
    return cudaGetLastError();
}

template <int W, int KS, int SPLIT, int NPAR>
cudaError_t launch_pl(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                      const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                      cudaStream_t st) {
    if constexpr (NPAR == 3) {           // two channels per round: one block per SM only
        if (ta.cpr == 2)
            return ta.planar
                       ? launch_t<W, KS, SPLIT, NPAR, true, 2>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                       : launch_t<W, KS, SPLIT, NPAR, false, 2>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
    }
    return ta.planar ? launch_t<W, KS, SPLIT, NPAR, true, 1>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                     : launch_t<W, KS, SPLIT, NPAR, false, 1>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
}

template <int W, int SPLIT, int NPAR, int RW, bool PLANAR = true>
cudaError_t launch_sp(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                      const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                      cudaStream_t st) {
    const size_t smem = backproject_tc_smem_bytes(ta);
    constexpr int NSET = 2;
    cudaError_t e = cudaFuncSetAttribute(k_backproject_tc_sp<W, SPLIT, NPAR, NSET, RW, PLANAR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int total = backproject_tc_blocks(p, ta);
    const int nblk = ta.nblk > 0 ? ta.nblk : total - ta.blk0;
    if (ta.blk0 < 0 || nblk <= 0 || ta.blk0 + nblk > total) return cudaErrorInvalidValue;
    k_backproject_tc_sp<W, SPLIT, NPAR, NSET, RW, PLANAR>
        <<<nblk, SpWarps<NPAR, NSET>::threads, smem, st>>>(p, ct, ta, tm, tgeo, kc_hl, G, err);
    return cudaGetLastError();
}

template <int SPLIT, int NPAR>
cudaError_t launch_spw(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                       const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                       cudaStream_t st) {
    if (ta.rw == 32 && ta.planar) {     // planar layout, 32-row windows (two classes)
        if constexpr (NPAR == 2) {
            switch (p.w) {
                case 4: return launch_sp<4, SPLIT, 2, 32, true>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                case 6: return launch_sp<6, SPLIT, 2, 32, true>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                case 8: return launch_sp<8, SPLIT, 2, 32, true>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                default: return cudaErrorInvalidValue;
            }
        }
        return cudaErrorInvalidValue;
    }
    if (ta.rw == 32) {                  // interleaved layout, 32-row windows
        switch (p.w) {
            case 4: return launch_sp<4, SPLIT, NPAR, 32, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
            case 6: return launch_sp<6, SPLIT, NPAR, 32, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
            case 8: return launch_sp<8, SPLIT, NPAR, 32, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (!ta.planar) {                   // interleaved layout, 16-row windows
        if constexpr (SPLIT == 3) {
            switch (p.w) {
                case 4: return launch_sp<4, 3, NPAR, 16, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                case 6: return launch_sp<6, 3, NPAR, 16, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                case 8: return launch_sp<8, 3, NPAR, 16, false>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
                default: return cudaErrorInvalidValue;
            }
        }
        return cudaErrorInvalidValue;
    }
    if (ta.rw == 12) {                  // 12-row windows: w <= 6
        switch (p.w) {
            case 4: return launch_sp<4, SPLIT, NPAR, 12>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
            case 6: return launch_sp<6, SPLIT, NPAR, 12>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (p.w) {
        case 4: return launch_sp<4, SPLIT, NPAR, 16>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        case 6: return launch_sp<6, SPLIT, NPAR, 16>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        case 8: return launch_sp<8, SPLIT, NPAR, 16>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int KS, int SPLIT, int NPAR>
cudaError_t launch_w(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                     const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                     cudaStream_t st) {
    switch (p.w) {
        case 4: return launch_pl<4, KS, SPLIT, NPAR>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        case 6: return launch_pl<6, KS, SPLIT, NPAR>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        case 8: return launch_pl<8, KS, SPLIT, NPAR>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int KS, int SPLIT>
cudaError_t launch_p(const BpDesc &p, const CoefTable &ct, const TcArgs &ta, const CUtensorMap &tm,
                     const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int *err,
                     cudaStream_t st) {
    if (ta.npar == 3) return launch_w<KS, SPLIT, 3>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
    if (ta.npar == 2) return launch_w<KS, SPLIT, 2>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace

int backproject_tc_blocks(const BpDesc &p, const TcArgs &ta) {
    return (p.nx + TCX - 1) / TCX * ((p.ny + TCY - 1) / TCY) * ta.n_utiles * ta.nsplit;
}

int backproject_tc_tile_x() { return TCX; }
int backproject_tc_tile_y() { return TCY; }

size_t backproject_tc_smem_bytes(const TcArgs &ta) {
    const size_t s = 1024 + (size_t)ta.nst * ta.slot_bytes + (2 * (size_t)ta.nst + 2 * 3 + 1) * 8 + 16;
    // (barriers: 2 per slot group plus the classes' and the accumulator's)
    // at most 2 blocks per SM (256 TMEM columns each), 1 when a block takes 512
    const size_t floor_b = ta.tmem_cols > 256 ? 120 * 1024 : 80 * 1024;
    return s < floor_b ? floor_b : s;
}

size_t backproject_tc_batch_smem_bytes(const TcArgs &ta) {
    return 1024 + (size_t)ta.nst * ta.slot_bytes;     // alignment slack + window slots
}

cudaError_t launch_backproject_tc_batch(const TcBatchMaps &maps, const CoefTable &ct,
                                        const TcScene *scenes, int n_scenes, int total, int split,
                                        int *counters, int *err, int grid, size_t smem,
                                        cudaStream_t st) {
    if (n_scenes < 1 || n_scenes > kTcBatchMaxScenes || grid < 1 || smem > 227 * 1024)
        return cudaErrorInvalidValue;
    auto kern = split == 3 ? k_backproject_tc_batch<6, 3> : k_backproject_tc_batch<6, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Warps<3>::threads, smem, st>>>(maps, ct, scenes, n_scenes, total, counters, err);
    return cudaGetLastError();
}

cudaError_t launch_backproject_tc(const BpDesc &p, const CoefTable &ct, const TcArgs &ta,
                                  const CUtensorMap &tm, const TileGeo *tgeo, const float2 *kc_hl,
                                  float2 *G, int *err, cudaStream_t st) {
    if (ta.sparse) {
        const bool ok = ta.cpr == 1 && ((ta.planar && ta.ks == 1 && ta.rw != 32) ||
                                        (ta.planar && ta.ks == 2 && ta.rw == 32 && ta.npar == 2) ||
                                        (!ta.planar && ta.ks == 2 && ta.rw == 32) ||
                                        (!ta.planar && ta.ks == 1 && ta.rw == 16 &&
                                         ta.split == 3));
        if (!ok) return cudaErrorInvalidValue;
        if (ta.npar == 3)
            return ta.split == 3 ? launch_spw<3, 3>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                                 : launch_spw<1, 3>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        if (ta.npar == 2)
            return ta.split == 3 ? launch_spw<3, 2>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                                 : launch_spw<1, 2>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
        return cudaErrorInvalidValue;
    }
    if (ta.ks == 1)
        return ta.split == 3 ? launch_p<1, 3>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                             : launch_p<1, 1>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
    if (ta.ks == 2)
        return ta.split == 3 ? launch_p<2, 3>(p, ct, ta, tm, tgeo, kc_hl, G, err, st)
                             : launch_p<2, 1>(p, ct, ta, tm, tgeo, kc_hl, G, err, st);
    return cudaErrorInvalidValue;
}
