// Back-projection (step 8b / 19b) with the interpolation on the tensor cores.
//
// Same sum as backproject.cu,
//   G_u(x,y) = sum_c e^{j (kappa_c,u delta + phi_c,u)} sum_t phi(a_c - l_{i0+t}) b_c[i0+t][u],
// but for each channel the w-tap interpolation of a warp's 16 pixels is a
// small dense product
//   X[p][col] = sum_{k < 16} A[p][k] B[k][col],   col = 2u + (re, im),
// with A[p][k] the ES weight of pixel p at window row base + k (zero outside
// its w taps) and B the table rows base .. base+15. Both operands are split
// into BF16 hi + lo parts and the product is hi.hi + hi.lo + lo.hi on
// mma.sync m16n8k16 with FP32 accumulation (relative error ~1e-5, below the
// NUFFT's). The FP32 pipe keeps only the carrier sin/cos and the complex
// multiply-accumulate.
//
// Block = 16 x 8 pixels (8 warps, each a 4 x 4 pixel block) x 4 NJ k_z bins.
// Thread (g, t) of a warp owns pixels g and g + 8 of its block and bins
// u = 4 j + t, j < NJ, exactly the rows and columns of its mma accumulator
// fragments, so products feed the carrier without data movement.
//
// The table comes in a tensor-core layout written by the range-table kernel:
// [channel][plane hi/lo][column][row] BF16, rows contiguous. A chunk of CCH
// channels' windows (S rows from the channel's first row rounded down to 8)
// is copied into shared memory with cp.async, double buffered.
#include <cuda_bf16.h>

#include "bp_body.cuh"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TCX = 16, TCY = 8;
constexpr int APAD = 24;          // A staging row stride (bf16), conflict-free fragment loads

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ldp(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const unsigned *>(p);
}

template <int NJ, int CCH>
struct TcSmem {
    static constexpr int NCOL = 8 * NJ;   // 2 columns (re, im) per bin, 4 NJ bins
    static size_t bytes(int S, int n_chan) {
        return (size_t)2 * CCH * 2 * NCOL * S * sizeof(__nv_bfloat16) +   // windows, 2 buffers
               (size_t)2 * CCH * sizeof(TileGeo) +                       // geometry
               (size_t)CCH * 4 * NJ * sizeof(float2) +                    // (kappa, phi)
               (size_t)8 * 2 * 16 * APAD * sizeof(__nv_bfloat16) +         // A staging per warp
               (size_t)8 * 16 * sizeof(float) +                           // delta per warp pixel
               (size_t)n_chan * sizeof(int);                              // first rows
    }
};

template <int W, int NJ, int CCH>
__global__ void __launch_bounds__(256, 2)
k_backproject_tc(BpDesc p, CoefTable ct, const __nv_bfloat16 *__restrict__ table,
                 const TileGeo *__restrict__ tgeo, const float2 *__restrict__ kc_hl,
                 float2 *__restrict__ G, int S, int tc_rows, int tc_cols) {
    constexpr int NCOL = 8 * NJ;
    constexpr int UT = 4 * NJ;
    constexpr int ND = W + 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *win = reinterpret_cast<__nv_bfloat16 *>(smem);      // [2][CCH][2][NCOL][S]
    TileGeo *geo = reinterpret_cast<TileGeo *>(win + (size_t)2 * CCH * 2 * NCOL * S);
    float2 *kphi = reinterpret_cast<float2 *>(geo + 2 * CCH);          // [CCH][UT]
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(kphi + CCH * UT);   // [8][2][16][APAD]
    float *dls = reinterpret_cast<float *>(As + 8 * 2 * 16 * APAD);    // [8][16]
    int *ilo8 = reinterpret_cast<int *>(dls + 8 * 16);                 // [n_chan]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wx = warp & 3, wy = warp >> 2;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int u0 = blockIdx.z * UT;
    const TileGeo *tg = tgeo + (size_t)tile * p.n_chan;
    // the pixel this lane prepares (lanes 16-31 repeat lanes 0-15)
    const int pp = lane & 15;
    const float ddx = ((float)(wx * 4 + (pp & 3)) - 0.5f * (TCX - 1)) * p.dxf;
    const float ddy = ((float)(wy * 4 + (pp >> 2)) - 0.5f * (TCY - 1)) * p.dyf;
    __nv_bfloat16 *Aw = As + warp * 2 * 16 * APAD;

    for (int c = threadIdx.x; c < p.n_chan; c += blockDim.x) ilo8[c] = tg[c].ilo & ~7;
    __syncthreads();

    auto issue = [&](int ck, int buf) {
        const int c0 = ck * CCH;
        const int ncc = min(CCH, p.n_chan - c0);
        const int cpc = S / 8;                             // 16-byte chunks per column
        const int per_c = 2 * NCOL * cpc;
        for (int idx = threadIdx.x; idx < ncc * per_c; idx += blockDim.x) {
            const int cl = idx / per_c;
            int rem = idx - cl * per_c;
            const int plane = rem / (NCOL * cpc);
            rem -= plane * NCOL * cpc;
            const int col = rem / cpc;
            const int ch = rem - col * cpc;
            const __nv_bfloat16 *src =
                table + (((size_t)(c0 + cl) * 2 + plane) * tc_cols + 2 * u0 + col) * tc_rows +
                ilo8[c0 + cl] + 8 * ch;
            __nv_bfloat16 *dst = win + ((((size_t)buf * CCH + cl) * 2 + plane) * NCOL + col) * S +
                                 8 * ch;
            bp::cp_async16(dst, src);
        }
        constexpr int G4 = sizeof(TileGeo) / 16;
        for (int idx = threadIdx.x; idx < ncc * G4; idx += blockDim.x)
            bp::cp_async16(reinterpret_cast<float4 *>(geo + buf * CCH) + idx,
                           reinterpret_cast<const float4 *>(tg + c0) + idx);
        bp::cp_commit();
    };

    float2 acc[NJ][2];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);

    const int n_chunks = (p.n_chan + CCH - 1) / CCH;
    issue(0, 0);
    for (int ck = 0; ck < n_chunks; ++ck) {
        const int buf = ck & 1;
        const int ncc = min(CCH, p.n_chan - ck * CCH);
        if (ck + 1 < n_chunks) {
            issue(ck + 1, buf ^ 1);
            bp::cp_wait<1>();
        } else {
            bp::cp_wait<0>();
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < ncc * UT; idx += blockDim.x) {
            const int cl = idx / UT;
            const int u = u0 + (idx - cl * UT);
            const TileGeo &gg = geo[buf * CCH + cl];
            const float2 k = u < p.n_pad ? kc_hl[u] : make_float2(0.f, 0.f);
            kphi[idx] = make_float2(k.x, bp::phase_ff(k.x, k.y, gg.a_hi, gg.a_lo));
        }
        __syncthreads();

        for (int cl = 0; cl < ncc; ++cl) {
            const TileGeo gc = geo[buf * CCH + cl];
            // geometry of pixel pp: delta = a - a* without cancellation
            float ex = gc.dxt + ddx, ey = gc.dyt + ddy;
            float num = fmaf(ddx, 2.0f * gc.dxt + ddx, ddy * (2.0f * gc.dyt + ddy));
            float r2 = fmaf(ex, ex, ey * ey);
            float delta = num * __frcp_rn(fmaf(r2, rsqrtf(r2), gc.rt));
            if (p.mode == 1) {
                ex = gc.dxr + ddx; ey = gc.dyr + ddy;
                num = fmaf(ddx, 2.0f * gc.dxr + ddx, ddy * (2.0f * gc.dyr + ddy));
                r2 = fmaf(ex, ex, ey * ey);
                delta += num * __frcp_rn(fmaf(r2, rsqrtf(r2), gc.rr));
            }
            // position in window rows (row 0 = the channel's first row rounded to 8)
            const float pos = (delta + gc.off) * p.inv_h + (float)(gc.ilo & 7);
            const int i0 = (int)ceilf(pos - 0.5f * W);
            int base = __reduce_min_sync(0xffffffffu, i0) & ~1;
            base = max(0, min(base, S - 16));
            const int o = min(max(i0 - base, 0), 16 - W);
            const float s = fmaf(2.0f, pos - (float)(base + o), -(float)(W - 1));
            // A operand: zero this warp's 16 x 16 (x2 planes), then the w taps
            {
                uint4 *z = reinterpret_cast<uint4 *>(Aw);
                const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
                for (int k = lane; k < 2 * 16 * APAD / 8; k += 32) z[k] = zero;
            }
            __syncwarp();
#pragma unroll
            for (int tap = 0; tap < W; ++tap) {
                float wv = ct.c[tap][ND - 1];
#pragma unroll
                for (int d = ND - 2; d >= 0; --d) wv = fmaf(wv, s, ct.c[tap][d]);
                if ((tap < W / 2) == (lane < 16)) {
                    const __nv_bfloat16 hi = __float2bfloat16(wv);
                    Aw[pp * APAD + o + tap] = hi;
                    Aw[16 * APAD + pp * APAD + o + tap] = __float2bfloat16(wv - __bfloat162float(hi));
                }
            }
            if (lane < 16) dls[warp * 16 + pp] = delta;
            __syncwarp();
            unsigned ah[4], al[4];
            ah[0] = ldp(Aw + g * APAD + 2 * t);
            ah[1] = ldp(Aw + (g + 8) * APAD + 2 * t);
            ah[2] = ldp(Aw + g * APAD + 2 * t + 8);
            ah[3] = ldp(Aw + (g + 8) * APAD + 2 * t + 8);
            al[0] = ldp(Aw + 16 * APAD + g * APAD + 2 * t);
            al[1] = ldp(Aw + 16 * APAD + (g + 8) * APAD + 2 * t);
            al[2] = ldp(Aw + 16 * APAD + g * APAD + 2 * t + 8);
            al[3] = ldp(Aw + 16 * APAD + (g + 8) * APAD + 2 * t + 8);
            const float d0 = dls[warp * 16 + g], d1 = dls[warp * 16 + g + 8];
            const __nv_bfloat16 *wh = win + ((size_t)(buf * CCH + cl) * 2 + 0) * NCOL * S + base + 2 * t;
            const __nv_bfloat16 *wl = wh + NCOL * S;
            const float2 *kp = kphi + cl * UT;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int col = 8 * j + g;
                unsigned bh[2], bl[2];
                bh[0] = ldp(wh + col * S);
                bh[1] = ldp(wh + col * S + 8);
                bl[0] = ldp(wl + col * S);
                bl[1] = ldp(wl + col * S + 8);
                float x[4] = {0.f, 0.f, 0.f, 0.f};
                mma16816(x, ah, bh);
                mma16816(x, ah, bl);
                mma16816(x, al, bh);
                // x: (pixel g: re, im), (pixel g+8: re, im) of bin 4j + t
                const float2 k = kp[4 * j + t];
                float s0, c0, s1, c1;
                __sincosf(fmaf(k.x, d0, k.y), &s0, &c0);
                __sincosf(fmaf(k.x, d1, k.y), &s1, &c1);
                acc[j][0].x = fmaf(x[0], c0, fmaf(-x[1], s0, acc[j][0].x));
                acc[j][0].y = fmaf(x[0], s0, fmaf(x[1], c0, acc[j][0].y));
                acc[j][1].x = fmaf(x[2], c1, fmaf(-x[3], s1, acc[j][1].x));
                acc[j][1].y = fmaf(x[2], s1, fmaf(x[3], c1, acc[j][1].y));
            }
            __syncwarp();
        }
        __syncthreads();
    }

    const size_t plane_sz = (size_t)p.nx * p.ny;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int u = u0 + 4 * j + t;
        if (u >= p.n_pad) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int pl = g + 8 * h;
            const int ix = blockIdx.x * TCX + wx * 4 + (pl & 3);
            const int iy = blockIdx.y * TCY + wy * 4 + (pl >> 2);
            if (ix < p.nx && iy < p.ny) G[u * plane_sz + (size_t)iy * p.nx + ix] = acc[j][h];
        }
    }
}

template <int W, int NJ, int CCH>
cudaError_t launch_tc_t(const BpDesc &p, const CoefTable &ct, const void *table,
                        const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int S, int tc_rows,
                        int tc_cols, cudaStream_t st) {
    const size_t smem = TcSmem<NJ, CCH>::bytes(S, p.n_chan);
    cudaError_t e = cudaFuncSetAttribute(k_backproject_tc<W, NJ, CCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + TCX - 1) / TCX, (p.ny + TCY - 1) / TCY, (p.n_pad + 4 * NJ - 1) / (4 * NJ));
    k_backproject_tc<W, NJ, CCH><<<grid, 256, smem, st>>>(
        p, ct, (const __nv_bfloat16 *)table, tgeo, kc_hl, G, S, tc_rows, tc_cols);
    return cudaGetLastError();
}

template <int NJ, int CCH>
cudaError_t launch_tc_w(const BpDesc &p, const CoefTable &ct, const void *table,
                        const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int S, int tc_rows,
                        int tc_cols, cudaStream_t st) {
    switch (p.w) {
        case 4: return launch_tc_t<4, NJ, CCH>(p, ct, table, tgeo, kc_hl, G, S, tc_rows, tc_cols, st);
        case 6: return launch_tc_t<6, NJ, CCH>(p, ct, table, tgeo, kc_hl, G, S, tc_rows, tc_cols, st);
        case 8: return launch_tc_t<8, NJ, CCH>(p, ct, table, tgeo, kc_hl, G, S, tc_rows, tc_cols, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int backproject_tc_tile_x() { return TCX; }
int backproject_tc_tile_y() { return TCY; }

// Window rows staged per channel: at least R + 18 (even base + 16-row window
// + the 0-7 rows of rounding the first row down to 8), = 8 mod 16 so that
// fragment loads are free of bank conflicts.
int backproject_tc_window_rows(int R) {
    int s = R + 18;
    s = (s + 7) / 8 * 8;
    if ((s / 8) % 2 == 0) s += 8;
    return s;
}

size_t backproject_tc_smem_bytes(int S, int tile_u, int n_chan) {
    if (tile_u == 40) return TcSmem<10, 3>::bytes(S, n_chan);
    return TcSmem<8, 4>::bytes(S, n_chan);
}

cudaError_t launch_backproject_tc(const BpDesc &p, const CoefTable &ct, const void *table,
                                  const TileGeo *tgeo, const float2 *kc_hl, float2 *G, int S,
                                  int tc_rows, int tc_cols, cudaStream_t st) {
    if (p.tile_u == 40)
        return launch_tc_w<10, 3>(p, ct, table, tgeo, kc_hl, G, S, tc_rows, tc_cols, st);
    return launch_tc_w<8, 4>(p, ct, table, tgeo, kc_hl, G, S, tc_rows, tc_cols, st);
}
