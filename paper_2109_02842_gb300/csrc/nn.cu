// Learned fast path: kernels of a 3-D convolutional encoder-decoder that maps
// features of a cheap reconstruction to the full one (the network is
// described in paper_2109_02842_gb300/learned.py; the paper has no learned
// component).
//
// Volumes are channels-last: x[v][c] with v = (z H + y) W + x. Convolutions
// are 3 x 3 x 3, stride 1, 'same' zero padding; weights w[co][k] with
// k = tap Cin + ci, tap = (dz 3 + dy) 3 + dx reading x[z+dz-1][y+dy-1][x+dx-1],
// rows padded with zeros to a multiple of 16.
//
// The convolution is an implicit GEMM on the tensor cores: out[v][co] =
// sum_k A[v][k] B[k][co] with A the (never materialised) im2col matrix and B
// the weights. The shapes the network runs at full size (Cin a multiple of
// 16, Cout 16..128, rows of 16..128 voxels) take the tcgen05 kernel of
// nn_tc.cu; the others (the 3-channel input layer, the 2-channel head, small
// or odd test volumes) the kernel below, BF16 mma.sync m16n8k16 with FP32
// accumulation. A block of 4
// warps owns 64 voxels x (8 NT) output channels; per 16-wide K chunk it
// stages the A tile (one 32-byte row per voxel when Cin is a multiple of 16,
// an element gather otherwise) and the B tile in shared memory.
// The backward pass reuses the forward kernel for the input gradient (the
// transposed convolution is a convolution with flipped taps and swapped
// channel roles) and has its own GEMM for the weight gradient, reducing over
// voxels in chunks: each chunk writes its partial dW, and a second kernel sums
// the partials in chunk order, so gradients are bitwise reproducible.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kRowPad = 24;   // bf16 per staged row: 16 + 8 (conflict-free fragment loads)

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4],
                                               const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const unsigned *>(p);
}

struct Vol {
    int D, H, W;
    __device__ __forceinline__ bool neighbour(int v, int tap, int &nv) const {
        const int x = v % W;
        const int y = (v / W) % H;
        const int z = v / (W * H);
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int zz = z + dz, yy = y + dy, xx = x + dx;
        if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) return false;
        nv = (zz * H + yy) * W + xx;
        return true;
    }
};

// out[v][co] = act(bias[co] + sum_k x~[v][k] w[co][k])
template <int NT, bool OUT_BF16>
__global__ void __launch_bounds__(128)
k_conv3d(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ w,
         const float *__restrict__ bias, void *__restrict__ out, Vol vol, int Cin, int Cout,
         int Kp, int relu) {
    constexpr int NTILE = 8 * NT;
    __shared__ __align__(16) __nv_bfloat16 As[64][kRowPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[NTILE][kRowPad];
    const int V = vol.D * vol.H * vol.W;
    const int v0 = blockIdx.x * 64;
    const int n0 = blockIdx.y * NTILE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int K = 27 * Cin;
    const bool vec = (Cin % 16) == 0;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    for (int k0 = 0; k0 < Kp; k0 += 16) {
        // A tile: 64 voxels x 16 k
        if (vec) {
            const int row = threadIdx.x >> 1, half = threadIdx.x & 1;
            const int tap = k0 / Cin, ci0 = k0 - tap * Cin;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            int nv;
            if (v0 + row < V && k0 < K && vol.neighbour(v0 + row, tap, nv))
                val = *reinterpret_cast<const uint4 *>(x + (size_t)nv * Cin + ci0 + 8 * half);
            *reinterpret_cast<uint4 *>(&As[row][8 * half]) = val;
        } else {
            for (int e = threadIdx.x; e < 64 * 16; e += 128) {
                const int row = e >> 4, kk = e & 15;
                const int k = k0 + kk;
                __nv_bfloat16 val = __float2bfloat16(0.f);
                int nv;
                if (v0 + row < V && k < K) {
                    const int tap = k / Cin, ci = k - tap * Cin;
                    if (vol.neighbour(v0 + row, tap, nv)) val = x[(size_t)nv * Cin + ci];
                }
                As[row][kk] = val;
            }
        }
        // B tile: NTILE output channels x 16 k (k contiguous per channel)
        for (int e = threadIdx.x; e < NTILE * 2; e += 128) {
            const int n = e >> 1, half = e & 1;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (n0 + n < Cout)
                val = *reinterpret_cast<const uint4 *>(w + (size_t)(n0 + n) * Kp + k0 + 8 * half);
            *reinterpret_cast<uint4 *>(&Bs[n][8 * half]) = val;
        }
        __syncthreads();
        unsigned a[4];
        const int r0 = warp * 16;
        a[0] = ld_pair(&As[r0 + g][2 * t]);
        a[1] = ld_pair(&As[r0 + g + 8][2 * t]);
        a[2] = ld_pair(&As[r0 + g][2 * t + 8]);
        a[3] = ld_pair(&As[r0 + g + 8][2 * t + 8]);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            unsigned b[2];
            b[0] = ld_pair(&Bs[j * 8 + g][2 * t]);
            b[1] = ld_pair(&Bs[j * 8 + g][2 * t + 8]);
            mma_bf16_16816(acc[j], a, b);
        }
        __syncthreads();
    }
    // epilogue: rows g, g+8 of this warp's 16 voxels; columns 2t, 2t+1 of each n-tile
#pragma unroll
    for (int j = 0; j < NT; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = v0 + warp * 16 + g + 8 * h;
            if (v >= V) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int co = n0 + j * 8 + 2 * t + q;
                if (co >= Cout) continue;
                float r = acc[j][2 * h + q] + (bias ? bias[co] : 0.f);
                if (relu) r = fmaxf(r, 0.f);
                if (OUT_BF16)
                    reinterpret_cast<__nv_bfloat16 *>(out)[(size_t)v * Cout + co] = __float2bfloat16(r);
                else
                    reinterpret_cast<float *>(out)[(size_t)v * Cout + co] = r;
            }
        }
    }
}

// gw[co][k] += sum_v gy[v][co] x~[v][k]  (k < 27 Cin), over a chunk of voxels.
// Block: 4 warps, 32 k-columns (8 per warp), all Cout (MT m-tiles of 16).
template <int MT>
__global__ void __launch_bounds__(128)
k_conv3d_wgrad(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ gy,
               float *__restrict__ part, Vol vol, int Cin, int Cout, int Kp, int chunk) {
    __shared__ __align__(16) __nv_bfloat16 As[16 * MT][kRowPad];   // [co][16 voxels]
    __shared__ __align__(16) __nv_bfloat16 Bs[32][kRowPad];        // [k col][16 voxels]
    const int V = vol.D * vol.H * vol.W;
    const int K = 27 * Cin;
    const int kc0 = blockIdx.x * 32;
    const int vbeg = blockIdx.y * chunk;
    const int vend = min(V, vbeg + chunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float acc[MT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int vs = vbeg; vs < vend; vs += 16) {
        for (int e = threadIdx.x; e < 16 * 16 * MT; e += 128) {
            const int vv = e / (16 * MT), co = e - vv * (16 * MT);
            const int v = vs + vv;
            As[co][vv] = (v < vend && co < Cout) ? gy[(size_t)v * Cout + co] : __float2bfloat16(0.f);
        }
        for (int e = threadIdx.x; e < 32 * 16; e += 128) {
            const int kc = e >> 4, vv = e & 15;
            const int k = kc0 + kc, v = vs + vv;
            __nv_bfloat16 val = __float2bfloat16(0.f);
            int nv;
            if (v < vend && k < K) {
                const int tap = k / Cin, ci = k - tap * Cin;
                if (vol.neighbour(v, tap, nv)) val = x[(size_t)nv * Cin + ci];
            }
            Bs[kc][vv] = val;
        }
        __syncthreads();
        unsigned b[2];
        b[0] = ld_pair(&Bs[warp * 8 + g][2 * t]);
        b[1] = ld_pair(&Bs[warp * 8 + g][2 * t + 8]);
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            unsigned a[4];
            a[0] = ld_pair(&As[i * 16 + g][2 * t]);
            a[1] = ld_pair(&As[i * 16 + g + 8][2 * t]);
            a[2] = ld_pair(&As[i * 16 + g][2 * t + 8]);
            a[3] = ld_pair(&As[i * 16 + g + 8][2 * t + 8]);
            mma_bf16_16816(acc[i], a, b);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int co = i * 16 + g + 8 * h;
                const int k = kc0 + warp * 8 + 2 * t + q;
                if (co < Cout && k < K)
                    part[((size_t)blockIdx.y * Cout + co) * Kp + k] = acc[i][2 * h + q];
            }
}

// gw[i] += sum_c part[c][i] in chunk order (deterministic)
__global__ void k_sum_parts(const float *__restrict__ part, float *__restrict__ gw, int nparts,
                            size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * n + i];
    gw[i] += s;
}

// part[chunk][co] = sum over the chunk's voxels of gy[v][co]
__global__ void k_bias_grad(const __nv_bfloat16 *__restrict__ gy, float *__restrict__ part, int V,
                            int C, int chunk) {
    const int co = threadIdx.x;
    if (co >= C) return;
    const int v0 = blockIdx.x * chunk, v1 = min(V, v0 + chunk);
    float s = 0.f;
    for (int v = v0; v < v1; ++v) s += __bfloat162float(gy[(size_t)v * C + co]);
    part[(size_t)blockIdx.x * C + co] = s;
}

// wt[ci][tap' Cout + co] = w[co][tap Cin + ci], tap' = 26 - tap
__global__ void k_weight_flip(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt,
                              int Cin, int Cout, int Kp, int Kpt) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Cin * Kpt) return;
    const int ci = idx / Kpt, k = idx - ci * Kpt;
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (k < 27 * Cout) {
        const int tp = k / Cout, co = k - tp * Cout;
        v = w[(size_t)co * Kp + (26 - tp) * Cin + ci];
    }
    wt[idx] = v;
}

// out (bf16) = g (f32) where y > 0, else 0
__global__ void k_relu_bwd(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ y,
                           __nv_bfloat16 *__restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(__bfloat162float(y[i]) > 0.f ? g[i] : 0.f);
}

__global__ void k_cast_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(a[i]);
}

__global__ void k_add_bf16(const __nv_bfloat16 *__restrict__ a, const __nv_bfloat16 *__restrict__ b,
                           __nv_bfloat16 *__restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void k_accum_f32(const float *__restrict__ a, float *__restrict__ acc, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] += a[i];
}

// y[Z][Y][X][c] = mean of the 2x2x2 block of x (D, H, W even)
__global__ void k_avgpool2(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y,
                           int D, int H, int W, int C) {
    const size_t n = (size_t)(D / 2) * (H / 2) * (W / 2) * C;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const size_t o = i / C;
    const int X = (int)(o % (W / 2)), Y = (int)((o / (W / 2)) % (H / 2)), Z = (int)(o / ((W / 2) * (H / 2)));
    float s = 0.f;
    for (int d = 0; d < 8; ++d) {
        const int z = 2 * Z + (d >> 2), yy = 2 * Y + ((d >> 1) & 1), xx = 2 * X + (d & 1);
        s += __bfloat162float(x[(((size_t)z * H + yy) * W + xx) * C + c]);
    }
    y[i] = __float2bfloat16(0.125f * s);
}

// gx[v] += gy[parent(v)] / 8
__global__ void k_avgpool2_bwd(const float *__restrict__ gy, float *__restrict__ gx, int D, int H,
                               int W, int C) {
    const size_t n = (size_t)D * H * W * C;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const size_t v = i / C;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((size_t)W * H));
    gx[i] += 0.125f * gy[(((size_t)(z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
}

// y (2D x 2H x 2W) = nearest x
__global__ void k_upsample2(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y,
                            int D, int H, int W, int C) {
    const size_t n = (size_t)8 * D * H * W * C;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const size_t v = i / C;
    const int W2 = 2 * W, H2 = 2 * H;
    const int xx = (int)(v % W2), yy = (int)((v / W2) % H2), zz = (int)(v / ((size_t)W2 * H2));
    y[i] = x[(((size_t)(zz / 2) * H + yy / 2) * W + xx / 2) * C + c];
}

// the same with 8 channels (16 bytes) per thread, for C a multiple of 8
__global__ void k_upsample2_v8(const uint4 *__restrict__ x, uint4 *__restrict__ y, int D, int H,
                               int W, int C8) {
    const size_t n = (size_t)8 * D * H * W * C8;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C8);
    const size_t v = i / C8;
    const int W2 = 2 * W, H2 = 2 * H;
    const int xx = (int)(v % W2), yy = (int)((v / W2) % H2), zz = (int)(v / ((size_t)W2 * H2));
    y[i] = x[(((size_t)(zz / 2) * H + yy / 2) * W + xx / 2) * C8 + c];
}

// gx[Z][Y][X] = sum of gy over the 8 children (gx has the small size D x H x W)
__global__ void k_upsample2_bwd(const float *__restrict__ gy, float *__restrict__ gx, int D, int H,
                                int W, int C) {
    const size_t n = (size_t)D * H * W * C;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const size_t o = i / C;
    const int X = (int)(o % W), Y = (int)((o / W) % H), Z = (int)(o / ((size_t)W * H));
    float s = 0.f;
    for (int d = 0; d < 8; ++d) {
        const int z = 2 * Z + (d >> 2), y = 2 * Y + ((d >> 1) & 1), x = 2 * X + (d & 1);
        s += gy[(((size_t)z * 2 * H + y) * 2 * W + x) * C + c];
    }
    gx[i] = s;
}

// *mx = max |img| (non-negative floats compare as integers)
__global__ void k_absmax(const float2 *__restrict__ img, size_t n, float *mx) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, hypotf(img[i].x, img[i].y));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(mx), __float_as_int(m));
}

// feat[v] = (Re g / s, Im g / s, |g| / s) as bf16 [v][3]
__global__ void k_features(const float2 *__restrict__ img, const float *__restrict__ scale,
                           __nv_bfloat16 *__restrict__ feat, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 z = img[i];
    const float a = hypotf(z.x, z.y);
    const float s = *scale > 0.f ? *scale : 1.f;
    feat[3 * i + 0] = __float2bfloat16(z.x / s);
    feat[3 * i + 1] = __float2bfloat16(z.y / s);
    feat[3 * i + 2] = __float2bfloat16(a / s);
}

// sums[0] = sum |target/s|^2, sums[1] = sum |pred - target/s|^2; one block of
// 1024 threads with a fixed-order tree, so the result is reproducible
__global__ void __launch_bounds__(1024)
k_loss_sums(const float *__restrict__ pred, const float2 *__restrict__ tgt,
            const float *__restrict__ scale, size_t n, float *sums) {
    __shared__ float st_s[1024], sd_s[1024];
    const float inv = 1.0f / (*scale > 0.f ? *scale : 1.f);
    float st = 0.f, sd = 0.f;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float tx = tgt[i].x * inv, ty = tgt[i].y * inv;
        const float dx = pred[2 * i] - tx, dy = pred[2 * i + 1] - ty;
        st += tx * tx + ty * ty;
        sd += dx * dx + dy * dy;
    }
    st_s[threadIdx.x] = st;
    sd_s[threadIdx.x] = sd;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            st_s[threadIdx.x] += st_s[threadIdx.x + o];
            sd_s[threadIdx.x] += sd_s[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = st_s[0];
        sums[1] = sd_s[0];
    }
}

// Acceptance check of a learned correction: out[0] = number of non-finite
// entries of corr ([n][2]), out[1] = sum of corr^2 over the finite ones,
// out[2] = sum |gain img / s|^2 (the scaled cheap image the correction is
// added to). Two passes with fixed orders (reproducible sums): 256 blocks of
// 256 threads write partial sums (block b takes the entries b, b + 256, ...
// in tree order), one block adds the partials in block order.
constexpr int kCheckBlocks = 256;
// the partial sums: a file-scope device array (the check allocates nothing;
// two checks running at the same time on different streams would race on it)
__device__ float g_check_part[3 * kCheckBlocks];
__global__ void __launch_bounds__(256)
k_check_part(const float *__restrict__ corr, const float2 *__restrict__ img,
             const float *__restrict__ scale, float gain, size_t n, float *part) {
    __shared__ float s_bad[256], s_c[256], s_i[256];
    const float k = gain / (*scale > 0.f ? *scale : 1.f);
    float bad = 0.f, sc = 0.f, si = 0.f;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)kCheckBlocks * 256) {
        const float a = corr[2 * i], b = corr[2 * i + 1];
        if (isfinite(a)) sc += a * a; else bad += 1.f;
        if (isfinite(b)) sc += b * b; else bad += 1.f;
        const float x = k * img[i].x, y = k * img[i].y;
        si += x * x + y * y;
    }
    s_bad[threadIdx.x] = bad;
    s_c[threadIdx.x] = sc;
    s_i[threadIdx.x] = si;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_bad[threadIdx.x] += s_bad[threadIdx.x + o];
            s_c[threadIdx.x] += s_c[threadIdx.x + o];
            s_i[threadIdx.x] += s_i[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s_bad[0];
        part[3 * blockIdx.x + 1] = s_c[0];
        part[3 * blockIdx.x + 2] = s_i[0];
    }
}

__global__ void __launch_bounds__(256) k_check_sum(const float *__restrict__ part, float *out) {
    __shared__ float s[3][kCheckBlocks];
    for (int q = 0; q < 3; ++q) s[q][threadIdx.x] = part[3 * threadIdx.x + q];
    __syncthreads();
    for (int o = kCheckBlocks / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = s[threadIdx.x][0];
}

// grad = 2 (pred - target/s) / sum|target/s|^2
__global__ void k_loss_grad(const float *__restrict__ pred, const float2 *__restrict__ tgt,
                            const float *__restrict__ scale, const float *__restrict__ sums,
                            float *__restrict__ grad, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float inv = 1.0f / (*scale > 0.f ? *scale : 1.f);
    const float k = 2.0f / fmaxf(sums[0], 1e-30f);
    grad[2 * i] = k * (pred[2 * i] - tgt[i].x * inv);
    grad[2 * i + 1] = k * (pred[2 * i + 1] - tgt[i].y * inv);
}

// pred[v] += gain (Re, Im) of img[v] / s
__global__ void k_residual(float *__restrict__ pred, const float2 *__restrict__ img,
                           const float *__restrict__ scale, float gain, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float k = gain / (*scale > 0.f ? *scale : 1.f);
    pred[2 * i] += k * img[i].x;
    pred[2 * i + 1] += k * img[i].y;
}

// img = s (pred.x + j pred.y)
__global__ void k_to_complex(const float *__restrict__ pred, const float *__restrict__ scale,
                             float2 *__restrict__ img, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = *scale > 0.f ? *scale : 1.f;
    img[i] = make_float2(s * pred[2 * i], s * pred[2 * i + 1]);
}

// Adam (Kingma & Ba 2015), bias-corrected; refreshes the BF16 copy.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, size_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
}

inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// launch wrappers (declared in kernels.h)
// ---------------------------------------------------------------------------
cudaError_t nn_conv3d(const void *x, const void *w, const float *bias, void *out, int D, int H,
                      int W, int Cin, int Cout, int Kp, int relu, int out_bf16, cudaStream_t st) {
    // the shapes the network runs at full size go to the tcgen05 kernel
    if (nn_conv3d_tc_supported(D, H, W, Cin, Cout, x, w, out))
        return nn_conv3d_tc(x, w, bias, out, D, H, W, Cin, Cout, Kp, relu, out_bf16, st);
    const int V = D * H * W;
    Vol vol{D, H, W};
    const auto *xb = (const __nv_bfloat16 *)x;
    const auto *wb = (const __nv_bfloat16 *)w;
    if (Cout <= 8) {
        dim3 grid((V + 63) / 64, (Cout + 7) / 8);
        if (out_bf16) k_conv3d<1, true><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
        else k_conv3d<1, false><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
    } else if (Cout <= 16) {
        dim3 grid((V + 63) / 64, (Cout + 15) / 16);
        if (out_bf16) k_conv3d<2, true><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
        else k_conv3d<2, false><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
    } else {
        dim3 grid((V + 63) / 64, (Cout + 31) / 32);
        if (out_bf16) k_conv3d<4, true><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
        else k_conv3d<4, false><<<grid, 128, 0, st>>>(xb, wb, bias, out, vol, Cin, Cout, Kp, relu);
    }
    return cudaGetLastError();
}

size_t nn_wgrad_work_floats(int D, int H, int W, int Cin, int Cout, int Kp) {
    const int V = D * H * W;
    const size_t chunks = (size_t)(V + 2047) / 2048;
    const size_t bchunks = (size_t)(V + 4095) / 4096;
    return chunks * Cout * Kp + bchunks * Cout;
}

cudaError_t nn_conv3d_wgrad(const void *x, const void *gy, float *gw, float *gb, float *work,
                            int D, int H, int W, int Cin, int Cout, int Kp, cudaStream_t st) {
    const int V = D * H * W;
    Vol vol{D, H, W};
    const int chunk = 2048;
    const int nch = (V + chunk - 1) / chunk;
    dim3 grid((27 * Cin + 31) / 32, nch);
    const auto *xb = (const __nv_bfloat16 *)x;
    const auto *gyb = (const __nv_bfloat16 *)gy;
    const int mt = (Cout + 15) / 16;
    // partials [chunk][Cout][Kp]; columns k >= 27 Cin stay zero
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(float) * (size_t)nch * Cout * Kp, st);
    if (e != cudaSuccess) return e;
    switch (mt) {
        case 1: k_conv3d_wgrad<1><<<grid, 128, 0, st>>>(xb, gyb, work, vol, Cin, Cout, Kp, chunk); break;
        case 2: k_conv3d_wgrad<2><<<grid, 128, 0, st>>>(xb, gyb, work, vol, Cin, Cout, Kp, chunk); break;
        case 4: k_conv3d_wgrad<4><<<grid, 128, 0, st>>>(xb, gyb, work, vol, Cin, Cout, Kp, chunk); break;
        case 8: k_conv3d_wgrad<8><<<grid, 128, 0, st>>>(xb, gyb, work, vol, Cin, Cout, Kp, chunk); break;
        default: return cudaErrorInvalidValue;
    }
    const size_t nw = (size_t)Cout * Kp;
    k_sum_parts<<<nblk(nw), 256, 0, st>>>(work, gw, nch, nw);
    if (gb) {
        const int bchunk = 4096;
        const int nb = (V + bchunk - 1) / bchunk;
        float *bpart = work + (size_t)nch * Cout * Kp;
        k_bias_grad<<<nb, ((Cout + 31) / 32) * 32, 0, st>>>(gyb, bpart, V, Cout, bchunk);
        k_sum_parts<<<nblk(Cout), 256, 0, st>>>(bpart, gb, nb, Cout);
    }
    return cudaGetLastError();
}

cudaError_t nn_weight_flip(const void *w, void *wt, int Cin, int Cout, int Kp, int Kpt,
                           cudaStream_t st) {
    k_weight_flip<<<nblk((size_t)Cin * Kpt), 256, 0, st>>>((const __nv_bfloat16 *)w,
                                                           (__nv_bfloat16 *)wt, Cin, Cout, Kp, Kpt);
    return cudaGetLastError();
}

cudaError_t nn_elementwise(int op, const void *a, const void *b, void *out, size_t n,
                           cudaStream_t st) {
    switch (op) {
        case 0: k_relu_bwd<<<nblk(n), 256, 0, st>>>((const float *)a, (const __nv_bfloat16 *)b,
                                                    (__nv_bfloat16 *)out, n); break;
        case 1: k_cast_bf16<<<nblk(n), 256, 0, st>>>((const float *)a, (__nv_bfloat16 *)out, n); break;
        case 2: k_add_bf16<<<nblk(n), 256, 0, st>>>((const __nv_bfloat16 *)a,
                                                     (const __nv_bfloat16 *)b,
                                                     (__nv_bfloat16 *)out, n); break;
        case 3: k_accum_f32<<<nblk(n), 256, 0, st>>>((const float *)a, (float *)out, n); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t nn_resample(int op, const void *x, void *y, int D, int H, int W, int C, cudaStream_t st) {
    // D, H, W: the fine (large) size for pooling ops, the coarse size for upsampling ops
    switch (op) {
        case 0: k_avgpool2<<<nblk((size_t)D * H * W * C / 8), 256, 0, st>>>(
                    (const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, D, H, W, C); break;
        case 1: k_avgpool2_bwd<<<nblk((size_t)D * H * W * C), 256, 0, st>>>(
                    (const float *)x, (float *)y, D, H, W, C); break;
        case 2:
            if (C % 8 == 0 && (uintptr_t)x % 16 == 0 && (uintptr_t)y % 16 == 0)
                k_upsample2_v8<<<nblk((size_t)D * H * W * C), 256, 0, st>>>(
                    (const uint4 *)x, (uint4 *)y, D, H, W, C / 8);
            else
                k_upsample2<<<nblk((size_t)8 * D * H * W * C), 256, 0, st>>>(
                    (const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, D, H, W, C);
            break;
        case 3: k_upsample2_bwd<<<nblk((size_t)D * H * W * C), 256, 0, st>>>(
                    (const float *)x, (float *)y, D, H, W, C); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t nn_features(const void *img, void *feat, float *scale, size_t n, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(scale, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    k_absmax<<<1024, 256, 0, st>>>((const float2 *)img, n, scale);
    k_features<<<nblk(n), 256, 0, st>>>((const float2 *)img, scale, (__nv_bfloat16 *)feat, n);
    return cudaGetLastError();
}

cudaError_t nn_loss(const float *pred, const void *target, const float *scale, float *sums,
                    float *grad, size_t n, cudaStream_t st) {
    k_loss_sums<<<1, 1024, 0, st>>>(pred, (const float2 *)target, scale, n, sums);
    if (grad) k_loss_grad<<<nblk(n), 256, 0, st>>>(pred, (const float2 *)target, scale, sums, grad, n);
    return cudaGetLastError();
}

cudaError_t nn_check(const float *corr, const void *img, const float *scale, float gain, size_t n,
                     float *out, cudaStream_t st) {
    float *part = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&part, g_check_part);
    if (e != cudaSuccess) return e;
    k_check_part<<<kCheckBlocks, 256, 0, st>>>(corr, (const float2 *)img, scale, gain, n, part);
    k_check_sum<<<1, kCheckBlocks, 0, st>>>(part, out);
    return cudaGetLastError();
}

cudaError_t nn_residual(float *pred, const void *img, const float *scale, float gain, size_t n,
                        cudaStream_t st) {
    k_residual<<<nblk(n), 256, 0, st>>>(pred, (const float2 *)img, scale, gain, n);
    return cudaGetLastError();
}

cudaError_t nn_to_complex(const float *pred, const float *scale, void *img, size_t n,
                          cudaStream_t st) {
    k_to_complex<<<nblk(n), 256, 0, st>>>(pred, scale, (float2 *)img, n);
    return cudaGetLastError();
}

cudaError_t nn_adam(float *p, const float *g, float *m, float *v, void *pb, size_t n, float lr,
                    float b1, float b2, float eps, int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<nblk(n), 256, 0, st>>>(p, g, m, v, (__nv_bfloat16 *)pb, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}
