// C ABI of the learned fast path's kernels (include/polyline.h, "Learned fast
// path"). Argument checks here; the kernels are in nn.cu.
#include <cuda_runtime.h>

#include "../../include/polyline.h"
#include "kernels.h"

namespace {

int padded_k(int cin) { return (27 * cin + 15) / 16 * 16; }

pl_status ret(cudaError_t e, const char *where) {
    return e == cudaSuccess ? PL_OK : pl_internal_cuda_fail(e, where);
}

bool dims_ok(int D, int H, int W) { return D > 0 && H > 0 && W > 0; }

}  // namespace

extern "C" {

int pl_nn_padded_k(int cin) { return padded_k(cin); }

pl_status pl_nn_conv3d(const void *x, const void *w, const float *bias, void *out, int D, int H,
                       int W, int Cin, int Cout, int relu, int out_bf16, void *stream) {
    if (!x || !w || !out || !dims_ok(D, H, W) || Cin <= 0 || Cout <= 0 || Cout > 1024)
        return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_conv3d arguments");
    return ret(nn_conv3d(x, w, bias, out, D, H, W, Cin, Cout, padded_k(Cin), relu, out_bf16,
                         (cudaStream_t)stream), "pl_nn_conv3d");
}

size_t pl_nn_wgrad_workspace(int D, int H, int W, int Cin, int Cout) {
    return sizeof(float) * nn_wgrad_work_floats(D, H, W, Cin, Cout, padded_k(Cin));
}

pl_status pl_nn_conv3d_wgrad(const void *x, const void *gy, float *gw, float *gb, void *work,
                             size_t work_bytes, int D, int H, int W, int Cin, int Cout,
                             void *stream) {
    const int mt = (Cout + 15) / 16;   // m-tiles of 16 output channels: 1, 2, 4 or 8
    if (!x || !gy || !gw || !dims_ok(D, H, W) || Cin <= 0 || Cout <= 0 ||
        !(mt == 1 || mt == 2 || mt == 4 || mt == 8))
        return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_conv3d_wgrad arguments "
                                            "(Cout must be at most 32, or 49-64, or 113-128)");
    if (!work || work_bytes < pl_nn_wgrad_workspace(D, H, W, Cin, Cout))
        return pl_internal_fail(PL_ERR_ARG, "pl_nn_conv3d_wgrad: workspace too small");
    return ret(nn_conv3d_wgrad(x, gy, gw, gb, (float *)work, D, H, W, Cin, Cout, padded_k(Cin),
                               (cudaStream_t)stream), "pl_nn_conv3d_wgrad");
}

pl_status pl_nn_weight_flip(const void *w, void *wt, int Cin, int Cout, void *stream) {
    if (!w || !wt || Cin <= 0 || Cout <= 0) return pl_internal_fail(PL_ERR_ARG, "bad weight_flip");
    return ret(nn_weight_flip(w, wt, Cin, Cout, padded_k(Cin), padded_k(Cout),
                              (cudaStream_t)stream), "pl_nn_weight_flip");
}

pl_status pl_nn_elementwise(int op, const void *a, const void *b, void *out, size_t n,
                            void *stream) {
    if (!a || !out || op < 0 || op > 3 || ((op == 0 || op == 2) && !b))
        return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_elementwise arguments");
    return ret(nn_elementwise(op, a, b, out, n, (cudaStream_t)stream), "pl_nn_elementwise");
}

pl_status pl_nn_resample(int op, const void *x, void *y, int D, int H, int W, int C,
                         void *stream) {
    if (!x || !y || !dims_ok(D, H, W) || C <= 0 || op < 0 || op > 3 ||
        (op <= 1 && ((D | H | W) & 1)))
        return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_resample arguments");
    return ret(nn_resample(op, x, y, D, H, W, C, (cudaStream_t)stream), "pl_nn_resample");
}

pl_status pl_nn_features(const void *img, void *feat, float *scale, size_t n, void *stream) {
    if (!img || !feat || !scale) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_features");
    return ret(nn_features(img, feat, scale, n, (cudaStream_t)stream), "pl_nn_features");
}

pl_status pl_nn_loss(const float *pred, const void *target, const float *scale, float *sums,
                     float *grad, size_t n, void *stream) {
    if (!pred || !target || !scale || !sums) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_loss");
    return ret(nn_loss(pred, target, scale, sums, grad, n, (cudaStream_t)stream), "pl_nn_loss");
}

pl_status pl_nn_residual(float *pred, const void *img, const float *scale, float gain, size_t n,
                         void *stream) {
    if (!pred || !img || !scale) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_residual");
    return ret(nn_residual(pred, img, scale, gain, n, (cudaStream_t)stream), "pl_nn_residual");
}

pl_status pl_nn_check(const float *corr, const void *img, const float *scale, float gain,
                      size_t n, float *out, void *stream) {
    if (!corr || !img || !scale || !out) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_check");
    return ret(nn_check(corr, img, scale, gain, n, out, (cudaStream_t)stream), "pl_nn_check");
}

pl_status pl_nn_to_complex(const float *pred, const float *scale, void *img, size_t n,
                           void *stream) {
    if (!pred || !scale || !img) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_to_complex");
    return ret(nn_to_complex(pred, scale, img, n, (cudaStream_t)stream), "pl_nn_to_complex");
}

pl_status pl_nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, size_t n,
                     float lr, float b1, float b2, float eps, int step, void *stream) {
    if (!p || !g || !m || !v || step < 1) return pl_internal_fail(PL_ERR_ARG, "bad pl_nn_adam");
    return ret(nn_adam(p, g, m, v, p_bf16, n, lr, b1, b2, eps, step, (cudaStream_t)stream),
               "pl_nn_adam");
}

}  // extern "C"
