// nn.cuh -- launchers of the warm-start network kernels (nn.cu) and of the
// solver-side feature / guess / target kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rf.h"
#include "rf_internal.cuh"

namespace rf {
namespace nn {

// Network shape: input convolution 4 -> 32 (channels padded to 8), four
// residual blocks of two 32 -> 32 convolutions, output convolution 32 -> 1
// (padded to 8).  All 3x3x3.
constexpr int N_LAYERS = 10;
constexpr int C_IN = 4, C_IN_P = 8, C_HID = 32, C_OUT = 1, C_OUT_P = 8;

__host__ __device__ constexpr int round16(int k) { return (k + 15) / 16 * 16; }

// Feature scales (mirrors rf_ws_scales).
struct WsScales {
    double h_scale, lnK_mean, lnK_std, q_scale, t_scale, out_scale;
};

// out[v][co] = act(sum_k A[v][k] W[co][k] + bias[co] (+ res[v][co])):
// BF16 in, FP32 accumulate; out_b (BF16) and/or out_f (FP32) written.
cudaError_t conv3d(cudaStream_t s, int cin, int cout, const void *in, const void *Wb, const float *bias,
                   const void *res, void *out_b, float *out_f, int B, int D, int H, int W, int relu);
// Convolutions on the tcgen05 tensor cores (conv_tc.cu).  in: cin_mem (8 or
// 32) BF16 channels per voxel, zero-padded to cinp (16 or 32) planes; Wb:
// nout x 27 cinp BF16 weights (K = tap cinp + c); nout GEMM columns (16 or
// 32), of which out_ch are written (the row stride of out_b / out_f; with
// nout = 16 only out_ch = 8 and FP32 output).  A device wait that runs out
// sets *fault (and the output is then undefined).
cudaError_t conv3d_tc(cudaStream_t s, int cin_mem, int cinp, int nout, int out_ch, const void *in, const void *Wb,
                      const float *bias, const void *res, void *out_b, float *out_f, int B, int D, int H, int W,
                      int relu, int *fault, int num_sms);
bool conv3d_tc_available(const void *in, const void *Wb);
// dst[n][tap cinp + c] = src[n][tap cin + c] (src rows of kp_src), zero for
// n >= n_src or c >= cin.
void prep_tc_weights(cudaStream_t s, const void *src, int n_src, int cin, int kp_src, int nout, int cinp, void *dst);
// Weight (and bias) gradient of a convolution on the tensor cores (mma.sync):
// X = the layer's BF16 input [voxel][cin], G = the BF16 output gradient
// [voxel][cout]; dW [cout][round16(27 cin)], db [cout] are accumulated into.
// (cin, cout) in {(32, 32), (8, 32), (32, 8)}.
cudaError_t wgrad_mma(cudaStream_t s, int cin, int cout, const void *X, const void *G, int B, int D, int H, int W,
                      float *dW, float *db, int num_sms);
// The 32 -> 32 weight (and bias) gradient on the tcgen05 tensor cores
// (conv_tc.cu), same arguments and accumulation as wgrad_mma; X and G 4-byte
// aligned (X 16 bytes).  A device wait that runs out sets *fault (the sums are then
// incomplete).
cudaError_t wgrad_tc32(cudaStream_t s, const void *X, const void *G, int B, int D, int H, int W, float *dW,
                       float *db, int *fault, int num_sms);
void relu_bwd(cudaStream_t s, const void *y, const float *dy, float *dx, long long n, const float *add);
void to_bf16(cudaStream_t s, const float *a, void *b, long long n);
void add(cudaStream_t s, float *a, const float *b, long long n);
void pad_features(cudaStream_t s, const float *x4, void *x8, long long M);
void mse(cudaStream_t s, const float *pred, const float *target, const float *mask, long long M, float inv_count,
         float *dpred, float *loss);
void adam(cudaStream_t s, float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
          float eps, float c1, float c2);
void prep_weights(cudaStream_t s, const float *W, int Cinp, int Coutp, int KP, int KPt, void *Wb, void *Wt);

// Solver side (one mesh, voxel = cell index p).
void ws_features_f32(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const double *Ks,
                     const WsScales &sc, float q_feat, float dt_feat, float *out);
void ws_features_bf16(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const double *Ks,
                      const WsScales &sc, float q_feat, float dt_feat, void *out);
void ws_guess(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h, const float *y, double scale,
              double *hk);
void ws_target(cudaStream_t s, const Grid &g, const uint8_t *flags, const double *h_new, const double *h_old,
               double inv_scale, float *target, float *mask);

}  // namespace nn
}  // namespace rf

// Warm-start guess of a mesh state (nn_api.cu): features of (h, Ks), the
// network's forward pass, hk = h + y scale on active cells; ordered on s.
rf_status rf_nn_mesh_guess(rf_nn *net, cudaStream_t s, const rf::Grid &g, const uint8_t *flags, const double *h,
                           const double *Ks, const rf::nn::WsScales &sc, float q_feat, float dt_feat, double scale,
                           double *hk, int *fault);
