// rid_mlp.cu -- the learned rank predictor: a 35 -> 128 -> 128 -> 1 MLP (tanh)
// in FP32 with hand-written inference, training (forward + backward) and Adam
// kernels.
//
// Inputs (features of the first sketch block, computed on the device):
//   f_i = log10(|U(i,i)| / |U(0,0)|), i < 32  -- leading LUPP pivot magnitudes
//   f_32 = log10 m, f_33 = log10 n, f_34 = log10(relative tolerance)
// standardised with (mu, sigma) stored after the weights.  The output, rescaled
// by (y_mu, y_sigma), is log2 of the rank that the adaptive loop returns.
// The paper relates the pivots of the sketch's LUPP to the spectrum (Remark 1);
// the network only proposes how many sketch rows the second pass draws; the
// plain loop still decides the rank.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "randid.h"
#include "rid_internal.h"

namespace rid {
namespace mlp {

constexpr int kIn = ID_MLP_IN, kH = ID_MLP_HIDDEN;
// parameter layout (floats)
constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kH * kIn;
constexpr int oW2 = oB1 + kH;
constexpr int oB2 = oW2 + kH * kH;
constexpr int oW3 = oB2 + kH;
constexpr int oB3 = oW3 + kH;
constexpr int kTrain = oB3 + 1;  // trainable parameters
constexpr int oMu = kTrain;
constexpr int oSig = oMu + kIn;
constexpr int oYmu = oSig + kIn;
constexpr int oYsig = oYmu + 1;
constexpr int kTotal = oYsig + 1;

// One sample's forward pass by a block of kH threads: thread j owns hidden unit j.
__device__ float forward_one(const float* __restrict__ P, const float* x_std, float* h1, float* h2, float* red) {
  const int j = threadIdx.x;
  float z = P[oB1 + j];
  for (int k = 0; k < kIn; ++k) z = fmaf(P[oW1 + j * kIn + k], x_std[k], z);
  h1[j] = tanhf(z);
  __syncthreads();
  z = P[oB2 + j];
  for (int k = 0; k < kH; ++k) z = fmaf(P[oW2 + j * kH + k], h1[k], z);
  h2[j] = tanhf(z);
  // y = w3 . h2 + b3 (warp shuffles, then across the 4 warps)
  float v = P[oW3 + j] * h2[j];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((j & 31) == 0) red[j >> 5] = v;
  __syncthreads();
  const float y = red[0] + red[1] + red[2] + red[3] + P[oB3];
  __syncthreads();
  return y;
}

__global__ void __launch_bounds__(kH) k_forward(const float* __restrict__ P, int64_t batch,
                                                 const float* __restrict__ x, float* __restrict__ y) {
  __shared__ float xs[kIn], h1[kH], h2[kH], red[4];
  for (int64_t i = blockIdx.x; i < batch; i += gridDim.x) {
    if (threadIdx.x < kIn) xs[threadIdx.x] = (x[i * kIn + threadIdx.x] - P[oMu + threadIdx.x]) / P[oSig + threadIdx.x];
    __syncthreads();
    const float out = forward_one(P, xs, h1, h2, red);
    if (threadIdx.x == 0) y[i] = out * P[oYsig] + P[oYmu];
    __syncthreads();
  }
}

// Gradient of L = mean_i (yhat_i - t_i)^2 over the trainable parameters, where
// yhat is the standardised output and t_i = (target_i - y_mu) / y_sigma.  One
// CTA walks the samples in order; thread j accumulates the gradient entries of
// hidden unit j (rows j of W1 and W2, b1[j], b2[j], w3[j]), so the sums are
// deterministic.  loss receives L.
__global__ void __launch_bounds__(kH) k_loss_grad(const float* __restrict__ P, int64_t batch,
                                                   const float* __restrict__ x, const float* __restrict__ target,
                                                   float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float xs[kIn], h1[kH], h2[kH], dz2[kH], red[4];
  __shared__ float s_dy;
  extern __shared__ float gW2[];  // kH x kH, row j accumulated by thread j only
  const int j = threadIdx.x;
  float gW1[kIn];
  for (int k = 0; k < kIn; ++k) gW1[k] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  for (int k = 0; k < kH; ++k) gW2[j * kH + ((k + j) & (kH - 1))] = 0.f;
  const float inv = 1.f / (float)batch;
  for (int64_t i = 0; i < batch; ++i) {
    if (j < kIn) xs[j] = (x[i * kIn + j] - P[oMu + j]) / P[oSig + j];
    __syncthreads();
    const float yhat = forward_one(P, xs, h1, h2, red);
    if (j == 0) {
      const float t = (target[i] - P[oYmu]) / P[oYsig];
      const float r = yhat - t;
      lsum += r * r;
      s_dy = 2.f * r * inv;
    }
    __syncthreads();
    const float dy = s_dy;
    if (j == 0) gb3 += dy;
    gw3 += dy * h2[j];
    const float d2 = dy * P[oW3 + j] * (1.f - h2[j] * h2[j]);
    dz2[j] = d2;
    gb2 += d2;
    // rotate the column order by j so that the 32 lanes of a warp hit 32 banks
    for (int kk = 0; kk < kH; ++kk) {
      const int k = (kk + j) & (kH - 1);
      gW2[j * kH + k] = fmaf(d2, h1[k], gW2[j * kH + k]);
    }
    __syncthreads();
    float dh1 = 0.f;  // (W2^T dz2)_j
    for (int r = 0; r < kH; ++r) dh1 = fmaf(P[oW2 + r * kH + j], dz2[r], dh1);
    const float d1 = dh1 * (1.f - h1[j] * h1[j]);
    gb1 += d1;
    for (int k = 0; k < kIn; ++k) gW1[k] = fmaf(d1, xs[k], gW1[k]);
    __syncthreads();
  }
  for (int k = 0; k < kH; ++k) grad[oW2 + j * kH + k] = gW2[j * kH + k];
  for (int k = 0; k < kIn; ++k) grad[oW1 + j * kIn + k] = gW1[k];
  grad[oB1 + j] = gb1;
  grad[oB2 + j] = gb2;
  grad[oW3 + j] = gw3;
  if (j == 0) {
    grad[oB3] = gb3;
    *loss = lsum * inv;
  }
}

// omb1 = 1 - beta1 and omb2 = 1 - beta2 come from the host in double precision:
// 1.f - 0.999f is 1.3e-5 away from 0.001 in relative terms.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float b1, float omb1, float b2, float omb2, float eps,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + omb1 * gi;
    const float b = b2 * m2[i] + omb2 * gi * gi;
    m1[i] = a;
    m2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// Features from the pivots of the first block, then one forward pass: the
// predicted rank is written to st->k_pred (rounded up, at least 1).
__device__ void features(const double* piv, int npiv, double m, double n, double rel_tol, float* f) {
  const double p0 = piv[0] > 0.0 ? piv[0] : 1.0;
  for (int i = 0; i < 32; ++i) {
    const double v = i < npiv ? piv[i] : 0.0;
    f[i] = (float)log10(fmax(v / p0, 1e-30));
  }
  f[32] = (float)log10(m);
  f[33] = (float)log10(n);
  f[34] = (float)log10(fmax(rel_tol, 1e-300));
}

__global__ void __launch_bounds__(kH) k_predict(const float* __restrict__ P, const double* piv, int npiv, double m,
                                                 double n, double tol, int tol_rel, DevState* st) {
  __shared__ float f[kIn], xs[kIn], h1[kH], h2[kH], red[4];
  if (threadIdx.x == 0) {
    const double rel = tol_rel ? tol : tol / fmax(sqrt(st->norm2_A), 1e-300);
    features(piv, npiv, m, n, rel, f);
  }
  __syncthreads();
  if (threadIdx.x < kIn) xs[threadIdx.x] = (f[threadIdx.x] - P[oMu + threadIdx.x]) / P[oSig + threadIdx.x];
  __syncthreads();
  const float y = forward_one(P, xs, h1, h2, red);
  if (threadIdx.x == 0) {
    const double lg = (double)(y * P[oYsig] + P[oYmu]);
    double k = exp2(fmin(lg, 40.0));
    if (!(k >= 1.0)) k = 1.0;
    st->k_pred = (int64_t)ceil(k);
  }
}

__global__ void k_features(const double* piv, int npiv, double m, double n, double rel_tol, float* x) {
  if (threadIdx.x == 0 && blockIdx.x == 0) features(piv, npiv, m, n, rel_tol, x);
}

}  // namespace mlp

cudaError_t mlp_predict_rank(const float* params, const double* piv, int npiv, int64_t m, int64_t n, double tol,
                             int tol_rel, DevState* st, cudaStream_t s) {
  mlp::k_predict<<<1, mlp::kH, 0, s>>>(params, piv, npiv, (double)m, (double)n, tol, tol_rel, st);
  return cudaGetLastError();
}

}  // namespace rid

// ====================================================================== C ABI
extern "C" {

int64_t id_mlp_param_count(void) { return rid::mlp::kTotal; }

int id_mlp_forward(const float* params, int64_t batch, const float* x, float* y, void* stream) {
  if (params == nullptr) return -1;
  if (batch < 0) return -2;
  if (x == nullptr && batch > 0) return -3;
  if (y == nullptr && batch > 0) return -4;
  if (batch == 0) return ID_OK;
  const int grid = (int)(batch < 4096 ? batch : 4096);
  rid::mlp::k_forward<<<grid, rid::mlp::kH, 0, static_cast<cudaStream_t>(stream)>>>(params, batch, x, y);
  return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

int id_mlp_loss_grad(const float* params, int64_t batch, const float* x, const float* target, float* grad,
                     float* loss, void* stream) {
  if (params == nullptr) return -1;
  if (batch < 1) return -2;
  if (x == nullptr) return -3;
  if (target == nullptr) return -4;
  if (grad == nullptr) return -5;
  if (loss == nullptr) return -6;
  const size_t smem = sizeof(float) * rid::mlp::kH * rid::mlp::kH;
  static rid::SmemLimit lim;
  if (rid::raise_smem(rid::mlp::k_loss_grad, smem, lim) != cudaSuccess) return ID_ERR_CUDA;
  rid::mlp::k_loss_grad<<<1, rid::mlp::kH, smem, static_cast<cudaStream_t>(stream)>>>(params, batch, x, target,
                                                                                     grad, loss);
  return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

int id_mlp_adam(float* params, const float* grad, float* m1, float* m2, int64_t step, float lr, void* stream) {
  if (params == nullptr) return -1;
  if (grad == nullptr) return -2;
  if (m1 == nullptr) return -3;
  if (m2 == nullptr) return -4;
  if (step < 1) return -5;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
  rid::mlp::k_adam<<<(rid::mlp::kTrain + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grad, m1, m2, rid::mlp::kTrain, lr, (float)b1, (float)(1.0 - b1), (float)b2, (float)(1.0 - b2),
      1e-8f, c1, c2);
  return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

int id_rank_features(const double* pivots, int64_t npiv, int64_t m, int64_t n, double rel_tol, float* x,
                     void* stream) {
  if (pivots == nullptr) return -1;
  if (npiv < 1) return -2;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!(rel_tol > 0.0)) return -5;
  if (x == nullptr) return -6;
  rid::mlp::k_features<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(pivots, (int)(npiv < 32 ? npiv : 32),
                                                                       (double)m, (double)n, rel_tol, x);
  return cudaGetLastError() == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

}  // extern "C"
