// rid_cond.cu -- the condition of L1 and an FP64 solve for X (the
// mixed-precision variant's "FP64 triangular solve for X when the L1 condition
// estimate demands it").
//
// L1 (k x k, unit lower) and L2 ((n-k) x k) are the LUPP multipliers of the
// skeleton rows J and of the other rows, in pivot order; X^T(J^c,:) = T =
// L2 L1^{-1} (Eq. inty).  The driver keeps T itself, updated block by block
// (T(rest,new) = L-hat(rest) L-hat(piv)^{-1}, T(rest,old) -= T(rest,new) T(piv,old)),
// and freezes the rows T(piv_t, 0:tb_t) of each block's pivots when they are
// chosen.  With D = diag(L-hat(piv_t)) and N the k x k strictly block-lower
// matrix whose block row t is T(piv_t, 0:tb_t), L1 = (I - N)^{-1} D: block row t
// of L1 is T(piv_t, 0:tb_t) L1(0:tb_t, 0:tb_t) next to L-hat(piv_t).  Hence
//     L1^{-1} = D^{-1} (I - N)
// explicitly, and ||L1^{-1}||_1 is a sum of small block products per column.
// ||L1||_1 is read from the stored multipliers.  The FP64 solve runs block
// back-substitution T L1 = L2 from the last column block to the first.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rid_internal.h"

namespace rid {

// L(act[i], tb:tb+bt) = this block's multipliers: all bt columns of the rows that
// stay active; for the pivot of step q, columns < q, then the unit diagonal, then 0.
template <typename T>
__global__ void k_store_l(int na, int bt, const T* __restrict__ S, int64_t lds, const int32_t* __restrict__ piv,
                          const int32_t* __restrict__ pivmark, const int32_t* __restrict__ act, T* __restrict__ L,
                          int64_t ldl, int64_t tb, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int64_t rest = (int64_t)na * bt;
  const int64_t total = rest + (int64_t)bt * bt;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < rest) {
      const int64_t i = e / bt;
      const int c = (int)(e - i * bt);
      if (!pivmark[i]) L[(int64_t)act[i] * ldl + tb + c] = S[i * lds + c];
    } else {
      const int64_t f = e - rest;
      const int q = (int)(f / bt), c = (int)(f - (int64_t)q * bt);
      const int32_t row = piv[q];
      const T v = c < q ? S[(int64_t)row * lds + c] : (c == q ? T(1) : T(0));
      L[(int64_t)act[row] * ldl + tb + c] = v;
    }
  }
}

template <typename T>
cudaError_t store_l(int na, int bt, const T* S, int64_t lds, const int32_t* piv, const int32_t* pivmark,
                    const int32_t* act, T* L, int64_t ldl, int64_t tb, const int32_t* done, cudaStream_t s) {
  const int64_t total = (int64_t)na * bt + (int64_t)bt * bt;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_store_l<T><<<(int)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(na, bt, S, lds, piv, pivmark, act, L, ldl, tb, done);
  return cudaGetLastError();
}

// Column sums of |L1|: 1 + sum_{q > c} |L(J[q], c)|.
template <typename T>
__global__ void k_l1_colsum(int64_t k, const int32_t* __restrict__ perm, const T* __restrict__ L, int64_t ldl,
                            double* __restrict__ colsum) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= k) return;
  double acc = 1.0;
  for (int64_t q = c + 1; q < k; ++q) acc += fabs((double)L[(int64_t)perm[q] * ldl + c]);
  colsum[c] = acc;
}

// Column sums of |L1^{-1}| = |D^{-1}(I - N)|: for column c (block tc) and every
// block t >= tc, the block's part of column c of (I - N) is e_(c - tc b) (t = tc)
// or -T(J[t b + r], c) (t > tc, read from the pivots' rows of T in X), times the
// block's inverse diagonal block Linv_t (row-major bt x bt).
constexpr int kColThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kColThreads)
    k_linv_colsum(int64_t k, int b, const int32_t* __restrict__ perm, const T* __restrict__ X, int64_t ldx,
                  const T* __restrict__ Linv_all, double* __restrict__ colsum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Li = reinterpret_cast<T*>(smem_raw);  // b x b
  const int64_t c = blockIdx.x * (int64_t)kColThreads + threadIdx.x;
  const int64_t c_first = blockIdx.x * (int64_t)kColThreads;
  const int64_t nblk = (k + b - 1) / b;
  const int64_t tc = c < k ? c / b : nblk;
  T v[kMaxBlockCond];
  double acc = 0.0;
  for (int64_t t = c_first / b; t < nblk; ++t) {
    const int bt = (int)((k - t * b) < b ? (k - t * b) : b);
    const T* src = Linv_all + t * (int64_t)b * b;
    for (int e = threadIdx.x; e < bt * bt; e += kColThreads) Li[e] = src[e];
    __syncthreads();
    if (t >= tc && c < k) {
      for (int r = 0; r < bt; ++r)
        v[r] = t == tc ? (r == c - t * b ? T(1) : T(0)) : -X[(int64_t)perm[t * b + r] * ldx + c];
      for (int r = 0; r < bt; ++r) {
        T w = T(0);
        for (int rp = 0; rp <= r; ++rp) w = fma(Li[r * bt + rp], v[rp], w);
        acc += fabs((double)w);
      }
    }
    __syncthreads();
  }
  if (c < k) colsum[c] = acc;
}

template <typename T>
cudaError_t cond_colsums(int64_t k, int b, const int32_t* perm, const T* L, int64_t ldl, const T* X, int64_t ldx,
                         const T* Linv_all, double* colsum_l1, double* colsum_inv, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if (b > kMaxBlockCond) return cudaErrorInvalidValue;
  const int blocks = (int)((k + kColThreads - 1) / kColThreads);
  if (L != nullptr) k_l1_colsum<T><<<blocks, kColThreads, 0, s>>>(k, perm, L, ldl, colsum_l1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)b * b * sizeof(T);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_linv_colsum<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_linv_colsum<T><<<blocks, kColThreads, smem, s>>>(k, b, perm, X, ldx, Linv_all, colsum_inv);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 solve
__global__ void k_iota(int64_t k, int32_t* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

// L1 (k x k, row-major, FP64): unit lower with the skeleton rows' multipliers.
template <typename T>
__global__ void k_gather_l1(int64_t k, const int32_t* __restrict__ perm, const T* __restrict__ L, int64_t ldl,
                            double* __restrict__ L1) {
  const int64_t total = k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / k, c = e - q * k;
    L1[e] = c < q ? (double)L[(int64_t)perm[q] * ldl + c] : (c == q ? 1.0 : 0.0);
  }
}

// T64 (na x k, row-major, FP64) = L2: the multipliers of the rows left active.
template <typename T>
__global__ void k_gather_l2(int64_t na, int64_t k, const int32_t* __restrict__ act, const T* __restrict__ L,
                            int64_t ldl, double* __restrict__ T64) {
  const int64_t total = na * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e - r * k;
    T64[e] = (double)L[(int64_t)act[r] * ldl + c];
  }
}

// Row r of the column block (bq wide, row stride ld) times Linv (bq x bq,
// row-major, lower): out(c) = sum_{c' >= c} in(c') Linv(c', c).
__global__ void k_rmul_linv(int64_t na, int bq, double* __restrict__ Tb, int64_t ld, const double* __restrict__ Linv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Li = reinterpret_cast<double*>(smem_raw);
  for (int e = threadIdx.x; e < bq * bq; e += blockDim.x) Li[e] = Linv[e];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < na; r += (int64_t)gridDim.x * blockDim.x) {
    double* row = Tb + r * ld;
    double in[kMaxBlockCond];
    for (int c = 0; c < bq; ++c) in[c] = row[c];
    for (int c = 0; c < bq; ++c) {
      double acc = 0.0;
      for (int cp = c; cp < bq; ++cp) acc = fma(in[cp], Li[cp * bq + c], acc);
      row[c] = acc;
    }
  }
}

// X(0:k, act[r]) = T64(r, :) in the working precision.
template <typename T>
__global__ void k_store_x(int64_t na, int64_t k, const int32_t* __restrict__ act, const double* __restrict__ T64,
                          T* __restrict__ X, int64_t ldx) {
  const int64_t total = na * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e - r * k;
    X[(int64_t)act[r] * ldx + c] = (T)T64[e];
  }
}

static int grid_for(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  return (int)(blocks < 1 ? 1 : blocks);
}

template <typename T>
cudaError_t resolve_x_f64(int64_t k, int b, int64_t na, const int32_t* perm, const int32_t* act, const T* L,
                          int64_t ldl, double* L1, double* T64, double* Linv64, int32_t* iota, T* X, int64_t ldx,
                          cudaStream_t s, int* launches) {
  if (k <= 0 || na <= 0) return cudaSuccess;
  if (b > kMaxBlockCond) return cudaErrorInvalidValue;
  int nl = 0;
  k_iota<<<grid_for(k), 256, 0, s>>>(k, iota);
  k_gather_l1<T><<<grid_for(k * k), 256, 0, s>>>(k, perm, L, ldl, L1);
  k_gather_l2<T><<<grid_for(na * k), 256, 0, s>>>(na, k, act, L, ldl, T64);
  nl += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nblk = (k + b - 1) / b;
  for (int64_t q = nblk - 1; q >= 0; --q) {
    const int64_t c0 = q * b;
    const int bq = (int)((k - c0) < b ? (k - c0) : b);
    const int64_t c1 = c0 + bq;
    if (k - c1 > 0) {
      // T(:, block q) -= T(:, c1:k) L1(c1:k, block q)
      Operand<double> a{T64, k, nullptr, c1};
      Operand<double> bop{L1 + c1 * k, k, nullptr, c0};
      EpiArgs<double> ep{T64 + c0, k, 0, nullptr, nullptr};
      e = gemm_gather<double>((int)na, bq, (int)(k - c1), 1, false, a, bop, kEpiSubRows, ep, nullptr, s);
      if (e != cudaSuccess) return e;
      ++nl;
    }
    // times the inverse of the unit-lower diagonal block L1(block q, block q)
    e = linv<double>(bq, L1 + c0, k, iota + c0, Linv64, nullptr, s);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)bq * bq * sizeof(double);
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_rmul_linv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_rmul_linv<<<grid_for(na), 256, smem, s>>>(na, bq, T64 + c0, k, Linv64);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nl += 2;
  }
  k_store_x<T><<<grid_for(na * k), 256, 0, s>>>(na, k, act, T64, X, ldx);
  ++nl;
  if (launches != nullptr) *launches += nl;
  return cudaGetLastError();
}

#define RID_COND_INST(T)                                                                                          \
  template cudaError_t store_l<T>(int, int, const T*, int64_t, const int32_t*, const int32_t*, const int32_t*, T*, \
                                  int64_t, int64_t, const int32_t*, cudaStream_t);                               \
  template cudaError_t cond_colsums<T>(int64_t, int, const int32_t*, const T*, int64_t, const T*, int64_t,      \
                                       const T*, double*, double*, cudaStream_t);                                \
  template cudaError_t resolve_x_f64<T>(int64_t, int, int64_t, const int32_t*, const int32_t*, const T*, int64_t, \
                                        double*, double*, double*, int32_t*, T*, int64_t, cudaStream_t, int*);

RID_COND_INST(float)
RID_COND_INST(double)

}  // namespace rid
