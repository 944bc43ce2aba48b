// rid_post.cu -- kernels of the steps that follow a column ID: the a-posteriori
// certificate of its error and the residual block U_r of Remark 1 (Sec. 3.2 of
// arXiv:2310.09417).  The heavy parts (the fresh sketch, the residual product,
// the LUPP of the extra rows) reuse the ID's own kernels; these are the index
// conversions and the reductions around them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_internal.h"

namespace rid {

// out[c] = (int32) J[c]; an index outside [0, n) records kErrBadIndex and maps to 0.
__global__ void k_index32(const int64_t* __restrict__ J, int64_t k, int64_t n, int32_t* __restrict__ out,
                          DevState* st) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = J[c];
    if (j < 0 || j >= n) {
      atomicOr(&st->err, kErrBadIndex);
      out[c] = 0;
    } else {
      out[c] = (int32_t)j;
    }
  }
}

cudaError_t index32(const int64_t* J, int64_t k, int64_t n, int32_t* out, DevState* st, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  int64_t blocks = (k + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_index32<<<(int)blocks, 256, 0, s>>>(J, k, n, out, st);
  return cudaGetLastError();
}

__global__ void k_iota32(int32_t* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

cudaError_t iota32(int32_t* a, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_iota32<<<(int)blocks, 256, 0, s>>>(a, n);
  return cudaGetLastError();
}

// U_r from the LUPP of the extra rows' Schur complement S (na x p, row stride lds):
// after the panel, pivot row piv[c] holds U(c, c:p) and is not updated again, so
// U_r(c, j) = S(piv[c], j) for j >= c.  One block writes U_r (p x p, column-major,
// ldu; zero below the diagonal), the columns act[piv[c]] of the extra pivots, and
// stats = {sum U_r(i,j)^2, max |U_r(i,j)|}.
template <typename T>
__global__ void k_ur_extract(int p, int na, const T* __restrict__ S, int64_t lds, const int32_t* __restrict__ piv,
                             const int32_t* __restrict__ act, T* __restrict__ U, int64_t ldu,
                             int64_t* __restrict__ Jx, double* __restrict__ stats) {
  double acc = 0.0, mx = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int c = e % p, j = e / p;  // consecutive threads write consecutive rows of a column
    const int r = piv[c];
    T u = T(0);
    if (j >= c && r >= 0 && r < na) u = S[(int64_t)r * lds + j];
    U[c + (int64_t)j * ldu] = u;
    const double d = (double)u;
    acc += d * d;
    mx = fmax(mx, fabs(d));
  }
  if (Jx != nullptr)
    for (int c = threadIdx.x; c < p; c += blockDim.x) Jx[c] = (piv[c] >= 0 && piv[c] < na) ? act[piv[c]] : -1;
  const double tot = block_sum(acc);
  __shared__ double s_mx[32];
  double m = mx;
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double g = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g = fmax(g, s_mx[w]);
    stats[0] = tot;
    stats[1] = g;
  }
}

template <typename T>
cudaError_t ur_extract(int p, int na, const T* S, int64_t lds, const int32_t* piv, const int32_t* act, T* U,
                       int64_t ldu, int64_t* Jx, double* stats, cudaStream_t s) {
  k_ur_extract<T><<<1, 256, 0, s>>>(p, na, S, lds, piv, act, U, ldu, Jx, stats);
  return cudaGetLastError();
}

template cudaError_t ur_extract<double>(int, int, const double*, int64_t, const int32_t*, const int32_t*, double*,
                                        int64_t, int64_t*, double*, cudaStream_t);
template cudaError_t ur_extract<float>(int, int, const float*, int64_t, const int32_t*, const int32_t*, float*,
                                       int64_t, int64_t*, double*, cudaStream_t);

}  // namespace rid
