// rid_sparse.cu -- the sparse-sign sketch (Sec. 5.1 of arXiv:2310.09417, "Sparse
// Sign", zeta = 8 by default): each column of each b-row block of Omega holds zeta
// entries +-sqrt(b/zeta) at distinct rows, so Y = Omega A is a gather-add over
// the rows of A instead of a dense product, bound by reading A once per pass.
//
// Definition (the same published generator on both sides of the parity tests):
// the words u_0, u_1, ... of column i in block t are Philox4x64-10 keyed
// (seed, 1) at counters (i, t, c, 0), c = 0, 1, ..., four words per counter;
// a partial Fisher-Yates shuffle of (0, ..., b-1) places nonzero j at row
// p[j] with r = j + ((u_j >> 32) (b - j)) >> 32 swapped into position j, and
// the entry is negative when u_j is odd.  The scale sqrt(b/zeta) makes
// E[Omega^T Omega] = b I, as for N(0,1) rows, so E = ||S||_F / sqrt(b) keeps
// its meaning.
//
// The sketch: k_sparse_pattern writes each column's zeta codes (row | sign << 7)
// once per pass; k_sparse_sketch stages a 256 x 32 tile of A in shared memory,
// turns the tile's codes into per-row bit masks (which tile rows hit sketch row
// r, and with which sign), and a warp per sketch row walks its mask in ascending
// order with one lane per column of A -- a fixed summation order, no atomics on
// the sums, and one read of A per pass.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_internal.h"

namespace rid {

constexpr int kSpI = 256;       // rows of A per tile
constexpr int kSpJ = 32;        // columns of A per tile (one per lane)
constexpr int kSpThreads = 256; // eight warps
constexpr int kSpWords = kSpI / 32;

// zeta codes of column i of block t: row | (negative << 7), rows distinct.
__device__ __forceinline__ void sparse_column(uint64_t seed, int64_t t, int64_t i, int b, int zeta,
                                              uint8_t* codes) {
  uint8_t p[kSparseMaxB];
  for (int r = 0; r < b; ++r) p[r] = (uint8_t)r;
  uint64_t w[4] = {0, 0, 0, 0};
  for (int j = 0; j < zeta; ++j) {
    if ((j & 3) == 0) {
      w[0] = (uint64_t)i;
      w[1] = (uint64_t)t;
      w[2] = (uint64_t)(j >> 2);
      w[3] = 0;
      philox4x64_10(w[0], w[1], w[2], w[3], seed, 1ull);
    }
    const uint64_t u = w[j & 3];
    const int r = j + (int)(((u >> 32) * (uint64_t)(b - j)) >> 32);
    const uint8_t tmp = p[j];
    p[j] = p[r];
    p[r] = tmp;
    codes[j] = (uint8_t)(p[j] | ((u & 1ull) << 7));
  }
}

__global__ void k_sparse_pattern(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta,
                                 uint8_t* __restrict__ P, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int64_t total = (int64_t)blocks * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / m, i = e - t * m;
    uint8_t c[kSparseMaxB];
    sparse_column(seed, t0 + t, i, b, zeta, c);
    uint8_t* o = P + e * zeta;
    for (int j = 0; j < zeta; ++j) o[j] = c[j];
  }
}

cudaError_t sparse_pattern(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, uint8_t* P,
                           const int32_t* done, cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)blocks * m;
  int64_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  k_sparse_pattern<<<(int)g, 256, 0, s>>>(seed, t0, blocks, b, m, zeta, P, done);
  return cudaGetLastError();
}

// Dense rows of the sparse-sign matrix: block t0 + q at rows q*b .. q*b+b-1 of out
// (row-major, row stride ld), one thread per (block, column).
template <typename T>
__global__ void k_sparse_dense(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, T v,
                               T* __restrict__ out, int64_t ld) {
  const int64_t total = (int64_t)blocks * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / m, i = e - q * m;
    T* col = out + q * b * ld + i;
    for (int r = 0; r < b; ++r) col[(int64_t)r * ld] = T(0);
    uint8_t c[kSparseMaxB];
    sparse_column(seed, t0 + q, i, b, zeta, c);
    for (int j = 0; j < zeta; ++j) col[(int64_t)(c[j] & 127) * ld] = (c[j] & 128) ? -v : v;
  }
}

template <typename T>
cudaError_t sparse_dense(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, T* out, int64_t ld,
                         cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)blocks * m;
  int64_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  const T v = (T)sqrt((double)b / (double)zeta);
  k_sparse_dense<T><<<(int)g, 256, 0, s>>>(seed, t0, blocks, b, m, zeta, v, out, ld);
  return cudaGetLastError();
}

__device__ __forceinline__ float load_as_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float load_as_f(const float* p) { return *p; }
__device__ __forceinline__ double load_as_f(const double* p) { return *p; }

// out[z][j][t*b + r] (row stride out_ld) = sqrt(b/zeta) * sum over the rows i of
// split z with a code for sketch row r of block t: sign * A(i, j).  Grid: x over
// 32-column tiles of A, y over groups of TG blocks, z over splits of the rows of A
// (ktiles tiles of 256 rows each).  Warp w owns rows r = w + 8q (q < RPW) of each
// block of its group; lane = column.  Sketch rows t*b + r >= rows (a last block
// cut short) are not written.
template <typename TA, typename TC, int RPW>
__global__ void __launch_bounds__(kSpThreads, sizeof(TC) == 8 ? 2 : 3)
    k_sparse_sketch(int64_t m, int64_t n, const TA* __restrict__ A, int64_t lda, const uint8_t* __restrict__ P,
                    int zeta, int b, int blocks, int64_t rows, int ktiles, TC* __restrict__ out, int64_t out_ld,
                    int64_t zstride, TC v, const int32_t* done) {
  constexpr int TG = 32 / RPW;  // blocks per CTA
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char sp_raw[];
  TC* As = reinterpret_cast<TC*>(sp_raw);                                   // [kSpJ][kSpI + 1]
  uint32_t* mask = reinterpret_cast<uint32_t*>(As + kSpJ * (kSpI + 1));      // [TG][8 RPW][kSpWords]
  uint32_t* negm = mask + TG * 8 * RPW * kSpWords;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * kSpJ;
  const int tg0 = blockIdx.y * TG;
  const int ng = min(TG, blocks - tg0);
  const int64_t itile0 = (int64_t)blockIdx.z * ktiles;
  const int64_t ntiles = (m + kSpI - 1) / kSpI;
  const int64_t itile1 = min(ntiles, itile0 + ktiles);
  TC acc[TG * RPW];
#pragma unroll
  for (int u = 0; u < TG * RPW; ++u) acc[u] = TC(0);
  const int nmask = TG * 8 * RPW * kSpWords;

  for (int64_t it = itile0; it < itile1; ++it) {
    const int64_t i0 = it * kSpI;
    // 1. the tile of A (zero outside), a warp per column, lanes along the rows
    for (int jj = wid; jj < kSpJ; jj += kSpThreads / 32) {
      const int64_t j = j0 + jj;
      TC* dst = As + jj * (kSpI + 1);
      if (j < n) {
        const TA* src = A + j * lda + i0;
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) {
          const int ii = lane + 32 * q;
          dst[ii] = (i0 + ii < m) ? (TC)load_as_f(src + ii) : TC(0);
        }
      } else {
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) dst[lane + 32 * q] = TC(0);
      }
    }
    for (int e = tid; e < 2 * nmask; e += kSpThreads) mask[e] = 0u;
    __syncthreads();
    // 2. masks: tile row ii hits sketch row r of block t (with sign)
    for (int e = tid; e < ng * kSpI; e += kSpThreads) {
      const int t = e / kSpI, ii = e - t * kSpI;
      const int64_t i = i0 + ii;
      if (i >= m) continue;
      const uint8_t* c = P + ((int64_t)(tg0 + t) * m + i) * zeta;
      const uint32_t bit = 1u << (ii & 31);
      for (int j = 0; j < zeta; ++j) {
        const int code = c[j];
        const int r = code & 127;
        const int slot = (t * 8 * RPW + r) * kSpWords + (ii >> 5);
        atomicOr(&mask[slot], bit);
        if (code & 128) atomicOr(&negm[slot], bit);
      }
    }
    __syncthreads();
    // 3. the gather-add: warp-uniform walk over each owned row's mask
    const TC* arow = As + lane * (kSpI + 1);
#pragma unroll
    for (int u = 0; u < TG * RPW; ++u) {
      const int t = u / RPW, r = wid + 8 * (u % RPW);
      if (t < ng && r < b) {
        const uint32_t* mw = mask + (t * 8 * RPW + r) * kSpWords;
        const uint32_t* nw = negm + (t * 8 * RPW + r) * kSpWords;
        TC s = acc[u];
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) {
          uint32_t bits = mw[q];
          const uint32_t neg = nw[q];
          while (bits) {
            const int bpos = __ffs(bits) - 1;
            bits &= bits - 1;
            const TC a = arow[32 * q + bpos];
            s = ((neg >> bpos) & 1u) ? s - a : s + a;
          }
        }
        acc[u] = s;
      }
    }
    __syncthreads();
  }
  const int64_t j = j0 + lane;
  if (j < n) {
    TC* o = out + (int64_t)blockIdx.z * zstride + j * out_ld;
#pragma unroll
    for (int u = 0; u < TG * RPW; ++u) {
      const int t = u / RPW, r = wid + 8 * (u % RPW);
      const int64_t c = (int64_t)(tg0 + t) * b + r;
      if (t < ng && r < b && c < rows) o[c] = acc[u] * v;
    }
  }
}

int sparse_splits(int64_t m, int64_t n, int sms) {
  const int64_t ctiles = (n + kSpJ - 1) / kSpJ;
  const int64_t ktiles = (m + kSpI - 1) / kSpI;
  int64_t s = (8 * (int64_t)sms + ctiles - 1) / ctiles;  // about four waves at two CTAs per SM
  if (s > 16) s = 16;
  if (s > ktiles) s = ktiles;
  if (s < 1) s = 1;
  // the count actually used: whole tiles per split
  const int64_t per = (ktiles + s - 1) / s;
  return (int)((ktiles + per - 1) / per);
}

template <typename TA, typename TC, int RPW>
static cudaError_t launch_sparse(int64_t m, int64_t n, const TA* A, int64_t lda, const uint8_t* P, int zeta, int b,
                                 int blocks, int64_t rows, int splits, TC* out, int64_t out_ld, int64_t zstride,
                                 const int32_t* done, cudaStream_t s) {
  constexpr int TG = 32 / RPW;
  const size_t smem = (size_t)kSpJ * (kSpI + 1) * sizeof(TC) + (size_t)2 * TG * 8 * RPW * kSpWords * 4;
  static SmemLimit lim;
  cudaError_t e = raise_smem(k_sparse_sketch<TA, TC, RPW>, smem, lim);
  if (e != cudaSuccess) return e;
  const int64_t ktiles = (m + kSpI - 1) / kSpI;
  const int per = (int)((ktiles + splits - 1) / splits);
  dim3 grid((unsigned)((n + kSpJ - 1) / kSpJ), (unsigned)((blocks + TG - 1) / TG), (unsigned)splits);
  const TC v = (TC)sqrt((double)b / (double)zeta);
  k_sparse_sketch<TA, TC, RPW><<<grid, kSpThreads, smem, s>>>(m, n, A, lda, P, zeta, b, blocks, rows, per, out,
                                                             out_ld, zstride, v, done);
  return cudaGetLastError();
}

template <typename TA, typename TC>
cudaError_t sparse_sketch(int64_t m, int64_t n, const TA* A, int64_t lda, const uint8_t* P, int zeta, int b,
                          int64_t rows, int splits, TC* out, int64_t out_ld, int64_t zstride, const int32_t* done,
                          cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b || rows < 1 || splits < 1) return cudaErrorInvalidValue;
  const int blocks = (int)((rows + b - 1) / b);
#define RID_SPARSE(R) launch_sparse<TA, TC, R>(m, n, A, lda, P, zeta, b, blocks, rows, splits, out, out_ld, zstride, done, s)
  if (b <= 8) return RID_SPARSE(1);
  if (b <= 16) return RID_SPARSE(2);
  if (b <= 32) return RID_SPARSE(4);
  if (b <= 64) return RID_SPARSE(8);
  return RID_SPARSE(16);
#undef RID_SPARSE
}

template cudaError_t sparse_sketch<double, double>(int64_t, int64_t, const double*, int64_t, const uint8_t*, int, int,
                                                   int64_t, int, double*, int64_t, int64_t, const int32_t*,
                                                   cudaStream_t);
template cudaError_t sparse_sketch<float, float>(int64_t, int64_t, const float*, int64_t, const uint8_t*, int, int,
                                                 int64_t, int, float*, int64_t, int64_t, const int32_t*, cudaStream_t);
template cudaError_t sparse_sketch<__nv_bfloat16, float>(int64_t, int64_t, const __nv_bfloat16*, int64_t,
                                                         const uint8_t*, int, int, int64_t, int, float*, int64_t,
                                                         int64_t, const int32_t*, cudaStream_t);
template cudaError_t sparse_dense<double>(uint64_t, int64_t, int, int, int64_t, int, double*, int64_t, cudaStream_t);
template cudaError_t sparse_dense<float>(uint64_t, int64_t, int, int, int64_t, int, float*, int64_t, cudaStream_t);

}  // namespace rid
