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
//
// FP64 input is summed exactly in integers: GB300 issues about two FP64
// instructions per clock per SM, and each element of A feeds zeta sums.  A is
// converted once per call to fixed point per column (F = round(A 2^(54-e)) for
// |A| < 2^e, an error of at most 2^-55 max|A(:,j)| per term, as the digits of the
// FP64-accurate tensor-core sketch), every entry of the sketch is the exact
// integer sum of +-F (int64 within a tile, 128 bits across tiles), and one
// conversion rounds it to FP64 (then the scale sqrt(b/zeta), one more rounding).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

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
__device__ __forceinline__ long long load_as_f(const long long* p) { return *p; }

// The accumulator of an entry and its final value: FP32 sums for FP32 / BF16 input;
// for the fixed-point FP64 input, exact int64 sums within a tile (a sketch row takes
// at most one term per tile row: 256 terms below 2^54 each stay below 2^62) folded
// into an exact 128-bit total once per tile.
template <typename TS>
struct SpAcc {
  using part = TS;
  using type = TS;
};
template <>
struct SpAcc<long long> {
  using part = long long;
  using type = __int128;
};
// s + a or s - a, branch-free: the sign flips a's sign bit (float) or negates by mask (int64)
__device__ __forceinline__ float sp_add(float s, float a, uint32_t neg) {
  return s + __int_as_float(__float_as_int(a) ^ (int)(neg << 31));
}
__device__ __forceinline__ long long sp_add(long long s, long long a, uint32_t neg) {
  const long long msk = -(long long)neg;
  return s + ((a ^ msk) - msk);
}
template <typename TS, typename TO>
__device__ __forceinline__ TO sp_final(typename SpAcc<TS>::type s, TO v, int ex) {
  if constexpr (sizeof(TS) == 8) {
    // s 2^ex: |s| < 2^54 times the terms (< 2^74), so s >> 32 fits 64 bits
    const long long hi = (long long)(s >> 32);
    const long long lo = (long long)(s & (__int128)0xFFFFFFFFll);
    return tcx::fixed_to_double(hi, lo, ex) * v;
  } else {
    return s * v;
  }
}

// F(i, j) = round(A(i, j) 2^(54 - e_j)) with |A(:, j)| < 2^e_j (column-major, ld m):
// |F| < 2^54, an error of at most 2^-55 max|A(:, j)| per term.
__global__ void k_sparse_fixed(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                               const int32_t* __restrict__ colexp, long long* __restrict__ F) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    F[e] = tcx::fixed_of<7>(A[i + j * lda], colexp[j] + 1);
  }
}

cudaError_t sparse_fixed_prepare(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* colexp, long long* F,
                                 cudaStream_t s) {
  cudaError_t e = f64_colexp(A, lda, m, n, colexp, s);
  if (e != cudaSuccess) return e;
  int64_t g = (m * n + 255) / 256;
  if (g > 8192) g = 8192;
  k_sparse_fixed<<<(int)g, 256, 0, s>>>(A, lda, m, n, colexp, F);
  return cudaGetLastError();
}

// Asynchronous copy of one element (4 or 8 bytes) or a BF16 pair (4 bytes) into shared
// memory; src_bytes < bytes zero-fills the rest (0: the whole element).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(tcx::smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ float tile_value(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float tile_value(const float* p) { return *p; }
__device__ __forceinline__ long long tile_value(const long long* p) { return *p; }

// out[z][j][t*b + r] (row stride out_ld) = sqrt(b/zeta) * sum over the rows i of
// split z with a code for sketch row r of block t: sign * A(i, j).  Grid: x over
// 32-column tiles of A, y over groups of TG blocks, z over splits of the rows of A
// (ktiles tiles of 256 rows each).  Per tile (the next one already in flight by
// cp.async into the other buffer):
//   1. per-row bit masks of the tile rows that hit each sketch row of the group
//      (word-major, so a warp's 32 tile rows spread over the banks);
//   2. the codes sorted by sketch row into a CSR list, ascending tile row within a
//      row (rank = popcount of the row's mask below the bit): a fixed order;
//   3. warp w sums rows r = w + 8q of every block of the group, lane = column,
//      four list entries at a time.
// Sketch rows t*b + r >= rows (a last block cut short) are not written.
template <typename TA, typename TS, typename TO, int RPW>
__global__ void __launch_bounds__(kSpThreads, sizeof(TS) == 8 ? 1 : 2)
    k_sparse_sketch(int64_t m, int64_t n, const TA* __restrict__ A, int64_t lda, const uint8_t* __restrict__ P,
                    int zeta, int b, int blocks, int64_t rows, int ktiles, TO* __restrict__ out, int64_t out_ld,
                    int64_t zstride, TO v, const int32_t* __restrict__ colexp, const int32_t* done) {
  using TC = decltype(tile_value((const TS*)nullptr));
  using Acc = typename SpAcc<TC>::type;
  constexpr int TG = (sizeof(Acc) > 8 ? 16 : 32) / RPW;  // blocks per CTA
  constexpr int NR = TG * 8 * RPW;                         // sketch rows of the group (padded)
  constexpr int LDT = kSpI + (sizeof(TS) == 2 ? 2 : 1);    // tile row stride (elements)
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char sp_raw[];
  TS* tiles = reinterpret_cast<TS*>(sp_raw);                                  // [2][kSpJ][LDT]
  uint32_t* mask = reinterpret_cast<uint32_t*>(tiles + 2 * kSpJ * LDT);      // [kSpWords][NR]
  uint32_t* negm = mask + kSpWords * NR;                                      // [kSpWords][NR]
  int* woff = reinterpret_cast<int*>(negm + kSpWords * NR);                   // [NR][kSpWords + 1]
  uint16_t* list = reinterpret_cast<uint16_t*>(woff + NR * (kSpWords + 1));  // [TG * kSpI * zeta]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * kSpJ;
  const int tg0 = blockIdx.y * TG;
  const int ng = min(TG, blocks - tg0);
  const int64_t itile0 = (int64_t)blockIdx.z * ktiles;
  const int64_t ntiles = (m + kSpI - 1) / kSpI;
  const int64_t itile1 = min(ntiles, itile0 + ktiles);
  Acc acc[TG * RPW];
#pragma unroll
  for (int u = 0; u < TG * RPW; ++u) acc[u] = Acc(0);

  // tile it of A into buffer bf: a warp per column, lanes along the rows
  auto issue = [&](int64_t it, int bf) {
    const int64_t i0 = it * kSpI;
    for (int jj = wid; jj < kSpJ; jj += kSpThreads / 32) {
      const int64_t j = j0 + jj;
      TS* dst = tiles + (bf * kSpJ + jj) * LDT;
      const TA* src = A + (j < n ? j : 0) * lda + i0;
      if constexpr (sizeof(TS) == 2) {  // BF16 pairs
#pragma unroll
        for (int q = 0; q < kSpI / 64; ++q) {
          const int ii = 2 * (lane + 32 * q);
          const int64_t left = j < n ? m - (i0 + ii) : 0;
          const int bytes = left >= 2 ? 4 : (left == 1 ? 2 : 0);
          cp_async<4>(dst + ii, bytes ? (const void*)(src + ii) : (const void*)A, bytes);
        }
      } else {
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) {
          const int ii = lane + 32 * q;
          const bool in = j < n && i0 + ii < m;
          cp_async<sizeof(TS)>(dst + ii, in ? (const void*)(src + ii) : (const void*)A, in ? (int)sizeof(TS) : 0);
        }
      }
    }
    cp_async_commit();
  };

  if (itile0 < itile1) issue(itile0, 0);
  for (int64_t it = itile0; it < itile1; ++it) {
    const int cur = (int)((it - itile0) & 1);
    const int64_t i0 = it * kSpI;
    if (it + 1 < itile1) {
      issue(it + 1, cur ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    // 1. masks
    for (int e = tid; e < 2 * kSpWords * NR; e += kSpThreads) mask[e] = 0u;
    __syncthreads();
    for (int e = tid; e < ng * kSpI; e += kSpThreads) {
      const int t = e / kSpI, ii = e - t * kSpI;
      const int64_t i = i0 + ii;
      if (i >= m) continue;
      const uint8_t* c = P + ((int64_t)(tg0 + t) * m + i) * zeta;
      const uint32_t bit = 1u << (ii & 31);
      for (int jz = 0; jz < zeta; ++jz) {
        const int code = c[jz];
        const int slot = (ii >> 5) * NR + t * 8 * RPW + (code & 127);
        atomicOr(&mask[slot], bit);
        if (code & 128) atomicOr(&negm[slot], bit);
      }
    }
    __syncthreads();
    // 2. row offsets (an exclusive scan of the rows' counts, one warp), then the list
    if (wid == 0) {
      int carry = 0;
      for (int r0 = 0; r0 < NR; r0 += 32) {
        const int r = r0 + lane;
        int cnt[kSpWords];
        int tot = 0;
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) {
          cnt[q] = __popc(mask[q * NR + r]);
          tot += cnt[q];
        }
        int incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += y;
        }
        int base = carry + incl - tot;
#pragma unroll
        for (int q = 0; q < kSpWords; ++q) {
          woff[r * (kSpWords + 1) + q] = base;
          base += cnt[q];
        }
        woff[r * (kSpWords + 1) + kSpWords] = base;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    for (int e = tid; e < ng * kSpI; e += kSpThreads) {
      const int t = e / kSpI, ii = e - t * kSpI;
      const int64_t i = i0 + ii;
      if (i >= m) continue;
      const uint8_t* c = P + ((int64_t)(tg0 + t) * m + i) * zeta;
      const uint32_t below = (1u << (ii & 31)) - 1u;
      for (int jz = 0; jz < zeta; ++jz) {
        const int code = c[jz];
        const int r = t * 8 * RPW + (code & 127);
        const int pos = woff[r * (kSpWords + 1) + (ii >> 5)] + __popc(mask[(ii >> 5) * NR + r] & below);
        list[pos] = (uint16_t)(ii | ((code & 128) << 8));
      }
    }
    __syncthreads();
    // 3. the gather-add
    const TS* arow = tiles + (cur * kSpJ + lane) * LDT;
#pragma unroll
    for (int u = 0; u < TG * RPW; ++u) {
      const int t = u / RPW, r = wid + 8 * (u % RPW);
      if (t < ng && r < b) {
        const int rr = t * 8 * RPW + r;
        const int e0 = woff[rr * (kSpWords + 1)], e1 = woff[rr * (kSpWords + 1) + kSpWords];
        // four independent partial sums (four entries in flight), combined in a fixed
        // order at the end of the tile: deterministic, and exact for the integer sums
        using Part = typename SpAcc<TC>::part;
        Part s0 = Part(0), s1 = Part(0), s2 = Part(0), s3 = Part(0);
        int e = e0;
        for (; e + 4 <= e1; e += 4) {
          const uint32_t l0 = list[e], l1 = list[e + 1], l2 = list[e + 2], l3 = list[e + 3];
          const TC a0 = tile_value(arow + (l0 & 0x7FFF)), a1 = tile_value(arow + (l1 & 0x7FFF));
          const TC a2 = tile_value(arow + (l2 & 0x7FFF)), a3 = tile_value(arow + (l3 & 0x7FFF));
          s0 = sp_add(s0, a0, l0 >> 15);
          s1 = sp_add(s1, a1, l1 >> 15);
          s2 = sp_add(s2, a2, l2 >> 15);
          s3 = sp_add(s3, a3, l3 >> 15);
        }
        for (; e < e1; ++e) {
          const uint32_t l = list[e];
          s0 = sp_add(s0, tile_value(arow + (l & 0x7FFF)), l >> 15);
        }
        acc[u] = acc[u] + (((Acc)s0 + (Acc)s1) + ((Acc)s2 + (Acc)s3));
      }
    }
    __syncthreads();
  }
  const int64_t j = j0 + lane;
  if (j < n) {
    TO* o = out + (int64_t)blockIdx.z * zstride + j * out_ld;
    const int ex = colexp != nullptr ? colexp[j] - 54 : 0;
#pragma unroll
    for (int u = 0; u < TG * RPW; ++u) {
      const int t = u / RPW, r = wid + 8 * (u % RPW);
      const int64_t c = (int64_t)(tg0 + t) * b + r;
      if (t < ng && r < b && c < rows) o[c] = sp_final<TC, TO>(acc[u], v, ex);
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

template <typename TA, typename TS, typename TO, int RPW>
static cudaError_t launch_sparse(int64_t m, int64_t n, const TA* A, int64_t lda, const uint8_t* P, int zeta, int b,
                                 int blocks, int64_t rows, int splits, TO* out, int64_t out_ld, int64_t zstride,
                                 const int32_t* colexp, const int32_t* done, cudaStream_t s) {
  using TC = decltype(tile_value((const TS*)nullptr));
  constexpr int TG = (sizeof(typename SpAcc<TC>::type) > 8 ? 16 : 32) / RPW;
  constexpr int NR = TG * 8 * RPW;
  constexpr int LDT = kSpI + (sizeof(TS) == 2 ? 2 : 1);
  const size_t smem = (size_t)2 * kSpJ * LDT * sizeof(TS) + (size_t)2 * kSpWords * NR * 4 +
                      (size_t)NR * (kSpWords + 1) * 4 + (size_t)TG * kSpI * zeta * 2;
  static SmemLimit lim;
  cudaError_t e = raise_smem(k_sparse_sketch<TA, TS, TO, RPW>, smem, lim);
  if (e != cudaSuccess) return e;
  const int64_t ktiles = (m + kSpI - 1) / kSpI;
  const int per = (int)((ktiles + splits - 1) / splits);
  dim3 grid((unsigned)((n + kSpJ - 1) / kSpJ), (unsigned)((blocks + TG - 1) / TG), (unsigned)splits);
  const TO v = (TO)sqrt((double)b / (double)zeta);
  k_sparse_sketch<TA, TS, TO, RPW><<<grid, kSpThreads, smem, s>>>(m, n, A, lda, P, zeta, b, blocks, rows, per, out,
                                                                 out_ld, zstride, v, colexp, done);
  return cudaGetLastError();
}

template <typename TA, typename TS, typename TO>
static cudaError_t dispatch_sparse(int64_t m, int64_t n, const TA* A, int64_t lda, const uint8_t* P, int zeta, int b,
                                   int64_t rows, int splits, TO* out, int64_t out_ld, int64_t zstride,
                                   const int32_t* colexp, const int32_t* done, cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b || rows < 1 || splits < 1) return cudaErrorInvalidValue;
  const int blocks = (int)((rows + b - 1) / b);
#define RID_SPARSE(R) \
  launch_sparse<TA, TS, TO, R>(m, n, A, lda, P, zeta, b, blocks, rows, splits, out, out_ld, zstride, colexp, done, s)
  if (b <= 8) return RID_SPARSE(1);
  if (b <= 16) return RID_SPARSE(2);
  if (b <= 32) return RID_SPARSE(4);
  if (b <= 64) return RID_SPARSE(8);
  return RID_SPARSE(16);
#undef RID_SPARSE
}

template <typename TA, typename TC>
cudaError_t sparse_sketch(int64_t m, int64_t n, const TA* A, int64_t lda, const uint8_t* P, int zeta, int b,
                          int64_t rows, int splits, TC* out, int64_t out_ld, int64_t zstride, const int32_t* done,
                          cudaStream_t s) {
  // the tile is staged in A's own type; BF16 pairs need 4-byte aligned rows
  if constexpr (sizeof(TA) == 2) {
    if ((lda & 1) != 0 || (reinterpret_cast<uintptr_t>(A) & 3) != 0) return cudaErrorInvalidValue;
  }
  return dispatch_sparse<TA, TA, TC>(m, n, A, lda, P, zeta, b, rows, splits, out, out_ld, zstride, nullptr, done, s);
}

cudaError_t sparse_sketch_fixed(int64_t m, int64_t n, const long long* F, const int32_t* colexp, const uint8_t* P,
                                int zeta, int b, int64_t rows, int splits, double* out, int64_t out_ld,
                                int64_t zstride, const int32_t* done, cudaStream_t s) {
  return dispatch_sparse<long long, long long, double>(m, n, F, m, P, zeta, b, rows, splits, out, out_ld, zstride,
                                                       colexp, done, s);
}

template cudaError_t sparse_sketch<float, float>(int64_t, int64_t, const float*, int64_t, const uint8_t*, int, int,
                                                 int64_t, int, float*, int64_t, int64_t, const int32_t*, cudaStream_t);
template cudaError_t sparse_sketch<__nv_bfloat16, float>(int64_t, int64_t, const __nv_bfloat16*, int64_t,
                                                         const uint8_t*, int, int, int64_t, int, float*, int64_t,
                                                         int64_t, const int32_t*, cudaStream_t);
template cudaError_t sparse_dense<double>(uint64_t, int64_t, int, int, int64_t, int, double*, int64_t, cudaStream_t);
template cudaError_t sparse_dense<float>(uint64_t, int64_t, int, int, int64_t, int, float*, int64_t, cudaStream_t);

}  // namespace rid
