// rid_kernels.cu -- SIMT kernels of the randomized column ID (FP64 and FP32).
//
// Column-ID orientation (the paper's row ID of A^T, Sec. 4): the sketch is
// Y = Omega A (b x n per block), stored transposed as G (n x rows, row-major:
// row j holds the sketch of column j of A).  LUPP runs on the rows of G.
// Rows are never physically swapped: the not-yet-pivoted rows are listed in
// `act` (ascending column index of A), pivots in `perm32` / J, and rows are
// gathered through these index lists.  The interpolation matrix is kept in
// the caller's X buffer throughout (column j of X = row j of L2 L1^{-1}).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "rid_internal.h"

namespace rid {

// Element conversions (round to nearest) shared by the FP64/FP32/BF16 instantiations.
template <typename T>
__device__ __forceinline__ T from_double(double x) {
  return static_cast<T>(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) {
  return __double2bfloat16(x);
}
template <>
__device__ __forceinline__ __nv_fp8_e4m3 from_double<__nv_fp8_e4m3>(double x) {
  __nv_fp8_e4m3 q;
  q.__x = __nv_cvt_double_to_fp8(x, __NV_SATFINITE, __NV_E4M3);  // nearest even, saturating at +-448
  return q;
}
template <typename T>
__device__ __forceinline__ double to_double(T x) {
  return static_cast<double>(x);
}
__device__ __forceinline__ double to_double(__nv_bfloat16 x) { return static_cast<double>(__bfloat162float(x)); }

// ============================================================ Gaussian rows
// FP32 / BF16 / E4M3 outputs are converted from the FP32 value directly (the same
// rounding of the same value as through FP64, without FP64 instructions: GB300
// issues about two per clock per SM); indices are 32-bit when they fit (a 64-bit
// division is an FP64-pipe routine).
template <typename T>
__device__ __forceinline__ T from_float(float x);
template <>
__device__ __forceinline__ float from_float<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __nv_fp8_e4m3 from_float<__nv_fp8_e4m3>(float x) {
  __nv_fp8_e4m3 q;
  q.__x = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);  // nearest even, saturating at +-448
  return q;
}

template <typename T, typename I>
__device__ __forceinline__ void gaussian_quad(uint64_t seed, int64_t row0, I e, I nq, int64_t m, T* __restrict__ out,
                                              int64_t ld) {
  const I i = e / nq, q = e - i * nq;
  uint64_t x0 = (uint64_t)q, x1 = (uint64_t)(row0 + (int64_t)i), x2 = 0, x3 = 0;
  philox4x64_10(x0, x1, x2, x3, seed, 0ull);
  T* o = out + (int64_t)i * ld + 4 * (int64_t)q;
  const int64_t lim = m - 4 * (int64_t)q;
  if constexpr (sizeof(T) == 8) {
    double z[4];
    box_muller(x0, x1, z[0], z[1]);
    box_muller(x2, x3, z[2], z[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < lim) o[j] = from_double<T>(z[j]);
  } else {
    float f[4];
    if constexpr (sizeof(T) <= 2) {  // BF16 / E4M3 output: Box-Muller in FP32 on 24-bit uniforms
      box_muller_f32(x0, x1, f[0], f[1]);
      box_muller_f32(x2, x3, f[2], f[3]);
    } else {  // FP32 output: FP32 evaluation on 53-bit uniforms
      box_muller_f32_53(x0, x1, f[0], f[1]);
      box_muller_f32_53(x2, x3, f[2], f[3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < lim) o[j] = from_float<T>(f[j]);
  }
}

template <typename T>
__global__ void k_gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, T* __restrict__ out,
                                int64_t ld, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int64_t nq = (m + 3) >> 2;
  const int64_t total = rows * nq;
  if (total + (int64_t)gridDim.x * blockDim.x < ((int64_t)1 << 31)) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (int)total; e += gridDim.x * blockDim.x)
      gaussian_quad<T, int>(seed, row0, e, (int)nq, m, out, ld);
  } else {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
      gaussian_quad<T, int64_t>(seed, row0, e, nq, m, out, ld);
  }
}

template <typename T>
cudaError_t gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, T* out, int64_t ld,
                          const int32_t* done, cudaStream_t s) {
  const int64_t total = rows * ((m + 3) >> 2);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_gaussian_rows<T><<<(int)blocks, 256, 0, s>>>(seed, row0, rows, m, out, ld, done);
  return cudaGetLastError();
}

// ============================================================ ||A||_F and finiteness
template <typename T>
__global__ void k_norm2_partial(int64_t m, int64_t n, const T* __restrict__ A, int64_t lda,
                                double* part, DevState* st) {
  double acc = 0.0;
  bool finite = true;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const T* a = A + j * lda;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const double v = to_double(a[i]);
      // finiteness from the exponent bits (integer pipe): one FP64 instruction per element
      finite = finite && ((__double_as_longlong(v) >> 52) & 0x7FF) != 0x7FF;
      acc += v * v;
    }
  }
  if (!finite) atomicOr(&st->err, kErrNonFinite);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// BF16 columns 16-byte aligned (lda a multiple of 8): eight elements per load, the
// squares summed exactly in FP32 and in float-float groups of 64 (sq_add_bits),
// folded into FP64 -- no per-element FP64 work, which on GB300 (about two FP64
// instructions per clock per SM) made this pass take ~20x its HBM time.
__global__ void k_norm2_bf16(int64_t m, int64_t n, const __nv_bfloat16* __restrict__ A, int64_t lda, double* part,
                             DevState* st) {
  double acc = 0.0;
  bool finite = true;
  const int64_t nv = m / 8;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const uint4* a = reinterpret_cast<const uint4*>(A + j * lda);
    float hi = 0.f, lo = 0.f;
    int grp = 0;
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
      const uint4 w = __ldg(a + v);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sq_add_bits(ws[q] << 16, hi, lo, acc, finite);
        sq_add_bits(ws[q] & 0xFFFF0000u, hi, lo, acc, finite);
      }
      if (++grp == 8) {
        acc += (double)hi + (double)lo;
        hi = lo = 0.f;
        grp = 0;
      }
    }
    const uint16_t* r = reinterpret_cast<const uint16_t*>(A + j * lda);
    for (int64_t i = nv * 8 + threadIdx.x; i < m; i += blockDim.x) sq_add_bits((uint32_t)r[i] << 16, hi, lo, acc, finite);
    acc += (double)hi + (double)lo;
  }
  if (!finite) atomicOr(&st->err, kErrNonFinite);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// FP32 columns: four elements per load when 16-byte aligned, each square's rounding
// error recovered exactly by an FMA and summed in float-float groups of 64
// (sq_add_f32), folded into FP64.
__global__ void k_norm2_f32(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda, double* part,
                            DevState* st) {
  double acc = 0.0;
  bool finite = true;
  const bool vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0;
  const int64_t nv = vec ? m / 4 : 0;
  float hi = 0.f, lo = 0.f;
  int grp = 0;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const float* a = A + j * lda;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
      const float4 w = __ldg(a4 + v);
      sq_add_f32(w.x, hi, lo, acc, finite);
      sq_add_f32(w.y, hi, lo, acc, finite);
      sq_add_f32(w.z, hi, lo, acc, finite);
      sq_add_f32(w.w, hi, lo, acc, finite);
      if (++grp == 16) {
        acc += (double)hi + (double)lo;
        hi = lo = 0.f;
        grp = 0;
      }
    }
    for (int64_t i = nv * 4 + threadIdx.x; i < m; i += blockDim.x) {
      sq_add_f32(a[i], hi, lo, acc, finite);
      if (++grp == 16) {
        acc += (double)hi + (double)lo;
        hi = lo = 0.f;
        grp = 0;
      }
    }
  }
  acc += (double)hi + (double)lo;
  if (!finite) atomicOr(&st->err, kErrNonFinite);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
cudaError_t norm2_partial(int64_t m, int64_t n, const T* A, int64_t lda, double* part, int nparts,
                          DevState* st, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    k_norm2_f32<<<nparts, 256, 0, s>>>(m, n, A, lda, part, st);
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 2) {
    if ((lda % 8) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0) {
      k_norm2_bf16<<<nparts, 256, 0, s>>>(m, n, A, lda, part, st);
      return cudaGetLastError();
    }
  }
  k_norm2_partial<T><<<nparts, 256, 0, s>>>(m, n, A, lda, part, st);
  return cudaGetLastError();
}

__global__ void k_norm2_final(const double* part, int nparts, DevState* st) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) st->norm2_A = tot;
}

cudaError_t norm2_final(const double* part, int nparts, DevState* st, cudaStream_t s) {
  k_norm2_final<<<1, 256, 0, s>>>(part, nparts, st);
  return cudaGetLastError();
}

// ============================================================ gather-GEMM
// 64 x 64 output tile per block, K step 16, 256 threads each owning a 4 x 4
// sub-tile strided by 16 (rows ty + 16 i, columns tx + 16 j), so that shared
// reads of a warp hit consecutive words and global writes are coalesced.
constexpr int kGM = 64, kGN = 64, kGK = 16;

template <typename T, bool BK, int EPI>
__global__ void __launch_bounds__(256)
    k_gemm_gather(int M, int N, int K, int kchunk, Operand<T> a, Operand<T> b, EpiArgs<T> ep,
                  const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ T As[kGK][kGM + 1];
  __shared__ T Bs[kGK][kGN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);

  // K-major loaders: row lr, four consecutive k starting at lk
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const T* arow = nullptr;
  if (m0 + lr < M) arow = a.base + (int64_t)(a.idx ? a.idx[m0 + lr] : m0 + lr) * a.ld + a.off;
  const T* brow_k = nullptr;
  if (BK && n0 + lr < N) brow_k = b.base + (int64_t)(b.idx ? b.idx[n0 + lr] : n0 + lr) * b.ld + b.off;
  // N-major loader: k row lq, four consecutive columns starting at lc
  const int lq = tid >> 4, lc = (tid & 15) * 4;

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += kGK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + lk + u;
      As[lk + u][lr] = (arow != nullptr && k < kend) ? arow[k] : T(0);
    }
    if (BK) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + lk + u;
        Bs[lk + u][lr] = (brow_k != nullptr && k < kend) ? brow_k[k] : T(0);
      }
    } else {
      const int q = k0 + lq;
      const T* br = nullptr;
      if (q < kend) br = b.base + (int64_t)(b.idx ? b.idx[q] : q) * b.ld + b.off;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = n0 + lc + u;
        Bs[lq][lc + u] = (br != nullptr && c < N) ? br[c] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= M) continue;
    if (EPI == kEpiStore) {
      T* o = ep.out + blockIdx.z * ep.zstride + (int64_t)r * ep.out_ld;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = n0 + tx + 16 * j;
        if (c < N) o[c] = acc[i][j];
      }
    } else {
      if (ep.skip != nullptr && ep.skip[r] != 0) continue;
      T* o = ep.out + (int64_t)(ep.out_idx ? ep.out_idx[r] : r) * ep.out_ld;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = n0 + tx + 16 * j;
        if (c < N) o[c] -= acc[i][j];
      }
    }
  }
}

// Gather-GEMM for the store epilogue (the sketch and Schur products, FP32 and FP64):
// 128 x 64 tile, 256 threads each owning 8 rows x 4 columns (thread (ty, tx) =
// (tid / 16, tid % 16): a warp reads two A fragments and sixteen B fragments of
// shared memory per k, broadcast across its lanes), K steps of 32 double-buffered
// through registers and shared memory.  Tiles are stored transposed (As[k][m],
// Bs[k][n]) with rows padded by 4 floats: a warp's 8 k x 4 rows of a load land
// in 32 distinct banks and the 16-byte fragment reads stay aligned.
constexpr int kSM = 128, kSN = 64, kSK = 32;
constexpr int kSAld = kSM + 4, kSBld = kSN + 4;
template <typename T>
constexpr size_t sgemm_smem() {
  return (size_t)2 * kSK * (kSAld + kSBld) * sizeof(T);
}

// Vector of four for the fragment reads.
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_32a;
};

template <typename T, bool BK>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    k_sgemm_gather(int M, int N, int K, int kchunk, Operand<T> a, Operand<T> b, EpiArgs<T> ep,
                   const int32_t* done) {
  using V4 = typename Vec4<T>::type;
  if (done != nullptr && *done) return;
  extern __shared__ __align__(32) unsigned char sg_raw[];
  T* As = reinterpret_cast<T*>(sg_raw);  // [2][kSK][kSAld]
  T* Bs = As + 2 * kSK * kSAld;          // [2][kSK][kSBld]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kSM, n0 = blockIdx.y * kSN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int ntiles = kend > kbeg ? (kend - kbeg + kSK - 1) / kSK : 0;

  // loader coordinates: lanes cover 8 consecutive k of 4 rows
  const int lk = lane & 7, lr = warp * 4 + (lane >> 3);  // lr < 32
  const T* ap[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int m = m0 + g * 32 + lr;
    ap[g] = m < M ? a.base + (int64_t)(a.idx ? a.idx[m] : m) * a.ld + a.off : nullptr;
  }
  const T* bp[2];
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int n = n0 + g * 32 + lr;
    bp[g] = (BK && n < N) ? b.base + (int64_t)(b.idx ? b.idx[n] : n) * b.ld + b.off : nullptr;
  }
  T ra[16], rb[8];
  auto load = [&](int k0) {
#pragma unroll
    for (int it = 0; it < 16; ++it) {
      const int k = k0 + (it & 3) * 8 + lk;
      const T* p = ap[it >> 2];
      ra[it] = (p != nullptr && k < kend) ? p[k] : T(0);
    }
    if (BK) {
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int k = k0 + (it & 3) * 8 + lk;
        const T* p = bp[it >> 2];
        rb[it] = (p != nullptr && k < kend) ? p[k] : T(0);
      }
    } else {
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int e = it * 256 + tid, kk = e >> 6, n = e & 63;
        const int k = k0 + kk;
        rb[it] = (k < kend && n0 + n < N) ? b.base[(int64_t)(b.idx ? b.idx[k] : k) * b.ld + b.off + n0 + n] : T(0);
      }
    }
  };
  auto store = [&](int buf) {
    T* as = As + buf * kSK * kSAld;
    T* bs = Bs + buf * kSK * kSBld;
#pragma unroll
    for (int it = 0; it < 16; ++it) as[((it & 3) * 8 + lk) * kSAld + (it >> 2) * 32 + lr] = ra[it];
    if (BK) {
#pragma unroll
      for (int it = 0; it < 8; ++it) bs[((it & 3) * 8 + lk) * kSBld + (it >> 2) * 32 + lr] = rb[it];
    } else {
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int e = it * 256 + tid;
        bs[(e >> 6) * kSBld + (e & 63)] = rb[it];
      }
    }
  };

  T acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  if (ntiles > 0) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  for (int t = 0; t < ntiles; ++t) {
    if (t + 1 < ntiles) load(kbeg + (t + 1) * kSK);
    const T* as = As + (t & 1) * kSK * kSAld + ty * 8;
    const T* bs = Bs + (t & 1) * kSK * kSBld + tx * 4;
#pragma unroll 8
    for (int kk = 0; kk < kSK; ++kk) {
      const V4 a0 = *reinterpret_cast<const V4*>(as + kk * kSAld);
      const V4 a1 = *reinterpret_cast<const V4*>(as + kk * kSAld + 4);
      const V4 bv = *reinterpret_cast<const V4*>(bs + kk * kSBld);
      const T av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const T bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bw[j], acc[i][j]);
    }
    if (t + 1 < ntiles) store((t + 1) & 1);
    __syncthreads();
  }

  T* out = ep.out + blockIdx.z * ep.zstride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + ty * 8 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx * 4 + j;
      if (c < N) out[(int64_t)r * ep.out_ld + c] = acc[i][j];
    }
  }
}

static int split_chunk(int K, int splits) {
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  return ((kchunk + kGK - 1) / kGK) * kGK;
}

int gemm_splits(int K, int splits) {
  if (K <= 0) return 1;
  const int kchunk = split_chunk(K, splits);
  return (K + kchunk - 1) / kchunk;
}

template <typename T>
cudaError_t gemm_gather(int M, int N, int K, int splits, bool b_kmajor, Operand<T> a, Operand<T> b,
                        int epi, EpiArgs<T> ep, const int32_t* done, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int kchunk = split_chunk(K, splits);
  splits = (K + kchunk - 1) / kchunk;
  // the double-buffered kernel for stores; in FP64 only for the sketch (K-major B):
  // its one block per SM measured slower than the 64 x 64 kernel on the Schur shapes
  if (epi == kEpiStore && (sizeof(T) == 4 || b_kmajor)) {
    constexpr size_t smem = sgemm_smem<T>();
    static SmemLimit lim_kmajor, lim_nmajor;
    cudaError_t e = raise_smem(k_sgemm_gather<T, true>, smem, lim_kmajor);
    if (e == cudaSuccess) e = raise_smem(k_sgemm_gather<T, false>, smem, lim_nmajor);
    if (e != cudaSuccess) return e;
    dim3 g((M + kSM - 1) / kSM, (N + kSN - 1) / kSN, splits);
    if (b_kmajor)
      k_sgemm_gather<T, true><<<g, 256, smem, s>>>(M, N, K, kchunk, a, b, ep, done);
    else
      k_sgemm_gather<T, false><<<g, 256, smem, s>>>(M, N, K, kchunk, a, b, ep, done);
    return cudaGetLastError();
  }
  dim3 grid((M + kGM - 1) / kGM, (N + kGN - 1) / kGN, splits);
  if (b_kmajor) {
    if (epi == kEpiStore)
      k_gemm_gather<T, true, kEpiStore><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, b, ep, done);
    else
      k_gemm_gather<T, true, kEpiSubRows><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, b, ep, done);
  } else {
    if (epi == kEpiStore)
      k_gemm_gather<T, false, kEpiStore><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, b, ep, done);
    else
      k_gemm_gather<T, false, kEpiSubRows><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, b, ep, done);
  }
  return cudaGetLastError();
}

// ============================================================ split-K reductions
// Threads over the rows of a row-block (x), rows of G over y and the grid: no
// 64-bit division per element; the partials are summed in split order.
template <typename T>
__global__ void k_splitk_reduce(int64_t n, int rows, int64_t ldp, int64_t ldg, int nz, int64_t zs,
                                const T* __restrict__ P, T* __restrict__ G, const int32_t* done) {
  if (done != nullptr && *done) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; j < n; j += (int64_t)gridDim.x * blockDim.y)
    for (int c = threadIdx.x; c < rows; c += blockDim.x) {
      const int64_t off = j * ldp + c;
      T acc = P[off];
      for (int z = 1; z < nz; ++z) acc += P[z * zs + off];
      G[j * ldg + c] = acc;
    }
}

template <typename T>
cudaError_t splitk_reduce_ld(int64_t n, int rows, int64_t ldp, int64_t ldg, int nz, int64_t zs, const T* P, T* G,
                             const int32_t* done, cudaStream_t s) {
  const int tx = rows >= 64 ? 64 : 32, ty = 256 / tx;
  int64_t blocks = (n + ty - 1) / ty;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  k_splitk_reduce<T><<<(int)blocks, dim3(tx, ty), 0, s>>>(n, rows, ldp, ldg, nz, zs, P, G, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t splitk_reduce(int64_t n, int rows, int64_t ldg, int nz, int64_t zs, const T* P, T* G,
                          const int32_t* done, cudaStream_t s) {
  return splitk_reduce_ld<T>(n, rows, ldg, ldg, nz, zs, P, G, done, s);
}

// S = G(act, col0:col0+w) - sum of the split-K partials of L2 L1^{-1} G(perm, .)
template <typename T>
__global__ void k_schur_finish(int na, int w, const int32_t* __restrict__ act, const T* __restrict__ G,
                               int64_t ldg, int64_t col0, int nz, int64_t zs, const T* __restrict__ P,
                               T* __restrict__ S, int64_t lds, double* e2part, const int32_t* done) {
  if (done != nullptr && *done) return;
  double acc2 = 0.0;
  float hi = 0.f, lo = 0.f;  // FP32: float-float sums of the squares (no per-element FP64 work)
  bool finite = true;
  int grp = 0;
  // a warp per row of S, lanes along the row
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < na; i += (int64_t)gridDim.x * wpb)
    for (int c = lane; c < w; c += 32) {
      T v = G[(int64_t)act[i] * ldg + col0 + c];
      T sub = T(0);
      for (int z = 0; z < nz; ++z) sub += P[z * zs + i * lds + c];
      v -= sub;
      S[i * lds + c] = v;
      if constexpr (sizeof(T) == 4) {
        sq_add_f32(v, hi, lo, acc2, finite);
        if (++grp == 64) {
          acc2 += (double)hi + (double)lo;
          hi = lo = 0.f;
          grp = 0;
        }
      } else {
        acc2 += (double)v * (double)v;
      }
    }
  if constexpr (sizeof(T) == 4) acc2 += finite ? (double)hi + (double)lo : (double)INFINITY;
  const double tot = block_sum(acc2);
  if (threadIdx.x == 0) e2part[blockIdx.x] = tot;
}

template <typename T>
cudaError_t schur_finish(int na, int w, const int32_t* act, const T* G, int64_t ldg, int64_t col0, int nz,
                         int64_t zs, const T* P, T* S, int64_t lds, double* e2part, int nparts,
                         const int32_t* done, cudaStream_t s) {
  k_schur_finish<T><<<nparts, 256, 0, s>>>(na, w, act, G, ldg, col0, nz, zs, P, S, lds, e2part, done);
  return cudaGetLastError();
}

__global__ void k_decide(const double* e2part, int nparts, int w, double tol, int tol_rel, int64_t tb,
                         int last, double* trace, int round, DevState* st) {
  if (st->done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += e2part[i];
  const double e2 = block_sum(acc);
  if (threadIdx.x == 0) {
    const double E = sqrt(e2 / (double)w);
    const double thr = tol_rel ? tol * sqrt(st->norm2_A) : tol;
    st->est = E;
    st->thr = thr;
    st->rounds = round + 1;
    if (trace != nullptr) trace[round] = E;
    if (E <= thr) {
      st->done = 1;
      st->k_final = tb;
    } else if (last) {
      st->done = 1;
      st->k_final = tb;
      st->tol_not_met = 1;
    }
  }
}

cudaError_t decide(const double* e2part, int nparts, int w, double tol, int tol_rel, int64_t tb, int last,
                   double* trace, int round, DevState* st, cudaStream_t s) {
  k_decide<<<1, 256, 0, s>>>(e2part, nparts, w, tol, tol_rel, tb, last, trace, round, st);
  return cudaGetLastError();
}

// ============================================================ LUPP panel
// One cooperative launch factors S (na x w) for `steps` pivots.  Block b owns
// rows [b*chunk, min(na, (b+1)*chunk)), staged in shared memory (row stride
// w + 1: column reads hit distinct banks) when they fit.  Each pivot step:
// block-local argmax of |S(i,c)| over unselected rows (ties to the smallest row
// index = smallest column index of A, since `act` is ascending), publication of
// the block's candidate, one bounded grid barrier, the global pivot and its
// row, then division by the pivot and the rank-1 update (Eq. lupps) of the
// block's unselected rows.  Rows are marked, never swapped.  Look-ahead: column
// c+1 of the update, the candidate for pivot c+1 and the arrival at the next
// barrier come first; the remaining columns are updated while the barrier fills.
// Every entry receives the same single FMA per pivot as without look-ahead.
//
// The global pivot comes from two 64-bit atomic maxima that every block adds
// before the barrier: (top, ~row) and (top, row), top = the leading 32 bits of
// |S(i,c)|'s pattern.  The first names the smallest row among the candidates of
// largest top; when the second names the same row no other candidate shares
// that top, and the row is the exact argmax.  Otherwise (FP64 candidates equal
// in their leading 32 bits) every block compares the published full patterns.
// For FP32 the top is the whole pattern and the first key is exact.  A step thus
// costs the barrier and two L2 round trips on one or two lines, whatever the
// number of blocks.  Key slots rotate over three steps (block 0 clears the next
// one before it arrives at a barrier: every block has read the slot two steps
// back) and alternate between launches like the barrier counter (block 0 clears
// the other launch's slots).
constexpr int kPanelThreads = 256;
constexpr int kPanelMaxW = 128;

// Pivot search key: |S(i,c)| by its IEEE bit pattern (sign cleared; the order of
// the patterns is the order of the values), then the smaller row index: the
// largest key wins.  lo = ~row (never 0 for a row), so {0, 0} is "no candidate".
// Integer comparisons only (GB300 issues about two FP64 instructions per clock
// per SM).
struct PivKey {
  unsigned long long hi;
  unsigned lo;
};
__device__ __forceinline__ PivKey key_pick(PivKey a, PivKey b) {
  return (b.hi > a.hi || (b.hi == a.hi && b.lo > a.lo)) ? b : a;
}
__device__ __forceinline__ PivKey warp_key_max(PivKey a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    PivKey o;
    o.hi = __shfl_xor_sync(0xffffffffu, a.hi, off);
    o.lo = __shfl_xor_sync(0xffffffffu, a.lo, off);
    a = key_pick(a, o);
  }
  return a;
}
// Block-wide key maximum (every thread gets it); blockDim.x a multiple of 32.
__device__ __forceinline__ PivKey block_key_max(PivKey a) {
  __shared__ unsigned long long s_hi[32];
  __shared__ unsigned s_lo[32];
  a = warp_key_max(a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_hi[wid] = a.hi;
    s_lo[wid] = a.lo;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  PivKey b;
  b.hi = lane < nw ? s_hi[lane] : 0ull;
  b.lo = lane < nw ? s_lo[lane] : 0u;
  b = warp_key_max(b);  // every warp reduces the same values
  __syncthreads();      // s_hi / s_lo are reused by the next call
  return b;
}
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long mag_bits(float x) {
  return (unsigned long long)((unsigned)__float_as_int(x) & 0x7FFFFFFFu);
}
__device__ __forceinline__ unsigned mag_top(unsigned long long hi, double) { return (unsigned)(hi >> 31); }
__device__ __forceinline__ unsigned mag_top(unsigned long long hi, float) { return (unsigned)hi; }

// Grid barrier in two halves: every block adds its arrival (after its publications,
// ordered by the block barrier and the release), works on, then waits for the k-th
// barrier's (k+1) nblocks arrivals.  The wait is bounded as in grid_barrier.
__device__ __forceinline__ void grid_arrive(unsigned* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) red_release_add_u32(ctr, 1u);
}
__device__ __forceinline__ bool grid_wait(unsigned* ctr, unsigned target, DevState* st) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if ((int)(ld_acquire_u32(ctr) - target) < 0) {
      const uint64_t t0 = globaltimer_ns();
      unsigned spins = 0;
      while ((int)(ld_acquire_u32(ctr) - target) < 0) {
        if ((++spins & 255u) == 0u) {
          if (ld_acquire_u32(&st->err) & kErrTimeout) { ok = 0; break; }
          if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicOr(&st->err, kErrTimeout);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
    k_panel_lupp(int na, int w, int steps, T* __restrict__ S, int64_t lds, int chunk, int use_smem, int par,
                 int32_t* piv, int32_t* pivmark, double* pivdiag, double* cand_v, int32_t* cand_i,
                 T* cand_rows, DevState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T prow[kPanelMaxW];
  __shared__ int s_piv;
  const int nb = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  if (bid == 0 && tid < 6) (&st->pkey[par ^ 1][0][0])[tid] = 0ull;  // the previous launch has ended
  if (bid == 0 && tid == 0) st->bar[par ^ 1] = 0u;
  if (st->done) return;  // set before the launch or never during it: uniform over the grid
  unsigned* ctr = &st->bar[par];
  unsigned long long* cand_k = reinterpret_cast<unsigned long long*>(cand_v);
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = bid * chunk;
  const int nr = max(0, min(na, r0 + chunk) - r0);
  T* Ss = use_smem ? reinterpret_cast<T*>(smem_raw) : S + (int64_t)r0 * lds;
  const int64_t ldl = use_smem ? w + 1 : lds;
  unsigned char* sel = smem_raw + (use_smem ? (size_t)chunk * (w + 1) * sizeof(T) : 0);

  if (use_smem)
    for (int e = tid; e < nr * w; e += blockDim.x) {
      const int r = e / w, c = e - r * w;
      Ss[(int64_t)r * ldl + c] = S[(int64_t)(r0 + r) * lds + c];
    }
  for (int r = tid; r < chunk; r += blockDim.x) sel[r] = 0;
  __syncthreads();

  // Publish this block's candidate for pivot c (its row complete in every column)
  // and add the arrival at barrier c.
  auto publish = [&](int c, PivKey loc) {
    const int lidx = loc.lo == 0u ? -1 : (int)~loc.lo;
    const int base = (c & 1) * nb;
    unsigned long long* key = &st->pkey[par][c % 3][0];
    if (tid == 0) {
      if (bid == 0) {
        unsigned long long* next = &st->pkey[par][(c + 1) % 3][0];
        next[0] = 0ull;
        next[1] = 0ull;
      }
      if (lidx >= 0) {
        const unsigned long long top = mag_top(loc.hi, T(0));
        red_max_u64(&key[0], (top << 32) | (unsigned long long)loc.lo);
        red_max_u64(&key[1], (top << 32) | (unsigned long long)(unsigned)lidx);
      }
      __stcg(&cand_k[base + bid], loc.hi);
      __stcg(&cand_i[base + bid], lidx);
    }
    if (lidx >= 0) {
      const T* src = Ss + (int64_t)(lidx - r0) * ldl;
      for (int cc = tid; cc < w; cc += blockDim.x) __stcg(&cand_rows[(int64_t)(base + bid) * w + cc], src[cc]);
    }
    grid_arrive(ctr);
  };

  // pivot 0's candidate
  if (steps > 0) {
    PivKey loc{0ull, 0u};
    for (int r = tid; r < nr; r += blockDim.x)
      loc = key_pick(loc, PivKey{mag_bits(Ss[(int64_t)r * ldl]), ~(unsigned)(r0 + r)});
    publish(0, block_key_max(loc));
  }

  for (int c = 0; c < steps; ++c) {
    // 1. every block's candidate for pivot c is published
    if (!grid_wait(ctr, (unsigned)(c + 1) * (unsigned)nb, st)) return;
    const int base = (c & 1) * nb;
    const unsigned long long* key = &st->pkey[par][c % 3][0];
    // 2. global pivot (warp 0 of every block, identically) and its row
    if (wid == 0) {
      const unsigned long long k0 = __ldcg(&key[0]), k1 = __ldcg(&key[1]);
      int gi = k0 == 0ull ? -1 : (int)~(unsigned)k0;
      if (gi >= 0 && sizeof(T) == 8 && (int)(unsigned)k1 != gi) {
        // candidates tie in their leading 32 bits: compare the full patterns
        PivKey g{0ull, 0u};
        for (int q = lane; q < nb; q += 32) {
          const int i = __ldcg(&cand_i[base + q]);
          const unsigned long long h = __ldcg(&cand_k[base + q]);
          if (i >= 0) g = key_pick(g, PivKey{h, ~(unsigned)i});
        }
        g = warp_key_max(g);
        gi = (int)~g.lo;
      }
      if (gi >= 0) {
        const int pblk = gi / chunk;  // the block that published row gi
        for (int cc = lane; cc < w; cc += 32) prow[cc] = __ldcg(&cand_rows[(int64_t)(base + pblk) * w + cc]);
      }
      __syncwarp();
      if (lane == 0) {
        s_piv = gi;
        const T pv = gi >= 0 ? prow[c] : T(0);
        if (gi >= r0 && gi < r0 + nr) sel[gi - r0] = (unsigned char)1;
        if (bid == 0) {
          piv[c] = gi;
          if (pivdiag != nullptr) pivdiag[c] = (double)tabs(pv);
          if (pv == T(0)) atomicAdd(&st->zero_pivots, 1u);
        }
      }
    }
    __syncthreads();
    const T pv = s_piv >= 0 ? prow[c] : T(0);
    const bool elim = pv != T(0);  // a zero column below: nothing to eliminate
    // 3. multipliers l(i) = S(i,c) / pivot
    if (elim)
      for (int r = tid; r < nr; r += blockDim.x)
        if (!sel[r]) Ss[(int64_t)r * ldl + c] = Ss[(int64_t)r * ldl + c] / pv;
    __syncthreads();
    // 4. look-ahead: column c+1 of the rank-1 update (Eq. lupps), the candidate for
    //    pivot c+1 and its row's remaining columns, then the arrival at barrier c+1
    int cand = -1;  // local row of the published candidate (updated already)
    if (c + 1 < steps) {
      const T p1 = prow[c + 1];
      PivKey loc{0ull, 0u};
      for (int r = tid; r < nr; r += blockDim.x)
        if (!sel[r]) {
          T* row = Ss + (int64_t)r * ldl;
          if (elim) row[c + 1] = fma(-row[c], p1, row[c + 1]);
          loc = key_pick(loc, PivKey{mag_bits(row[c + 1]), ~(unsigned)(r0 + r)});
        }
      loc = block_key_max(loc);
      cand = loc.lo == 0u ? -1 : (int)~loc.lo - r0;
      if (elim && cand >= 0 && wid == 0) {
        T* row = Ss + (int64_t)cand * ldl;
        const T l = row[c];
        for (int cc = c + 2 + lane; cc < w; cc += 32) row[cc] = fma(-l, prow[cc], row[cc]);
      }
      __syncthreads();      // the candidate row is complete before it is published
      publish(c + 1, loc);
    }
    // 5. the rest of the rank-1 update while the barrier fills: a warp per row,
    //    lanes along the row, four rows at a time with their loads ahead of the stores
    const int cfirst = c + 1 < steps ? c + 2 : c + 1;
    if (elim && cfirst < w) {
      T p[kPanelMaxW / 32];
#pragma unroll
      for (int j = 0; j < kPanelMaxW / 32; ++j) {
        const int cc = cfirst + lane + 32 * j;
        p[j] = cc < w ? prow[cc] : T(0);
      }
      for (int r = wid; r < nr; r += 4 * nw) {
        T* rp[4];
        T l[4];
        bool live[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int rr = r + u * nw;
          live[u] = rr < nr && !sel[rr] && rr != cand;
          rp[u] = Ss + (int64_t)(live[u] ? rr : 0) * ldl;
          l[u] = live[u] ? rp[u][c] : T(0);
        }
#pragma unroll
        for (int j = 0; j < kPanelMaxW / 32; ++j) {
          const int cc = cfirst + lane + 32 * j;
          if (cc < w) {
            T x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = live[u] ? rp[u][cc] : T(0);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (live[u]) rp[u][cc] = fma(-l[u], p[j], x[u]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (use_smem)
    for (int e = tid; e < nr * w; e += blockDim.x) {
      const int r = e / w, c = e - r * w;
      S[(int64_t)(r0 + r) * lds + c] = Ss[(int64_t)r * ldl + c];
    }
  for (int r = tid; r < nr; r += blockDim.x) pivmark[r0 + r] = sel[r];
}

// Blocks of the panel: one per SM, at least 32 rows each, and enough for the
// rows of a block to fit in shared memory.  With the key exchange a step's
// barrier and round trips cost about the same for any number of blocks (measured
// on GB300: 3.2 - 5.3 us per pivot for 4000 - 20000 rows, FP32 and FP64 alike,
// fastest with the most blocks), so the rows are spread as thin as possible.
// RANDID_PANEL_BLOCKS fixes the count (tuning).
static int panel_blocks_env() {
  static int blocks = -1;
  if (blocks < 0) {
    blocks = 0;
    if (const char* env = getenv("RANDID_PANEL_BLOCKS")) {
      const int v = atoi(env);
      if (v >= 1 && v <= 1024) blocks = v;
    }
  }
  return blocks;
}

template <typename T>
PanelCfg panel_layout(int na, int w, int grid);

template <typename T>
PanelCfg panel_config(int na, int w, int num_sms) {
  const size_t budget = (size_t)200 * 1024;
  const int fit = (int)(budget / ((size_t)(w + 1) * sizeof(T) + 1));  // rows staged in shared memory
  const int need = (na + fit - 1) / fit;
  int most = (na + 31) / 32;
  if (most > num_sms) most = num_sms;
  if (most < 1) most = 1;
  int grid = panel_blocks_env();
  if (grid == 0) grid = most;
  if (grid < need) grid = need;
  if (grid > most) grid = most;
  return panel_layout<T>(na, w, grid);
}

// Rows per block and shared memory for a given block count: rows staged at
// stride w + 1, then one selection byte per row (16-byte padded).
static size_t panel_smem_bytes(int chunk, int w, size_t esz, bool staged) {
  const size_t sel_bytes = ((size_t)chunk + 15) & ~(size_t)15;
  return (staged ? (size_t)chunk * (w + 1) * esz : 0) + sel_bytes;
}

template <typename T>
PanelCfg panel_layout(int na, int w, int grid) {
  PanelCfg cfg;
  if (grid < 1) grid = 1;
  if (na < 1) na = 1;
  int chunk = (na + grid - 1) / grid;
  grid = (na + chunk - 1) / chunk;
  cfg.grid = grid;
  cfg.chunk = chunk;
  cfg.use_smem = panel_smem_bytes(chunk, w, sizeof(T), true) <= (size_t)201 * 1024;
  cfg.smem = panel_smem_bytes(chunk, w, sizeof(T), cfg.use_smem != 0);
  return cfg;
}

template <typename T>
cudaError_t panel_lupp(const PanelCfg& cfg, int na, int w, int steps, int par, T* S, int64_t lds, int32_t* piv,
                       int32_t* pivmark, double* pivdiag, double* cand_v, int32_t* cand_i, T* cand_rows,
                       DevState* st, cudaStream_t s) {
  static SmemLimit lim;
  if (w > kPanelMaxW || (par != 0 && par != 1)) return cudaErrorInvalidValue;
  // the kernel addresses chunk rows at stride w + 1 and the selection bytes after them
  if (cfg.chunk < 1 || (int64_t)cfg.chunk * cfg.grid < na ||
      cfg.smem < panel_smem_bytes(cfg.chunk, w, sizeof(T), cfg.use_smem != 0))
    return cudaErrorInvalidValue;
  cudaError_t e = raise_smem(k_panel_lupp<T>, cfg.smem, lim);
  if (e != cudaSuccess) return e;
  int chunk = cfg.chunk, use_smem = cfg.use_smem;
  void* args[] = {&na, &w, &steps, &S, &lds, &chunk, &use_smem, &par, &piv, &pivmark,
                  &pivdiag, &cand_v, &cand_i, &cand_rows, &st};
  return cudaLaunchCooperativeKernel((const void*)k_panel_lupp<T>, dim3(cfg.grid), dim3(kPanelThreads), args,
                                     cfg.smem, s);
}

// ============================================================ re-blocking
// Inverse X of the unit lower triangular L-hat(piv(0:bt), 0:bt) (bt x bt, row-major),
// X(i, j) = -sum_{c=j}^{i-1} L(i, c) X(c, j) for j < i, each sum taken as four
// interleaved partial sums (c = j + p mod 4, ascending, one FMA per term from 0)
// combined as (s0 + s1) + (s2 + s3) -- the order the batched kernel uses, so both
// give the same bits.  Column j is one CTA with a thread per row i: once X(c, j)
// is final (thread c has added every term c' < c), it is published and every row
// i > c adds its term c to partial (c - j) mod 4.  The same sums in the same order
// as a row-by-row solve, but the dependent chain is one step per row (a combine,
// a block barrier and one FMA) instead of a row's whole dot product and two
// shuffles.  At least 256 threads gather L's pivot rows, eight loads in flight
// per thread.
constexpr int kLinvLoadThreads = 256;
template <typename T>
__global__ void __launch_bounds__(1024)
    k_linv_cols(int bt, const T* __restrict__ S, int64_t lds, const int32_t* __restrict__ piv, T* __restrict__ Linv,
                const int32_t* done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  T* Lp = reinterpret_cast<T*>(smem_raw);  // bt x bt: L(i, c) for j <= c < i
  T* xs = Lp + bt * bt;                    // X(c, j), c >= j
  const int j = blockIdx.x, i = threadIdx.x;
  const int nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < bt * bt; e0 += 8 * nt) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nt, r = e / bt, c = e - r * bt;
      v[u] = (e < bt * bt && r > j && c >= j && c < r) ? S[(int64_t)piv[r] * lds + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u * nt < bt * bt) Lp[e0 + u * nt] = v[u];
  }
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  __syncthreads();
  for (int c = j; c < bt; ++c) {
    if (i == c) xs[c] = c == j ? T(1) : -((s0 + s1) + (s2 + s3));
    __syncthreads();
    if (i > c && i < bt) {
      const T l = Lp[i * bt + c], x = xs[c];
      const int p = (c - j) & 3;
      if (p == 0) s0 = fma(l, x, s0);
      else if (p == 1) s1 = fma(l, x, s1);
      else if (p == 2) s2 = fma(l, x, s2);
      else s3 = fma(l, x, s3);
    }
  }
  if (i < bt) Linv[i * bt + j] = i < j ? T(0) : xs[i];  // xs[i] was written by this thread
}

template <typename T>
cudaError_t linv(int bt, const T* S, int64_t lds, const int32_t* piv, T* Linv, const int32_t* done,
                 cudaStream_t s) {
  static SmemLimit lim;
  if (bt <= 0) return cudaSuccess;
  if (bt > 1024) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)bt * bt + (size_t)bt) * sizeof(T);
  if (smem > (size_t)227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = raise_smem(k_linv_cols<T>, smem, lim);
  if (e != cudaSuccess) return e;
  const int threads = bt > kLinvLoadThreads ? (bt + 31) / 32 * 32 : kLinvLoadThreads;
  k_linv_cols<T><<<bt, threads, smem, s>>>(bt, S, lds, piv, Linv, done);
  return cudaGetLastError();
}

// N(i, c) = sum_{c' >= c} L-hat(i, c') Linv(c', c) for non-pivot rows; the new
// columns tb..tb+bt of X(:, act[i]) are N(i, :) (the new block of L2 L1^{-1}).
// Each sum runs in ascending c' (one FMA per term from 0).  A thread takes the
// columns q and bt-1-q of a row (bt + 1 terms together), so the lanes of a warp
// do equal work: one thread per column spent a third of the FP64 pipe on the
// short sums' idle lanes.
template <typename T>
__global__ void k_make_n(int na, int bt, const T* __restrict__ S, int64_t lds, const T* __restrict__ Linv,
                         const int32_t* __restrict__ pivmark, const int32_t* __restrict__ act, T* __restrict__ Nbuf,
                         T* __restrict__ X, int64_t ldx, int64_t tb, const int32_t* __restrict__ piv,
                         int32_t* __restrict__ pivorig, const int32_t* done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  T* Li = reinterpret_cast<T*>(smem_raw);
  for (int e = threadIdx.x; e < bt * bt; e += blockDim.x) Li[e] = Linv[e];
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < bt; c += blockDim.x) pivorig[c] = act[piv[c]];
  __syncthreads();
  const int hb = (bt + 1) / 2;
  const int64_t total = (int64_t)na * hb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / hb;
    const int q = (int)(e - i * hb);
    if (pivmark[i]) continue;
    const T* l = S + i * lds;
    T* xr = X + (int64_t)act[i] * ldx + tb;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int c = h == 0 ? q : bt - 1 - q;
      if (h == 1 && c == q) break;  // the middle column of an odd bt
      T acc = T(0);
#pragma unroll 8
      for (int cp = c; cp < bt; ++cp) acc = fma(l[cp], Li[cp * bt + c], acc);
      Nbuf[i * bt + c] = acc;
      xr[c] = acc;
    }
  }
}

template <typename T>
cudaError_t make_n(int na, int bt, const T* S, int64_t lds, const T* Linv, const int32_t* pivmark,
                   const int32_t* act, T* Nbuf, T* X, int64_t ldx, int64_t tb, const int32_t* piv,
                   int32_t* pivorig, const int32_t* done, cudaStream_t s) {
  static SmemLimit lim;
  cudaError_t e = raise_smem(k_make_n<T>, (size_t)bt * bt * sizeof(T), lim);
  if (e != cudaSuccess) return e;
  int64_t blocks = ((int64_t)na * ((bt + 1) / 2) + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  if (blocks < 1) blocks = 1;
  k_make_n<T><<<(int)blocks, 256, (size_t)bt * bt * sizeof(T), s>>>(na, bt, S, lds, Linv, pivmark, act, Nbuf, X,
                                                                      ldx, tb, piv, pivorig, done);
  return cudaGetLastError();
}

// Stable removal of this round's pivots from the active list; one block.
constexpr int kCompactPer = 8;
__global__ void __launch_bounds__(1024)
    k_compact(int na, int bt, const int32_t* __restrict__ act_in, int32_t* __restrict__ act_out,
              int32_t* __restrict__ pivmark, const int32_t* __restrict__ piv, int64_t* __restrict__ J,
              int32_t* __restrict__ perm32, int64_t tb, double* pivots_out, const double* pivdiag,
              const int32_t* done) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  if (done != nullptr && *done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < bt; c += blockDim.x) {
    const int32_t j = act_in[piv[c]];
    J[tb + c] = j;
    perm32[tb + c] = j;
    if (pivots_out != nullptr) pivots_out[tb + c] = pivdiag[c];
  }
  if (tid == 0) s_base = 0;
  __syncthreads();
  // kCompactPer consecutive entries per thread (their loads all in flight), an
  // exclusive scan of the per-thread counts; the kept entries keep their order
  const int nw = blockDim.x >> 5;
  for (int start = 0; start < na; start += blockDim.x * kCompactPer) {
    const int i0 = start + tid * kCompactPer;
    int32_t a[kCompactPer], pm[kCompactPer];
#pragma unroll
    for (int u = 0; u < kCompactPer; ++u) {
      const bool in = i0 + u < na;
      pm[u] = in ? pivmark[i0 + u] : 1;
      a[u] = in ? act_in[i0 + u] : 0;
    }
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < kCompactPer; ++u) cnt += pm[u] == 0;
    int incl = cnt;  // inclusive scan over the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = lane < nw ? s_warp[lane] : 0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += t;
      }
      s_warp[lane] = v;  // inclusive prefix over the warps
    }
    __syncthreads();
    int pos = s_base + (warp == 0 ? 0 : s_warp[warp - 1]) + incl - cnt;
#pragma unroll
    for (int u = 0; u < kCompactPer; ++u) {
      if (pm[u] == 0) act_out[pos++] = a[u];
      if (i0 + u < na) pivmark[i0 + u] = 0;
    }
    __syncthreads();
    if (tid == 0) s_base += s_warp[nw - 1];
    __syncthreads();
  }
}

cudaError_t compact(int na, int bt, const int32_t* act_in, int32_t* act_out, int32_t* pivmark, const int32_t* piv,
                    int64_t* J, int32_t* perm32, int64_t tb, double* pivots_out, const double* pivdiag,
                    const int32_t* done, cudaStream_t s) {
  k_compact<<<1, 1024, 0, s>>>(na, bt, act_in, act_out, pivmark, piv, J, perm32, tb, pivots_out, pivdiag, done);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_finalize_x(int64_t k, const int32_t* __restrict__ perm32, T* __restrict__ X, int64_t ldx) {
  const int64_t total = k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / k, c = e - q * k;
    X[(int64_t)perm32[q] * ldx + c] = (c == q) ? T(1) : T(0);
  }
}

template <typename T>
cudaError_t finalize_x(int64_t k, const int32_t* perm32, T* X, int64_t ldx, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  int64_t blocks = (k * k + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_finalize_x<T><<<(int)blocks, 256, 0, s>>>(k, perm32, X, ldx);
  return cudaGetLastError();
}

// G (m x k, row-major) = A(:, J): the panel whose rows are LU-pivoted to pick the
// row skeletons of C = A(:, J).  Out-of-range column indices set kErrBadIndex.
template <typename T>
__global__ void k_gather_panel(const T* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                               const int64_t* __restrict__ J, int64_t k, T* __restrict__ G, DevState* st) {
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k, c = e - i * k;
    const int64_t j = J[c];
    if (j < 0 || j >= n) {
      atomicOr(&st->err, kErrBadIndex);
      G[e] = T(0);
    } else {
      G[e] = A[i + j * lda];
    }
  }
}

template <typename T>
cudaError_t gather_panel(const T* A, int64_t lda, int64_t m, int64_t n, const int64_t* J, int64_t k, T* G,
                         DevState* st, cudaStream_t s) {
  int64_t blocks = (m * k + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_gather_panel<T><<<(int)blocks, 256, 0, s>>>(A, lda, m, n, J, k, G, st);
  return cudaGetLastError();
}

// W (m x k, column-major, ldw) from the interpolation buffer X (k x m, column-major,
// ldx): W(i, c) = X(c, i).
template <typename T>
__global__ void k_transpose_w(const T* __restrict__ X, int64_t ldx, int64_t m, int64_t k, T* __restrict__ W,
                              int64_t ldw) {
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, i = e - c * m;  // consecutive threads write consecutive i
    W[i + c * ldw] = X[c + i * ldx];
  }
}

template <typename T>
cudaError_t transpose_w(const T* X, int64_t ldx, int64_t m, int64_t k, T* W, int64_t ldw, cudaStream_t s) {
  int64_t blocks = (m * k + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_transpose_w<T><<<(int)blocks, 256, 0, s>>>(X, ldx, m, k, W, ldw);
  return cudaGetLastError();
}

__global__ void k_init_state(DevState* st, int32_t* act, int32_t* pivmark, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    st->norm2_A = 0.0;
    st->est = 0.0;
    st->thr = 0.0;
    st->k_final = -1;
    st->k_pred = 0;
    st->done = 0;
    st->tol_not_met = 0;
    st->rounds = 0;
    st->err = 0u;
    st->zero_pivots = 0u;
    st->bar[0] = 0u;
    st->bar[1] = 0u;
    for (int q = 0; q < 12; ++q) (&st->pkey[0][0][0])[q] = 0ull;
  }
  if (i < n) {
    act[i] = (int32_t)i;
    pivmark[i] = 0;
  }
}

cudaError_t init_state(DevState* st, int32_t* act, int32_t* pivmark, int64_t n, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  k_init_state<<<(int)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(st, act, pivmark, n);
  return cudaGetLastError();
}

// ============================================================ instantiations
#define RID_INST(T)                                                                                         \
  template cudaError_t gemm_gather<T>(int, int, int, int, bool, Operand<T>, Operand<T>, int, EpiArgs<T>,    \
                                      const int32_t*, cudaStream_t);                                        \
  template cudaError_t gaussian_rows<T>(uint64_t, int64_t, int64_t, int64_t, T*, int64_t, const int32_t*,   \
                                        cudaStream_t);                                                      \
  template cudaError_t norm2_partial<T>(int64_t, int64_t, const T*, int64_t, double*, int, DevState*,       \
                                        cudaStream_t);                                                      \
  template cudaError_t splitk_reduce<T>(int64_t, int, int64_t, int, int64_t, const T*, T*, const int32_t*,  \
                                        cudaStream_t);                                                      \
  template cudaError_t splitk_reduce_ld<T>(int64_t, int, int64_t, int64_t, int, int64_t, const T*, T*,       \
                                           const int32_t*, cudaStream_t);                                   \
  template cudaError_t schur_finish<T>(int, int, const int32_t*, const T*, int64_t, int64_t, int, int64_t,  \
                                       const T*, T*, int64_t, double*, int, const int32_t*, cudaStream_t);  \
  template PanelCfg panel_config<T>(int, int, int);                                                         \
  template PanelCfg panel_layout<T>(int, int, int);                                                         \
  template cudaError_t panel_lupp<T>(const PanelCfg&, int, int, int, int, T*, int64_t, int32_t*, int32_t*,       \
                                     double*, double*, int32_t*, T*, DevState*, cudaStream_t);              \
  template cudaError_t linv<T>(int, const T*, int64_t, const int32_t*, T*, const int32_t*, cudaStream_t);   \
  template cudaError_t make_n<T>(int, int, const T*, int64_t, const T*, const int32_t*, const int32_t*, T*, \
                                 T*, int64_t, int64_t, const int32_t*, int32_t*, const int32_t*,            \
                                 cudaStream_t);                                                             \
  template cudaError_t finalize_x<T>(int64_t, const int32_t*, T*, int64_t, cudaStream_t);                  \
  template cudaError_t gather_panel<T>(const T*, int64_t, int64_t, int64_t, const int64_t*, int64_t, T*,     \
                                       DevState*, cudaStream_t);                                            \
  template cudaError_t transpose_w<T>(const T*, int64_t, int64_t, int64_t, T*, int64_t, cudaStream_t);

RID_INST(double)
RID_INST(float)
template cudaError_t gaussian_rows<__nv_bfloat16>(uint64_t, int64_t, int64_t, int64_t, __nv_bfloat16*, int64_t,
                                                  const int32_t*, cudaStream_t);
template cudaError_t gaussian_rows<__nv_fp8_e4m3>(uint64_t, int64_t, int64_t, int64_t, __nv_fp8_e4m3*, int64_t,
                                                  const int32_t*, cudaStream_t);
template cudaError_t norm2_partial<__nv_bfloat16>(int64_t, int64_t, const __nv_bfloat16*, int64_t, double*, int,
                                                  DevState*, cudaStream_t);

}  // namespace rid
