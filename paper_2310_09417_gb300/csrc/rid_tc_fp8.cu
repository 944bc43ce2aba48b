// rid_tc_fp8.cu -- the sketch Y = Omega A with A stored in FP8 E4M3 and one FP32
// scale per 128-row block of each column (mixed-precision sketch, Sec. 2.4 with
// the low-precision storage of the mixed-precision variant).
//
// A (m x n, column-major, E4M3) and Omega (rows x m, row-major, E4M3) are K-major
// (K = m) and go through TMA into 128-byte-swizzled shared memory: one stage is
// one 128-row scale block (128 E4M3 = one swizzle row).  tcgen05.mma kind::f8f6f4
// (E4M3 x E4M3, exact products, FP32 accumulation) sums one block into one of
// kAcc tensor-memory accumulators; the epilogue warps multiply each block sum by
// its column's scale and add it to FP32 registers, while the MMAs of the next
// blocks run into the other accumulators.
//
//   warp 0    one lane issues the TMA loads
//   warp 1    allocates tensor memory; one lane issues the MMAs
//   warps 2-  scaled accumulation and the FP32 rows of G (four warps for one
//             64-row block of Omega per CTA, eight for four blocks)
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "randid.h"
#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {
namespace tc8 {

using namespace tcx;

constexpr int kBM = 128;       // columns of A per tile (MMA M)
constexpr int kBN = 64;        // rows of Omega per sub-tile (one sketch block)
constexpr int kBK = 128;       // K per stage = one scale block
constexpr int kStages = 4;

// NT = 1: one 64-row block of Omega per CTA, four accumulators of 64 columns (256
// tensor-memory columns: two CTAs share an SM), 4 stages of 24 KB, four epilogue
// warps.  NT = 4: four blocks per CTA (a pass of several blocks reads each tile of
// A once per CTA, not once per block) with one MMA of N = 256 per K step, two
// accumulators of 256 columns (the SM's 512), 4 stages of 48 KB, eight epilogue
// warps of 128 columns each.
template <int NT>
struct Cfg {
  static constexpr int kAcc = NT == 1 ? 4 : 2;
  static constexpr int kCols = NT * kBN;  // columns of one accumulator = MMA N
  static constexpr int kEpiWarps = NT == 1 ? 4 : 8;
  static constexpr int kWarpCols = kCols * 4 / kEpiWarps;  // columns an epilogue warp drains
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static constexpr int kMinBlocks = NT == 1 ? 2 : 1;
  static constexpr uint32_t kTmemCols = kAcc * kCols;
};

template <int NT>
struct Smem {
  alignas(1024) uint8_t a[kStages][kBM * kBK];       // 16 KB per stage
  alignas(1024) uint8_t w[kStages][NT * kBN * kBK];  // 8 KB per block per stage
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[Cfg<NT>::kAcc];   // the MMAs of a scale block landed in accumulator a
  uint64_t acc_empty[Cfg<NT>::kAcc];  // the epilogue has read accumulator a
  uint64_t drain;
  uint32_t tmem_base;
};

// Grid: x = tiles of A's columns, y = groups of NT 64-row blocks of Omega, z = K
// splits of kchunk (a multiple of kBK).  scale: column-major nbs x n block scales.
// out: FP32 partial (n x rows, row stride out_ld) of split blockIdx.z.  Every entry
// gets the same sums (block sums in K order, scaled and added in block order)
// whatever NT is.
template <int NT>
__global__ void __launch_bounds__(Cfg<NT>::kThreads, Cfg<NT>::kMinBlocks)
    k_sketch_tc_fp8(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
                    const float* __restrict__ scale, int64_t nbs, int n, int rows, int K, int kchunk,
                    float* __restrict__ out, int64_t out_ld, int64_t zstride, DevState* st, const int32_t* done) {
  using C = Cfg<NT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem<NT>& sm = *reinterpret_cast<Smem<NT>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.y * C::kCols;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nkb = (kend - kbeg + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < C::kAcc; ++a) {
      mbar_init(&sm.acc_full[a], 1);
      mbar_init(&sm.acc_empty[a], C::kEpiWarps);  // one arrival per epilogue warp
    }
    mbar_init(&sm.drain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(&sm.tmem_base, C::kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(&sm.empty[s], ((kb / kStages) + 1) & 1, st)) break;
      mbar_expect_tx(&sm.full[s], (kBM + C::kCols) * kBK);
      const int k0 = kbeg + kb * kBK;
      tma_load_2d(sm.a[s], &map_a, &sm.full[s], k0, m0);
      tma_load_2d(sm.w[s], &map_w, &sm.full[s], k0, n0);  // one box of NT x 64 rows (at most 256)
      issued = kb + 1;
    }
    for (int kb = issued - kStages < 0 ? 0 : issued - kStages; kb < issued; ++kb)
      mbar_wait_drain(&sm.full[kb % kStages], (kb / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: scale block kb -> accumulator kb % kAcc
    constexpr uint32_t idesc = idesc_e4m3(kBM, C::kCols);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages, a = kb % C::kAcc;
      if (kb >= C::kAcc && !mbar_wait(&sm.acc_empty[a], ((kb / C::kAcc) + 1) & 1, st)) break;
      if (!mbar_wait(&sm.full[s], (kb / kStages) & 1, st)) break;
      fence_after_sync();
      const uint64_t da = desc_sw128(sm.a[s]);
      const uint64_t dw = desc_sw128(sm.w[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 32; ++kk)  // 32 E4M3 = 32 bytes per MMA
        mma_e4m3(tmem + a * C::kCols, da + 2 * kk, dw + 2 * kk, idesc, kk != 0);
      mma_commit(&sm.empty[s]);
      mma_commit(&sm.acc_full[a]);
    }
    mma_commit(&sm.drain);  // every MMA issued completes before tensor memory is freed
    mbar_wait_drain(&sm.drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: scaled FP32 accumulation of the block sums
    const int quarter = warp & 3;          // TMEM lanes this warp may read
    const int col0 = ((warp - 2) >> 2) * C::kWarpCols;  // its columns of the accumulator
    const int row = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + col0;
    const float* sc = scale + static_cast<int64_t>(row < n ? row : 0) * nbs + kbeg / kBK;
    float acc[C::kWarpCols];
#pragma unroll
    for (int c = 0; c < C::kWarpCols; ++c) acc[c] = 0.f;
    bool ok = true;
    float s_next = __ldg(sc);
    for (int kb = 0; kb < nkb; ++kb) {
      const int a = kb % C::kAcc;
      const float s_kb = s_next;
      if (kb + 1 < nkb) s_next = __ldg(sc + kb + 1);
      if (!mbar_wait(&sm.acc_full[a], (kb / C::kAcc) & 1, st)) {
        ok = false;
        break;
      }
      fence_after_sync();
#pragma unroll
      for (int cb = 0; cb < C::kWarpCols; cb += 32) {  // 32 columns per wait on tensor memory
        float v[32];
        tmem_ld32(lane_base + a * C::kCols + cb, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[cb + i] = fmaf(v[i], s_kb, acc[cb + i]);
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[a]);
    }
    if (ok && row < n) {
      float* o = out + blockIdx.z * zstride + static_cast<int64_t>(row) * out_ld + n0 + col0;
      const int lim = rows - n0 - col0;
#pragma unroll
      for (int c = 0; c < C::kWarpCols; ++c)
        if (c < lim) o[c] = acc[c];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, C::kTmemCols);
  }
}

// ------------------------------------------------------------------ ||A||_F^2 and finiteness
// One block per column at a time: sum of (fp8(i,j) * scale(i/128, j))^2 in FP64.
__global__ void k_norm2_fp8(int64_t m, int64_t n, const uint8_t* __restrict__ A, int64_t lda,
                            const float* __restrict__ scale, int64_t nbs, double* part, DevState* st) {
  double acc = 0.0;
  bool finite = true;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const uint8_t* a = A + j * lda;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      __nv_fp8_e4m3 q;
      q.__x = a[i];
      const double s = (double)scale[j * nbs + i / kBK];
      const double v = (double)static_cast<float>(q) * s;
      finite = finite && isfinite(v);
      acc += v * v;
    }
  }
  if (!finite) atomicOr(&st->err, kErrNonFinite);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// ||A||_F^2 with 16 E4M3 values per load (columns 16-byte aligned: lda a multiple of
// 16).  A vector's 16 values share one block scale; their squares are exact in
// FP32 (at most 8 significant bits, between 2^-18 and 448^2) and are summed in
// float-float (sq_twosum), then scaled by scale^2 and added in FP64: a few FP64
// operations per 16 values instead of several per value.
__global__ void k_norm2_fp8v(int64_t m, int64_t n, const uint8_t* __restrict__ A, int64_t lda,
                             const float* __restrict__ scale, int64_t nbs, double* part, DevState* st) {
  double acc = 0.0;
  bool finite = true;
  const int64_t nv = (m + 15) / 16;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const uint4* a = reinterpret_cast<const uint4*>(A + j * lda);
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
      const uint4 w = __ldg(a + v);
      uint32_t ws[4] = {w.x, w.y, w.z, w.w};
      const int64_t left = m - 16 * v;
      if (left < 16) {  // the last vector of the column: rows past m are ignored
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (4 * q + k >= left) ws[q] &= ~(0xFFu << (8 * k));
      }
      const float sc = scale[j * nbs + (16 * v) / kBK];
      if (!isfinite(sc)) finite = false;
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (__vcmpeq4(ws[q] & 0x7F7F7F7Fu, 0x7F7F7F7Fu) != 0u) finite = false;  // E4M3 NaN
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const __half2_raw hr =
              __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((ws[q] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
          const float2 f = __half22float2(__half2(hr));
          sq_twosum(__fmul_rn(f.x, f.x), hi, lo);
          sq_twosum(__fmul_rn(f.y, f.y), hi, lo);
        }
      }
      const double sd = (double)sc;
      acc += ((double)hi + (double)lo) * (sd * sd);
    }
  }
  if (!finite) atomicOr(&st->err, kErrNonFinite);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// ------------------------------------------------------------------ quantisation
template <typename T>
__device__ __forceinline__ float as_float(T x) {
  return static_cast<float>(x);
}
template <>
__device__ __forceinline__ float as_float<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// One warp per (128-row block, column): amax -> scale -> E4M3 (round to nearest
// even, saturating at +-448).  FP64 input is divided in FP64, FP32/BF16 in FP32.
template <typename T>
__global__ void k_quantize_fp8(int64_t m, int64_t n, const T* __restrict__ A, int64_t lda, uint8_t* __restrict__ Q,
                               int64_t ldq, float* __restrict__ scale, int64_t nbs, int pow2) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t blk = wid; blk < nbs * n; blk += nw) {
    const int64_t j = blk / nbs, kb = blk - j * nbs;
    const int64_t i0 = kb * kBK, i1 = min(m, i0 + kBK);
    const T* a = A + j * lda;
    float amax = 0.f;
    bool nan_seen = false;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
      const float v = as_float(a[i]);
      nan_seen = nan_seen || isnan(v);
      amax = fmaxf(amax, fabsf(v));
    }
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    nan_seen = __any_sync(0xffffffffu, nan_seen);
    float s = 1.f;
    if (nan_seen) {
      s = __int_as_float(0x7fc00000);  // a NaN scale marks the block non-finite
    } else if (amax > 0.f) {
      s = amax / 448.f;
      if (pow2) {  // the power of two >= amax / 448
        int e;
        const float f = frexpf(s, &e);  // s = f 2^e, 0.5 <= f < 1
        s = ldexpf(1.f, f == 0.5f ? e - 1 : e);
      }
    }
    if (lane == 0) scale[j * nbs + kb] = s;
    uint8_t* q = Q + j * ldq;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
      __nv_fp8_e4m3 v;
      if constexpr (sizeof(T) == 8)
        v.__x = __nv_cvt_double_to_fp8(static_cast<double>(a[i]) / static_cast<double>(s), __NV_SATFINITE, __NV_E4M3);
      else
        v.__x = __nv_cvt_float_to_fp8(as_float(a[i]) / s, __NV_SATFINITE, __NV_E4M3);
      q[i] = v.__x;
    }
  }
}

bool make_map_u8(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t ld, int box_rows) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc8

bool tc_fp8_supported(const void* A, int64_t lda, const void* W, int64_t ldw) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(A), w = reinterpret_cast<uintptr_t>(W);
  return (a % 16) == 0 && (w % 16) == 0 && (lda % 16) == 0 && (ldw % 16) == 0 && tensor_map_encoder() != nullptr;
}

int tc_fp8_splits(int64_t m, int64_t n, int64_t rows, int sms) {
  const int64_t tiles = ((n + tc8::kBM - 1) / tc8::kBM) * ((rows + tc8::kBN - 1) / tc8::kBN);
  int64_t s = (8 * (int64_t)sms + tiles - 1) / tiles;           // about eight waves of one CTA per SM
  const int64_t kmax = (m + 8 * tc8::kBK - 1) / (8 * tc8::kBK);  // >= 8 K-stages per CTA
  if (s > kmax) s = kmax;
  if (s > 32) s = 32;
  return (int)(s < 1 ? 1 : s);
}

int tc_fp8_effective_splits(int64_t m, int splits) {
  int64_t kchunk = (m + splits - 1) / splits;
  kchunk = (kchunk + tc8::kBK - 1) / tc8::kBK * tc8::kBK;
  return (int)((m + kchunk - 1) / kchunk);
}

template <int NT>
static cudaError_t launch_fp8(const CUtensorMap& ma, const CUtensorMap& mw, const float* scale, int64_t nbs,
                              int64_t m, int64_t n, int64_t rows, int64_t kchunk, int nz, float* out, int64_t out_ld,
                              int64_t zstride, DevState* st, const int32_t* done, cudaStream_t s) {
  static_assert(sizeof(tc8::Smem<NT>) + 1024 <= 232448, "shared memory of k_sketch_tc_fp8 exceeds 227 KB");
  const size_t smem = sizeof(tc8::Smem<NT>) + 1024;
  static SmemLimit lim;
  cudaError_t e = raise_smem(tc8::k_sketch_tc_fp8<NT>, smem, lim);
  if (e != cudaSuccess) return e;
  const int64_t ytiles = (rows + tc8::Cfg<NT>::kCols - 1) / tc8::Cfg<NT>::kCols;
  if (ytiles > 65535 || nz > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((n + tc8::kBM - 1) / tc8::kBM), (unsigned)ytiles, (unsigned)nz);
  tc8::k_sketch_tc_fp8<NT><<<grid, tc8::Cfg<NT>::kThreads, smem, s>>>(ma, mw, scale, nbs, (int)n, (int)rows, (int)m,
                                                                     (int)kchunk, out, out_ld, zstride, st, done);
  return cudaGetLastError();
}

cudaError_t tc_sketch_fp8(const void* A, int64_t lda, int64_t m, int64_t n, const float* scale, const void* W,
                          int64_t ldw, int64_t rows, float* out, int64_t out_ld, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s) {
  // a pass of several blocks: four 64-row blocks of Omega per CTA
  const int nt = rows > tc8::kBN ? 4 : 1;
  CUtensorMap ma, mw;
  if (!tc8::make_map_u8(&ma, A, m, n, lda, tc8::kBM)) return cudaErrorInvalidValue;
  if (!tc8::make_map_u8(&mw, W, m, rows, ldw, nt * tc8::kBN)) return cudaErrorInvalidValue;
  int64_t kchunk = (m + splits - 1) / splits;
  kchunk = (kchunk + tc8::kBK - 1) / tc8::kBK * tc8::kBK;
  const int nz = (int)((m + kchunk - 1) / kchunk);
  if (nz != splits) return cudaErrorInvalidValue;  // the reduction reads exactly `splits` partials
  const int64_t nbs = (m + tc8::kBK - 1) / tc8::kBK;
  if (nt == 4) return launch_fp8<4>(ma, mw, scale, nbs, m, n, rows, kchunk, nz, out, out_ld, zstride, st, done, s);
  return launch_fp8<1>(ma, mw, scale, nbs, m, n, rows, kchunk, nz, out, out_ld, zstride, st, done, s);
}

cudaError_t norm2_fp8(int64_t m, int64_t n, const void* A, int64_t lda, const float* scale, double* part, int nparts,
                      DevState* st, cudaStream_t s) {
  const int64_t nbs = (m + tc8::kBK - 1) / tc8::kBK;
  if ((lda % 16) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0)
    tc8::k_norm2_fp8v<<<nparts, 256, 0, s>>>(m, n, static_cast<const uint8_t*>(A), lda, scale, nbs, part, st);
  else
    tc8::k_norm2_fp8<<<nparts, 256, 0, s>>>(m, n, static_cast<const uint8_t*>(A), lda, scale, nbs, part, st);
  return cudaGetLastError();
}

cudaError_t quantize_fp8(int dtype, int64_t m, int64_t n, const void* A, int64_t lda, void* Q, int64_t ldq,
                         float* scale, int pow2, cudaStream_t s) {
  const int64_t nbs = (m + tc8::kBK - 1) / tc8::kBK;
  int64_t blocks = (nbs * n * 32 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  uint8_t* q = static_cast<uint8_t*>(Q);
  if (dtype == ID_F64)
    tc8::k_quantize_fp8<double><<<(int)blocks, 256, 0, s>>>(m, n, static_cast<const double*>(A), lda, q, ldq, scale,
                                                           nbs, pow2);
  else if (dtype == ID_F32)
    tc8::k_quantize_fp8<float><<<(int)blocks, 256, 0, s>>>(m, n, static_cast<const float*>(A), lda, q, ldq, scale,
                                                          nbs, pow2);
  else
    tc8::k_quantize_fp8<__nv_bfloat16><<<(int)blocks, 256, 0, s>>>(m, n, static_cast<const __nv_bfloat16*>(A), lda,
                                                                   q, ldq, scale, nbs, pow2);
  return cudaGetLastError();
}

}  // namespace rid
