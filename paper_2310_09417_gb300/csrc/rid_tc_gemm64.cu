// rid_tc_gemm64.cu -- GEMMs on the BF16 tensor cores by exact digit slicing:
//   * k_gemm_emu<7, double> (FP64 accuracy): the Schur complement of the
//     FP64-emulated path, P = T(act, 0:K) G(perm, cols) (Algorithm 1's Schur step in
//     the T = L2 L1^{-1} form), written as FP64 split-K partials for the Schur finish;
//   * k_sketch_f32emu (FP32 accuracy, 3 digits per operand): the sketch Y = Omega A
//     of an FP32 matrix (Sec. 2.4), FP32 split-K partials; A is sliced once per
//     call, Omega once per pass (described at the kernel).
//
// Both operands change every round, so both are sliced here, with integer
// operations on the FP64 bit patterns (GB300 issues about two FP64
// instructions per clock per SM):
//   * A (M x K, rows gathered): per row an exponent e_m (max_k |A| < 2^e_m) and
//     the 56-bit fixed-point value F = round(A 2^(55 - e_m)) written as seven
//     balanced 8-bit digits, A / 2^(e_m+1) = sum_s d_s 2^(-8(s+1)), |d_s| <= 128.
//   * B (K x N, rows gathered): the same per column, exponent f_n.
// The products of equal weight 2^(-8(g+2)), g = s + t <= 6, share FP32 group g in
// tensor memory.  Over a chunk of 128 K a group sums at most 7 pairs x 128 terms
// of magnitude <= 2^14 (< 2^24): exact.  Epilogue warps fold each chunk into two
// int64 accumulators per entry while the MMAs of the next chunk run into the
// other half of tensor memory; the end value is assembled as an FP64 with
// integer operations.  Dropped pairs (g >= 7) and the digit rounding bound each
// entry's error by about 2^-46 K max|A(m,:)| max|B(:,n)|.
//
//   warp 0    TMA: B's 7 digit tiles per K step (two buffers), then A's digit
//             tiles one slice per stage
//   warp 1    tensor memory; per (K step, slice s) 4 MMAs M=128 N=32 (7 - s) K=16 against
//             B's planes stacked along N
//   warps 2-5 epilogue
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {
namespace tcg {

using namespace tcx;

constexpr int kBM = 128;      // rows of A per tile
constexpr int kBK = 64;       // K per step
constexpr int kThreads = 192;
// Exact chunk: a group sums at most KD pairs of products <= 2^14, so fewer than
// 2^24 / (KD 2^14) = 1024 / KD terms: 128 K for KD = 7.
// Columns of B per tile: two accumulator sets of KD groups fit the 512
// tensor-memory columns.
template <int KD>
struct Cfg {
  static constexpr int kBN = 32;
  static constexpr int kChunkStepsC = (1024 / KD) / kBK;
  static constexpr int kAStages = 6 / kChunkStepsC;  // stages of A in flight, one (chunk, slice) each
  static constexpr int kChunkSteps = (1024 / KD) / kBK;
  static constexpr int kGroupCols = KD * kBN;  // tensor-memory columns per accumulator set
  static constexpr uint32_t kTmemCols = 2 * kGroupCols <= 256 ? 256 : 512;
};

// Stage order (chunk c, slice s): a stage holds one digit plane of A's rows at every
// K step of the chunk (one barrier per 16 KB x chunk steps: a TMA stream with one
// barrier per 16 KB box runs well below HBM bandwidth at one CTA per SM); B's digits
// of a whole chunk stay resident (two chunk buffers).
template <int KD>
struct Smem {
  alignas(1024) __nv_bfloat16 a[Cfg<KD>::kAStages][Cfg<KD>::kChunkStepsC][kBM * kBK];  // 16 KB per K step
  alignas(1024) __nv_bfloat16 b[2][Cfg<KD>::kChunkSteps][KD][Cfg<KD>::kBN * kBK];      // 4 KB each
  uint64_t a_full[Cfg<KD>::kAStages];
  uint64_t a_empty[Cfg<KD>::kAStages];
  uint64_t b_full[2];
  uint64_t b_empty[2];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
};
static_assert(sizeof(Smem<7>) + 1024 <= 232448, "shared memory of k_gemm_emu exceeds 227 KB");


// Grid: x = column tiles of B (fastest: CTAs sharing an A tile run together), y = row
// tiles of A, z = K splits of kchunk (a multiple of 128).  out[z]: FP64 partial
// (M x N, row stride ldo).
template <int KD, typename TOut>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_emu(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M, int N,
               int K, int kchunk, const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
               TOut* __restrict__ out, int64_t ldo, int64_t zstride, DevState* st, const int32_t* done) {
  constexpr int kD = KD;
  constexpr int kBN = Cfg<KD>::kBN;
  constexpr int kAStages = Cfg<KD>::kAStages;
  constexpr int kChunkSteps = Cfg<KD>::kChunkSteps;
  constexpr int kGroupCols = Cfg<KD>::kGroupCols;
  constexpr uint32_t kTmemCols = Cfg<KD>::kTmemCols;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem<KD>& sm = *reinterpret_cast<Smem<KD>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kBN;
  const int m0 = blockIdx.y * kBM;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nsteps = (kend - kbeg + kBK - 1) / kBK;
  const int nchunks = (nsteps + kChunkSteps - 1) / kChunkSteps;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kAStages; ++i) {
      mbar_init(&sm.a_full[i], 1);
      mbar_init(&sm.a_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.b_full[i], 1);
      mbar_init(&sm.b_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.acc_full[i], 1);
      mbar_init(&sm.acc_empty[i], 4);
    }
    mbar_init(&sm.drain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(&sm.tmem_base, kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: per chunk, B's digits of all its K steps, then A's
    // slices in the order (slice, K step)
    int ai = 0, cb = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int bb = c & 1;
      if (c >= 2 && !mbar_wait(&sm.b_empty[bb], ((c >> 1) + 1) & 1, st)) break;
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      mbar_expect_tx(&sm.b_full[bb], steps_c * kD * kBN * kBK * 2);
      for (int jj = 0; jj < steps_c; ++jj)
        for (int t = 0; t < kD; ++t)
          tma_load_3d(sm.b[bb][jj][t], &map_b, &sm.b_full[bb], kbeg + (c * kChunkSteps + jj) * kBK, n0, t);
      cb = c + 1;
      for (int s = 0; s < kD && ok; ++s, ++ai) {
        const int st_ = ai % kAStages;
        if (ai >= kAStages && !mbar_wait(&sm.a_empty[st_], ((ai / kAStages) + 1) & 1, st)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&sm.a_full[st_], steps_c * kBM * kBK * 2);
        for (int jj = 0; jj < steps_c; ++jj)
          tma_load_3d(sm.a[st_][jj], &map_a, &sm.a_full[st_], kbeg + (c * kChunkSteps + jj) * kBK, m0, s);
      }
    }
    // copies still in flight land before the CTA may exit
    for (int i = ai - kAStages < 0 ? 0 : ai - kAStages; i < ai; ++i)
      mbar_wait_drain(&sm.a_full[i % kAStages], (i / kAStages) & 1);
    for (int c = cb - 2 < 0 ? 0 : cb - 2; c < cb; ++c) mbar_wait_drain(&sm.b_full[c & 1], (c >> 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int ai = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int u = c & 1;  // accumulator set and B chunk buffer
      if (c >= 2 && !mbar_wait(&sm.acc_empty[u], ((c >> 1) + 1) & 1, st)) break;
      if (!mbar_wait(&sm.b_full[u], (c >> 1) & 1, st)) break;
      fence_after_sync();
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int s = 0; s < kD && ok; ++s, ++ai) {
        const int st_ = ai % kAStages;
        if (!mbar_wait(&sm.a_full[st_], (ai / kAStages) & 1, st)) {
          ok = false;
          break;
        }
        fence_after_sync();
        for (int jj = 0; jj < steps_c; ++jj) {
          const uint64_t da = desc_sw128(sm.a[st_][jj]);
          // B's planes 0 .. KD-1-s lie back to back: one MMA with N = kBN (KD - s) writes
          // groups s .. KD-1; every group is first written at slice 0, K step 0 of the chunk
          const uint64_t db = desc_sw128(sm.b[u][jj][0]);
          const uint32_t dst = tmem + u * kGroupCols + s * kBN;
          const uint32_t idn = idesc_bf16(kBM, kBN * (kD - s));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            mma_bf16(dst, da + 2 * kk, db + 2 * kk, idn, (jj > 0 || s > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&sm.a_empty[st_]);
      }
      if (ok) {
        mma_commit(&sm.b_empty[u]);
        mma_commit(&sm.acc_full[u]);
      }
    }
    mma_commit(&sm.drain);
    mbar_wait_drain(&sm.drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: exact folding of each chunk into int64
    const int quarter = warp & 3;
    const int m = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
    long long hi[kBN], lo[kBN];
#pragma unroll
    for (int i = 0; i < kBN; ++i) hi[i] = lo[i] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int u = c & 1;
      if (!mbar_wait(&sm.acc_full[u], (c >> 1) & 1, st)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const uint32_t base = lane_base + u * kGroupCols;
#pragma unroll
      for (int cb = 0; cb < kBN; cb += 16) {
        float v[16];
        // groups 0..2 into hi with weights 2^(8(2-g)), groups 3..6 into lo with 2^(8(6-g))
        tmem_ld16(base + 0 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<16>(hi[cb + i], v[i]);
        tmem_ld16(base + 1 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<8>(hi[cb + i], v[i]);
        tmem_ld16(base + 2 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<0>(hi[cb + i], v[i]);
        if constexpr (KD > 3) {
          tmem_ld16(base + 3 * kBN + cb, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) add_scaled<24>(lo[cb + i], v[i]);
          tmem_ld16(base + 4 * kBN + cb, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) add_scaled<16>(lo[cb + i], v[i]);
          tmem_ld16(base + 5 * kBN + cb, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) add_scaled<8>(lo[cb + i], v[i]);
          tmem_ld16(base + 6 * kBN + cb, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) add_scaled<0>(lo[cb + i], v[i]);
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[u]);
    }
    if (ok && m < M) {
      const int em = ea[m];
      TOut* o = out + blockIdx.z * zstride + (int64_t)m * ldo;
#pragma unroll
      for (int i = 0; i < kBN; ++i)
        if (n0 + i < N) o[n0 + i] = (TOut)fixed_to_double(hi[i], lo[i], em + eb[n0 + i] + 2 - 64);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------------ slicing by integer operations
// A rows: row r of the result is src[idx[r] * lds + k] for k < K (idx null: r).
// One warp per row: the row's largest |x| (integer comparison of bit patterns),
// then the digits D[s][r][k] (row stride Kp), zero for K <= k < Kq.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float x) {
  return (unsigned long long)((unsigned int)__float_as_int(x) & 0x7FFFFFFFu);
}
__device__ __forceinline__ int exp_above(unsigned long long b, double) { return exp_above_f64bits(b); }
__device__ __forceinline__ int exp_above(unsigned long long b, float) { return exp_above_f32bits((unsigned int)b); }

template <typename T, int KD>
__global__ void k_slice_rows(int M, int K, int Kq, int64_t Kp, const T* __restrict__ src, int64_t lds,
                             const int32_t* __restrict__ idx, __nv_bfloat16* __restrict__ D, int64_t plane,
                             int32_t* __restrict__ ex, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < M; r += nw) {
    const T* row = src + (int64_t)(idx ? idx[r] : r) * lds;
    // four consecutive k per lane: a warp covers 128 elements per step
    unsigned long long mx = 0;
    for (int k = 4 * lane; k < K; k += 128) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (k + e < K) mx = max(mx, abs_bits(row[k + e]));
    }
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const int e = exp_above(mx, T(0));
    if (lane == 0) ex[r] = e;
    for (int k = 4 * lane; k < Kq; k += 128) {  // Kq is a multiple of 64
      long long F[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) F[q] = k + q < K ? fixed_of<KD>(row[k + q], e) : 0ll;
      write_digits4<KD>(F, D + r * Kp + k, plane);
    }
  }
}

// The same for few, long rows: the row maxima by atomics over blocks of K (rowmax
// starts at 0), then one thread per element.
template <typename T>
__global__ void k_rows_max(int M, int K, const T* __restrict__ src, int64_t lds,
                           unsigned long long* __restrict__ rowmax, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int r = blockIdx.y;
  unsigned long long mx = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, abs_bits(src[(int64_t)r * lds + k]));
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx != 0) atomicMax(&rowmax[r], mx);
}
template <typename T, int KD>
__global__ void k_rows_digits(int M, int K, int Kq, int64_t Kp, const T* __restrict__ src, int64_t lds,
                              const unsigned long long* __restrict__ rowmax, __nv_bfloat16* __restrict__ D,
                              int64_t plane, int32_t* __restrict__ ex, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int r = blockIdx.y;
  const int e = exp_above(rowmax[r], T(0));
  if (blockIdx.x == 0 && threadIdx.x == 0) ex[r] = e;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Kq; k += (int64_t)gridDim.x * blockDim.x)
    write_digits<KD>(k < K ? fixed_of<KD>(src[(int64_t)r * lds + k], e) : 0ll, D + (int64_t)r * Kp + k, plane);
}

// B (K x N): element (k, n) = src[idx[k] * lds + off + n].  First the largest
// |B(:, n)| bit pattern per column (blocks over K, n fastest for coalesced reads,
// atomicMax into colmax, which starts at 0) ...
constexpr int kColTile = 64;
template <typename T>
__global__ void k_col_max(int K, int N, const T* __restrict__ src, int64_t lds, int64_t off,
                          const int32_t* __restrict__ idx, unsigned long long* __restrict__ colmax,
                          const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ unsigned long long red[256];
  const int n = threadIdx.x % kColTile, kl = threadIdx.x / kColTile;  // 4 rows per pass
  unsigned long long mx = 0;
  if (n < N)
    for (int k = blockIdx.x * kColTile + kl; k < min(K, (int)(blockIdx.x + 1) * kColTile); k += 4)
      mx = max(mx, abs_bits(src[(int64_t)idx[k] * lds + off + n]));
  red[threadIdx.x] = mx;
  __syncthreads();
  if (kl == 0 && n < N) {
    for (int q = 1; q < 4; ++q) mx = max(mx, red[q * kColTile + n]);
    if (mx != 0) atomicMax(&colmax[n], mx);
  }
}

// ... then the digits, one block per 64 rows of K: the tile goes through shared
// memory so that digit writes D[t][n][k] are contiguous in k.
template <typename T, int KD>
__global__ void k_col_digits(int K, int N, int Kp, const T* __restrict__ src, int64_t lds, int64_t off,
                             const int32_t* __restrict__ idx, const unsigned long long* __restrict__ colmax,
                             __nv_bfloat16* __restrict__ D, int64_t plane, int32_t* __restrict__ ex,
                             const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ T tile[kColTile][kColTile + 1];
  const int k0 = blockIdx.x * kColTile;
  for (int e = threadIdx.x; e < kColTile * kColTile; e += blockDim.x) {
    const int kl = e / kColTile, n = e % kColTile;
    const int k = k0 + kl;
    tile[kl][n] = (k < K && n < N) ? src[(int64_t)idx[k] * lds + off + n] : T(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kColTile * kColTile; e += blockDim.x) {
    const int n = e / kColTile, kl = e % kColTile;  // k fastest: contiguous writes
    const int k = k0 + kl;
    if (n < N && k < Kp) {
      const int en = exp_above(colmax[n], T(0));
      write_digits<KD>(k < K ? fixed_of<KD>(tile[kl][n], en) : 0ll, D + (int64_t)n * Kp + k, plane);
      if (blockIdx.x == 0 && kl == 0) ex[n] = en;
    }
  }
}

bool make_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int box_rows, int planes) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One launch of the digit GEMM over pre-sliced operands: A digits (KD planes of arows x
// Kp), B digits (KD planes of brows x Kp), both K-major.
template <int KD, typename TOut>
cudaError_t launch(int M, int N, int K, int64_t Kp, const void* adig, int64_t arows, const int32_t* aexp,
                   const void* bdig, int64_t brows, const int32_t* bexp, TOut* out, int64_t ldo, int64_t zstride,
                   int splits, DevState* st, const int32_t* done, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, adig, Kp, arows, kBM, KD)) return cudaErrorInvalidValue;
  if (!make_map(&mb, bdig, Kp, brows, Cfg<KD>::kBN, KD)) return cudaErrorInvalidValue;
  constexpr int chunk = Cfg<KD>::kChunkSteps * kBK;
  const int64_t chunks = (K + chunk - 1) / chunk;
  const int64_t per = (chunks + splits - 1) / splits;
  const int kchunk = (int)(per * chunk);
  const int nz = (int)((K + kchunk - 1) / kchunk);
  if (nz != splits) return cudaErrorInvalidValue;  // the reduction reads exactly `splits` partials
  const size_t smem = sizeof(Smem<KD>) + 1024;
  static SmemLimit lim;
  cudaError_t e = raise_smem(k_gemm_emu<KD, TOut>, smem, lim);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((N + Cfg<KD>::kBN - 1) / Cfg<KD>::kBN), (unsigned)((M + kBM - 1) / kBM), (unsigned)nz);
  k_gemm_emu<KD, TOut><<<grid, kThreads, smem, s>>>(ma, mb, M, N, K, kchunk, aexp, bexp, out, ldo, zstride, st, done);
  return cudaGetLastError();
}

// Split count over exact chunks.  One CTA per SM holds a (tile, split); its time is
// about its chunks plus a fixed cost, so a launch takes waves x (chunks per split +
// c0); the count (at most `cap`) minimising that is taken.
template <int KD>
int splits_for(int64_t M, int64_t N, int64_t K, int sms, int cap) {
  const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + Cfg<KD>::kBN - 1) / Cfg<KD>::kBN);
  constexpr int chunk = Cfg<KD>::kChunkSteps * kBK;
  const int64_t chunks = (K + chunk - 1) / chunk;
  int best = 1;
  double best_t = 1e300;
  for (int64_t s = 1; s <= cap && s <= chunks; ++s) {
    const int64_t per = (chunks + s - 1) / s;
    const int64_t eff = (chunks + per - 1) / per;
    if (eff != s) continue;
    const int64_t waves = (tiles * eff + sms - 1) / sms;
    const double t = (double)waves * ((double)per + 0.5) + 0.02 * (double)eff;
    if (t < best_t) {
      best_t = t;
      best = (int)eff;
    }
  }
  return best;
}

// ------------------------------------------------------------------ FP32-accurate sketch
// (W A)^T for an FP32 A: A's columns and W's rows as 3 balanced 8-bit digit planes
// each (per-row exponents).  A stage holds one K step of 64 for both operands, all
// planes: A 3 x 128 rows, W 3 x 64 rows stacked along N.  Per K step of 16 and A's
// plane s one MMA (M = 128, N = 64 (3 - s)) against W's planes 0 .. 2-s writes groups
// s .. 2 (group g = s + t collects the products of weight 2^(-8(g+2))).  A chunk of 5
// K steps (320 K) keeps every group below 3 x 320 x 2^14 < 2^24: exact in FP32.  Two
// accumulator sets (2 x 3 groups x 64 columns) let the epilogue fold chunk c into
// int64 while the MMAs of chunk c+1 run.
namespace f32s {
constexpr int kBM = 128, kBN = 64, kBK = 64, kD = 3;
constexpr int kStages = 3;
constexpr int kChunkSteps = 5;
constexpr int kSet = kD * kBN;     // tensor-memory columns of one accumulator set
constexpr int kEpiWarps = 8;       // two per lane quarter, 32 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;

struct Smem {
  alignas(1024) __nv_bfloat16 a[kStages][kD][kBM * kBK];  // 3 x 16 KB per stage
  alignas(1024) __nv_bfloat16 w[kStages][kD][kBN * kBK];  // 3 x 8 KB per stage, back to back
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
};
static_assert(sizeof(Smem) + 1024 <= 232448, "shared memory of k_sketch_f32emu exceeds 227 KB");

// Grid: x = tiles of A's columns (M), y = tiles of W's rows (N), z = K splits of kchunk
// (a multiple of the chunk).  out[z]: FP32 partial (M x N, row stride ldo).
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_f32emu(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w, int M,
                    int N, int K, int kchunk, const int32_t* __restrict__ ea, const int32_t* __restrict__ ew,
                    float* __restrict__ out, int64_t ldo, int64_t zstride, DevState* st, const int32_t* done) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nsteps = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;
  const int nchunks = (nsteps + kChunkSteps - 1) / kChunkSteps;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sm.full[i], 1);
      mbar_init(&sm.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.acc_full[i], 1);
      mbar_init(&sm.acc_empty[i], kEpiWarps);
    }
    mbar_init(&sm.drain, 1);
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(&sm.tmem_base, 512);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: one stage per K step, every plane of both operands
    int it = 0;
    for (; it < nsteps; ++it) {
      const int b = it % kStages;
      if (it >= kStages && !mbar_wait(&sm.empty[b], ((it / kStages) + 1) & 1, st)) break;
      mbar_expect_tx(&sm.full[b], kD * (kBM + kBN) * kBK * 2);
      const int k0 = kbeg + it * kBK;
      for (int p = 0; p < kD; ++p) {
        tma_load_3d(sm.a[b][p], &map_a, &sm.full[b], k0, m0, p);
        tma_load_3d(sm.w[b][p], &map_w, &sm.full[b], k0, n0, p);
      }
    }
    for (int t = it - kStages < 0 ? 0 : it - kStages; t < it; ++t)
      mbar_wait_drain(&sm.full[t % kStages], (t / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int it = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int u = c & 1;
      if (c >= 2 && !mbar_wait(&sm.acc_empty[u], ((c >> 1) - 1) & 1, st)) break;
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int jj = 0; jj < steps_c; ++jj, ++it) {
        const int b = it % kStages;
        if (!mbar_wait(&sm.full[b], (it / kStages) & 1, st)) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint64_t dw = desc_sw128(sm.w[b][0]);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)
#pragma unroll
          for (int s = 0; s < kD; ++s)
            mma_bf16(tmem + u * kSet + s * kBN, desc_sw128(sm.a[b][s]) + 2 * kk, dw + 2 * kk,
                     idesc_bf16(kBM, kBN * (kD - s)), (jj > 0 || kk > 0 || s > 0) ? 1u : 0u);
        mma_commit(&sm.empty[b]);
      }
      if (ok) mma_commit(&sm.acc_full[u]);
    }
    mma_commit(&sm.drain);
    mbar_wait_drain(&sm.drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: lane = row of A's tile, 32 of the 64 columns per warp;
    // W = G_0 2^16 + G_1 2^8 + G_2 summed exactly over the chunks in int64
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int m = m0 + quarter * 32 + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + half * 32;
    long long acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int u = c & 1;
      if (!mbar_wait(&sm.acc_full[u], (c >> 1) & 1, st)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const uint32_t base = lane_base + u * kSet;
#pragma unroll
      for (int cb = 0; cb < 32; cb += 16) {
        float v[16];
        tmem_ld16(base + 0 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<16>(acc[cb + i], v[i]);
        tmem_ld16(base + 1 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<8>(acc[cb + i], v[i]);
        tmem_ld16(base + 2 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<0>(acc[cb + i], v[i]);
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[u]);
    }
    if (ok && m < M) {
      const int em = ea[m];
      float* o = out + blockIdx.z * zstride + (int64_t)m * ldo;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int n = n0 + half * 32 + i;
        if (n < N) o[n] = i64_to_float(acc[i], em + ew[n] + 2 - 32);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// Split count: one CTA per SM, a launch takes waves x (chunks per split + a fixed cost).
int splits(int64_t M, int64_t N, int64_t K, int sms, int cap) {
  const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
  constexpr int chunk = kChunkSteps * kBK;
  const int64_t chunks = (K + chunk - 1) / chunk;
  int best = 1;
  double best_t = 1e300;
  for (int64_t s = 1; s <= cap && s <= chunks; ++s) {
    const int64_t per = (chunks + s - 1) / s;
    const int64_t eff = (chunks + per - 1) / per;
    if (eff != s) continue;
    const int64_t waves = (tiles * eff + sms - 1) / sms;
    const double t = (double)waves * ((double)per + 0.5) + 0.02 * (double)eff;
    if (t < best_t) {
      best_t = t;
      best = (int)eff;
    }
  }
  return best;
}
}  // namespace f32s
}  // namespace tcg

int64_t gemm_f64emu_kpad(int64_t K) { return (K + tcg::kBK - 1) / tcg::kBK * tcg::kBK; }
size_t gemm_f64emu_digit_bytes(int64_t rows, int64_t Kmax) {
  return (size_t)7 * rows * gemm_f64emu_kpad(Kmax) * 2;
}

int gemm_f64emu_splits(int64_t M, int64_t N, int64_t K, int sms) {
  return tcg::splits_for<7>(M, N, K, sms, 8);  // the Schur partial buffer holds 8
}

namespace tcg {
// Slice A's gathered rows and B's gathered columns, then one digit GEMM.
template <typename T, int KD>
cudaError_t gemm_emu_gather(int M, int N, int K, const T* A, int64_t lda, const int32_t* aidx, const T* B,
                            int64_t ldb, int64_t boff, const int32_t* bidx, void* adig, int64_t arows, int32_t* aexp,
                            void* bdig, int64_t brows, int32_t* bexp, unsigned long long* colmax, int64_t kmax,
                            T* out, int64_t ldo, int64_t zstride, int splits, DevState* st, const int32_t* done,
                            cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int64_t Kp = gemm_f64emu_kpad(kmax);
  if (K > kmax || M > arows || N > brows || N > kColTile) return cudaErrorInvalidValue;
  auto ad = static_cast<__nv_bfloat16*>(adig);
  auto bd = static_cast<__nv_bfloat16*>(bdig);
  const int Kq = (int)gemm_f64emu_kpad(K);  // slice only the K range in use
  int64_t g1 = ((int64_t)M * 32 + 255) / 256;
  if (g1 > 8192) g1 = 8192;
  k_slice_rows<T, KD><<<(int)g1, 256, 0, s>>>(M, K, Kq, Kp, A, lda, aidx, ad, arows * Kp, aexp, done);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(colmax, 0, (size_t)N * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int kt = (int)((K + kColTile - 1) / kColTile);
  k_col_max<T><<<kt, 256, 0, s>>>(K, N, B, ldb, boff, bidx, colmax, done);
  k_col_digits<T, KD><<<(Kq + kColTile - 1) / kColTile, 256, 0, s>>>(K, N, (int)Kp, B, ldb, boff, bidx, colmax, bd,
                                                                      brows * Kp, bexp, done);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch<KD, T>(M, N, K, Kp, ad, arows, aexp, bd, brows, bexp, out, ldo, zstride, splits, st, done, s);
}
}  // namespace tcg

cudaError_t gemm_f64emu(int M, int N, int K, const double* A, int64_t lda, const int32_t* aidx, const double* B,
                        int64_t ldb, int64_t boff, const int32_t* bidx, void* adig, int64_t arows, int32_t* aexp,
                        void* bdig, int64_t brows, int32_t* bexp, unsigned long long* colmax, int64_t kmax,
                        double* out, int64_t ldo, int64_t zstride, int splits, DevState* st, const int32_t* done,
                        cudaStream_t s) {
  return tcg::gemm_emu_gather<double, 7>(M, N, K, A, lda, aidx, B, ldb, boff, bidx, adig, arows, aexp, bdig, brows,
                                         bexp, colmax, kmax, out, ldo, zstride, splits, st, done, s);
}

// ---- FP32 sketch on the tensor cores (3 digits per operand)
size_t sketch_f32emu_digit_bytes(int64_t rows, int64_t K) {
  return (size_t)3 * rows * gemm_f64emu_kpad(K) * 2;
}

int sketch_f32emu_splits(int64_t m, int64_t n, int64_t unit_rows, int sms) {
  return tcg::f32s::splits(n, unit_rows, m, sms, 32);
}

cudaError_t sketch_f32emu_slice(int rows, int K, const float* src, int64_t lds, void* dig, int64_t rows_alloc,
                                int32_t* ex, unsigned long long* rowmax, const int32_t* done, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (rows > rows_alloc) return cudaErrorInvalidValue;
  const int64_t Kp = gemm_f64emu_kpad(K);
  auto d = static_cast<__nv_bfloat16*>(dig);
  if (rows >= 1024 || rowmax == nullptr || rows > 65535) {  // many rows: one warp per row
    int64_t g = ((int64_t)rows * 32 + 255) / 256;
    if (g > 8192) g = 8192;
    tcg::k_slice_rows<float, 3><<<(int)g, 256, 0, s>>>(rows, K, (int)Kp, Kp, src, lds, nullptr, d, rows_alloc * Kp,
                                                       ex, done);
    return cudaGetLastError();
  }
  // few long rows (a pass of Omega): blocks along K for every row
  cudaError_t e = cudaMemsetAsync(rowmax, 0, (size_t)rows * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int64_t bx = (Kp + 255) / 256;
  if (bx > 64) bx = 64;
  tcg::k_rows_max<float><<<dim3((unsigned)bx, (unsigned)rows), 256, 0, s>>>(rows, K, src, lds, rowmax, done);
  tcg::k_rows_digits<float, 3><<<dim3((unsigned)bx, (unsigned)rows), 256, 0, s>>>(rows, K, (int)Kp, Kp, src, lds,
                                                                                  rowmax, d, rows_alloc * Kp, ex,
                                                                                  done);
  return cudaGetLastError();
}

cudaError_t sketch_f32emu(int64_t m, int64_t n, int64_t rows, const void* adig, const int32_t* aexp, const void* wdig,
                          int64_t wrows, const int32_t* wexp, float* out, int64_t ldo, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s) {
  using namespace tcg;
  if (rows <= 0) return cudaSuccess;
  if (rows > wrows) return cudaErrorInvalidValue;
  const int64_t Kp = gemm_f64emu_kpad(m);
  CUtensorMap ma, mw;
  if (!make_map(&ma, adig, Kp, n, f32s::kBM, f32s::kD)) return cudaErrorInvalidValue;
  if (!make_map(&mw, wdig, Kp, wrows, f32s::kBN, f32s::kD)) return cudaErrorInvalidValue;
  constexpr int chunk = f32s::kChunkSteps * f32s::kBK;
  const int64_t chunks = (m + chunk - 1) / chunk;
  const int64_t per = (chunks + splits - 1) / splits;
  const int kchunk = (int)(per * chunk);
  const int nz = (int)((m + kchunk - 1) / kchunk);
  if (nz != splits) return cudaErrorInvalidValue;  // the reduction reads exactly `splits` partials
  const size_t smem = sizeof(f32s::Smem) + 1024;
  static SmemLimit lim;
  cudaError_t e = raise_smem(f32s::k_sketch_f32emu, smem, lim);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((n + f32s::kBM - 1) / f32s::kBM), (unsigned)((rows + f32s::kBN - 1) / f32s::kBN), (unsigned)nz);
  f32s::k_sketch_f32emu<<<grid, f32s::kThreads, smem, s>>>(ma, mw, (int)n, (int)rows, (int)m, kchunk, aexp, wexp, out,
                                                          ldo, zstride, st, done);
  return cudaGetLastError();
}

}  // namespace rid
