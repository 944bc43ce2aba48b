// rid_tc_gemm64.cu -- an FP64-accurate GEMM on the BF16 tensor cores for the
// Schur complement of the FP64-emulated path: P = T(act, 0:K) G(perm, cols)
// (Alg. 1 lines 10-11 in the T = L2 L1^{-1} form), written as FP64 split-K
// partials for the Schur finish.
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
//   warp 1    tensor memory; per (K step, slice s) 4 (7 - s) MMAs M=128 N=32 K=16
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
constexpr int kBN = 32;       // columns of B per tile
constexpr int kBK = 64;       // K per step
constexpr int kD = 7;         // digits
constexpr int kChunkSteps = 2;  // exact chunk: 128 K
constexpr int kAStages = 6;
constexpr int kThreads = 192;
constexpr int kGroupCols = kD * kBN;  // 224 tensor-memory columns per accumulator set

struct Smem {
  alignas(1024) __nv_bfloat16 a[kAStages][kBM * kBK];  // 16 KB each
  alignas(1024) __nv_bfloat16 b[2][kD][kBN * kBK];     // 2 x 7 x 4 KB
  uint64_t a_full[kAStages];
  uint64_t a_empty[kAStages];
  uint64_t b_full[2];
  uint64_t b_empty[2];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
};
static_assert(sizeof(Smem) + 1024 <= 232448, "shared memory of k_gemm_f64emu exceeds 227 KB");


// Grid: x = column tiles of B (fastest: CTAs sharing an A tile run together), y = row
// tiles of A, z = K splits of kchunk (a multiple of 128).  out[z]: FP64 partial
// (M x N, row stride ldo).
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_f64emu(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M, int N,
                  int K, int kchunk, const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                  double* __restrict__ out, int64_t ldo, int64_t zstride, DevState* st, const int32_t* done) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
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
      mbar_init(&sm.acc_full[i], 1);
      mbar_init(&sm.acc_empty[i], 4);
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
    // ---------------- TMA producer: per K step, B's digits, then A's seven slices
    int ai = 0, jb = 0;
    bool ok = true;
    for (int j = 0; j < nsteps && ok; ++j) {
      const int bb = j & 1;
      if (j >= 2 && !mbar_wait(&sm.b_empty[bb], ((j >> 1) + 1) & 1, st)) break;
      const int k0 = kbeg + j * kBK;
      mbar_expect_tx(&sm.b_full[bb], kD * kBN * kBK * 2);
      for (int t = 0; t < kD; ++t) tma_load_3d(sm.b[bb][t], &map_b, &sm.b_full[bb], k0, n0, t);
      jb = j + 1;
      for (int s = 0; s < kD; ++s, ++ai) {
        const int st_ = ai % kAStages;
        if (ai >= kAStages && !mbar_wait(&sm.a_empty[st_], ((ai / kAStages) + 1) & 1, st)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&sm.a_full[st_], kBM * kBK * 2);
        tma_load_3d(sm.a[st_], &map_a, &sm.a_full[st_], k0, m0, s);
      }
    }
    // copies still in flight land before the CTA may exit
    for (int i = ai - kAStages < 0 ? 0 : ai - kAStages; i < ai; ++i)
      mbar_wait_drain(&sm.a_full[i % kAStages], (i / kAStages) & 1);
    for (int j = jb - 2 < 0 ? 0 : jb - 2; j < jb; ++j) mbar_wait_drain(&sm.b_full[j & 1], (j >> 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(kBM, kBN);
    int ai = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int u = c & 1;  // accumulator set
      if (c >= 2 && !mbar_wait(&sm.acc_empty[u], ((c >> 1) + 1) & 1, st)) break;
      fence_after_sync();
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int jj = 0; jj < steps_c && ok; ++jj) {
        const int j = c * kChunkSteps + jj;
        const int bb = j & 1;
        if (!mbar_wait(&sm.b_full[bb], (j >> 1) & 1, st)) {
          ok = false;
          break;
        }
        fence_after_sync();
        for (int s = 0; s < kD; ++s, ++ai) {
          const int st_ = ai % kAStages;
          if (!mbar_wait(&sm.a_full[st_], (ai / kAStages) & 1, st)) {
            ok = false;
            break;
          }
          fence_after_sync();
          const uint64_t da = desc_sw128(sm.a[st_]);
          for (int t = 0; t + s < kD; ++t) {
            const uint64_t db = desc_sw128(sm.b[bb][t]);
            const uint32_t dst = tmem + u * kGroupCols + (s + t) * kBN;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              mma_bf16(dst, da + 2 * kk, db + 2 * kk, idesc, (jj > 0 || s > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&sm.a_empty[st_]);
        }
        if (ok) mma_commit(&sm.b_empty[bb]);
      }
      if (ok) mma_commit(&sm.acc_full[u]);
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
        tmem_ld16(base + 0 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<16>(hi[cb + i], v[i]);
        tmem_ld16(base + 1 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<8>(hi[cb + i], v[i]);
        tmem_ld16(base + 2 * kBN + cb, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) add_scaled<0>(hi[cb + i], v[i]);
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
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.acc_empty[u]);
    }
    if (ok && m < M) {
      const int em = ea[m];
      double* o = out + blockIdx.z * zstride + (int64_t)m * ldo;
#pragma unroll
      for (int i = 0; i < kBN; ++i)
        if (n0 + i < N) o[n0 + i] = fixed_to_double(hi[i], lo[i], em + eb[n0 + i] + 2 - 64);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ slicing by integer operations
// e with |x| < 2^e for the largest |x| whose bit pattern (sign cleared) is `bits`; 0 for zero.
__device__ __forceinline__ int exp_of_bits(unsigned long long bits) {
  if (bits == 0) return 0;
  const int E = (int)(bits >> 52);
  if (E == 0) return -1074 + (64 - __clzll((long long)bits));  // subnormal: 2^-1074 units
  return E - 1022;
}

// F = round(x 2^(55 - e)), |F| < 2^55, as seven balanced base-256 digits, most
// significant first: x / 2^(e+1) = sum_s d_s 2^(-8(s+1)).
__device__ __forceinline__ void digits_of(double x, int e, __nv_bfloat16* d, int64_t plane) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long frac = bits & ((1ull << 52) - 1);
  long long F = 0;
  if (E != 0 || frac != 0) {
    const unsigned long long m = E ? (frac | (1ull << 52)) : frac;  // x = m 2^(E' - 1075)
    const int sh = (E ? E : 1) - 1075 + 55 - e;                      // F = m 2^sh
    unsigned long long a;
    if (sh >= 0) {
      a = m << sh;  // only when x is tiny against 2^e: a < 2^55
    } else if (sh > -64) {
      const unsigned long long q = m >> (-sh);
      const unsigned long long r = m - (q << (-sh));
      const unsigned long long half = 1ull << (-sh - 1);
      a = q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull);
    } else {
      a = 0;
    }
    F = (bits >> 63) ? -(long long)a : (long long)a;
  }
  long long dg[kD];
#pragma unroll
  for (int s = kD - 1; s > 0; --s) {
    long long r = F & 255;
    if (r >= 128) r -= 256;  // balanced digit in [-128, 127]
    dg[s] = r;
    F = (F - r) >> 8;  // exact
  }
  dg[0] = F;  // |F| <= 128
#pragma unroll
  for (int s = 0; s < kD; ++s) d[s * plane] = __int2bfloat16_rn((int)dg[s]);
}

// A rows: row r of the result is src[idx[r] * lds + k] for k < K (idx null: r).
// One warp per row: the row's largest |x| (integer comparison of bit patterns),
// then the digits D[s][r][k] (row stride Kp), zero for K <= k < Kq.
__global__ void k_slice_rows(int M, int K, int Kq, int64_t Kp, const double* __restrict__ src, int64_t lds,
                             const int32_t* __restrict__ idx, __nv_bfloat16* __restrict__ D, int64_t plane,
                             int32_t* __restrict__ ex, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < M; r += nw) {
    const double* row = src + (int64_t)(idx ? idx[r] : r) * lds;
    unsigned long long mx = 0;
    for (int k = lane; k < K; k += 32)
      mx = max(mx, (unsigned long long)__double_as_longlong(row[k]) & 0x7FFFFFFFFFFFFFFFull);
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const int e = exp_of_bits(mx);
    if (lane == 0) ex[r] = e;
    for (int k = lane; k < Kq; k += 32) digits_of(k < K ? row[k] : 0.0, e, D + r * Kp + k, plane);
  }
}

// B (K x N): element (k, n) = src[idx[k] * lds + off + n].  First the largest
// |B(:, n)| bit pattern per column (blocks over K, n fastest for coalesced reads,
// atomicMax into colmax, which starts at 0) ...
constexpr int kColTile = 64;
__global__ void k_col_max(int K, int N, const double* __restrict__ src, int64_t lds, int64_t off,
                          const int32_t* __restrict__ idx, unsigned long long* __restrict__ colmax,
                          const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ unsigned long long red[256];
  const int n = threadIdx.x % kColTile, kl = threadIdx.x / kColTile;  // 4 rows per pass
  unsigned long long mx = 0;
  if (n < N)
    for (int k = blockIdx.x * kColTile + kl; k < min(K, (int)(blockIdx.x + 1) * kColTile); k += 4)
      mx = max(mx, (unsigned long long)__double_as_longlong(src[(int64_t)idx[k] * lds + off + n]) &
                       0x7FFFFFFFFFFFFFFFull);
  red[threadIdx.x] = mx;
  __syncthreads();
  if (kl == 0 && n < N) {
    for (int q = 1; q < 4; ++q) mx = max(mx, red[q * kColTile + n]);
    if (mx != 0) atomicMax(&colmax[n], mx);
  }
}

// ... then the digits, one block per 64 rows of K: the tile goes through shared
// memory so that digit writes D[t][n][k] are contiguous in k.
__global__ void k_col_digits(int K, int N, int Kp, const double* __restrict__ src, int64_t lds, int64_t off,
                             const int32_t* __restrict__ idx, const unsigned long long* __restrict__ colmax,
                             __nv_bfloat16* __restrict__ D, int64_t plane, int32_t* __restrict__ ex,
                             const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ double tile[kColTile][kColTile + 1];
  const int k0 = blockIdx.x * kColTile;
  for (int e = threadIdx.x; e < kColTile * kColTile; e += blockDim.x) {
    const int kl = e / kColTile, n = e % kColTile;
    const int k = k0 + kl;
    tile[kl][n] = (k < K && n < N) ? src[(int64_t)idx[k] * lds + off + n] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kColTile * kColTile; e += blockDim.x) {
    const int n = e / kColTile, kl = e % kColTile;  // k fastest: contiguous writes
    const int k = k0 + kl;
    if (n < N && k < Kp) {
      const int en = exp_of_bits(colmax[n]);
      digits_of(k < K ? tile[kl][n] : 0.0, en, D + (int64_t)n * Kp + k, plane);
      if (blockIdx.x == 0 && kl == 0) ex[n] = en;
    }
  }
}

bool make_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int box_rows) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)kD};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tcg

int64_t gemm_f64emu_kpad(int64_t K) { return (K + tcg::kBK - 1) / tcg::kBK * tcg::kBK; }
size_t gemm_f64emu_digit_bytes(int64_t rows, int64_t Kmax) {
  return (size_t)tcg::kD * rows * gemm_f64emu_kpad(Kmax) * 2;
}

int gemm_f64emu_splits(int64_t M, int64_t N, int64_t K, int sms) {
  const int64_t tiles = ((M + tcg::kBM - 1) / tcg::kBM) * ((N + tcg::kBN - 1) / tcg::kBN);
  const int64_t chunks = (K + 127) / 128;
  int64_t s = (sms + tiles - 1) / tiles;  // about one wave
  if (s > chunks) s = chunks;
  if (s > 8) s = 8;  // the Schur partial buffer holds 8
  if (s < 1) s = 1;
  const int64_t per = (chunks + s - 1) / s;
  return (int)((chunks + per - 1) / per);
}

cudaError_t gemm_f64emu(int M, int N, int K, const double* A, int64_t lda, const int32_t* aidx, const double* B,
                        int64_t ldb, int64_t boff, const int32_t* bidx, void* adig, int64_t arows, int32_t* aexp,
                        void* bdig, int64_t brows, int32_t* bexp, unsigned long long* colmax, int64_t kmax,
                        double* out, int64_t ldo,
                        int64_t zstride, int splits, DevState* st, const int32_t* done, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int64_t Kp = gemm_f64emu_kpad(kmax);
  if (K > kmax || M > arows || N > brows) return cudaErrorInvalidValue;
  auto ad = static_cast<__nv_bfloat16*>(adig);
  auto bd = static_cast<__nv_bfloat16*>(bdig);
  const int Kq = (int)gemm_f64emu_kpad(K);  // slice only the K range in use
  int64_t g1 = ((int64_t)M * 32 + 255) / 256;
  if (g1 > 8192) g1 = 8192;
  tcg::k_slice_rows<<<(int)g1, 256, 0, s>>>(M, K, Kq, Kp, A, lda, aidx, ad, arows * Kp, aexp, done);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (N > tcg::kColTile) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(colmax, 0, (size_t)N * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int kt = (int)((K + tcg::kColTile - 1) / tcg::kColTile);
  tcg::k_col_max<<<kt, 256, 0, s>>>(K, N, B, ldb, boff, bidx, colmax, done);
  tcg::k_col_digits<<<(Kq + tcg::kColTile - 1) / tcg::kColTile, 256, 0, s>>>(K, N, (int)Kp, B, ldb, boff, bidx, colmax,
                                                                              bd, brows * Kp, bexp, done);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb;
  if (!tcg::make_map(&ma, ad, Kp, arows, tcg::kBM)) return cudaErrorInvalidValue;
  if (!tcg::make_map(&mb, bd, Kp, brows, tcg::kBN)) return cudaErrorInvalidValue;
  const int64_t chunks = (K + 127) / 128;
  const int64_t per = (chunks + splits - 1) / splits;
  const int kchunk = (int)(per * 128);
  const int nz = (int)((K + kchunk - 1) / kchunk);
  if (nz != splits) return cudaErrorInvalidValue;
  const size_t smem = sizeof(tcg::Smem) + 1024;
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(tcg::k_gemm_f64emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)((N + tcg::kBN - 1) / tcg::kBN), (unsigned)((M + tcg::kBM - 1) / tcg::kBM), (unsigned)nz);
  tcg::k_gemm_f64emu<<<grid, tcg::kThreads, smem, s>>>(ma, mb, M, N, K, kchunk, aexp, bexp, out, ldo, zstride, st,
                                                        done);
  return cudaGetLastError();
}

}  // namespace rid
