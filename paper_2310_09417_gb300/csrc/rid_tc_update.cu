// rid_tc_update.cu -- the block update of the interpolation coefficients,
// T(rest, old) -= N T(piv, old) (Algorithm 1's re-blocking, in the
// T = L2 L1^{-1} form), on the BF16 tensor cores by exact digit slicing, for
// FP64 T (KD = 7 digits per operand) and FP32 T (KD = 3).
//
// K = bt <= 64.  Each row i of N gets an exponent e_i (max_q |N(i,q)| < 2^e_i) and
// each column c of P = T(piv, old) an exponent f_c (max_q |P(q,c)| < 2^f_c).
// N(i,:) / 2^(e_i+1) and P(:,c) / 2^(f_c+1) lie in (-1/2, 1/2) and are written as
// KD balanced 8-bit digits (|d| <= 128, exact in BF16: 56 bits for KD = 7, 24 for
// KD = 3).  The digit products of equal weight 2^(-8(g+2)), g = s + t < KD, share
// FP32 group g in tensor memory (KD groups x kBN columns, kBN = 32 for KD = 7 and 64
// for KD = 3, two sets); a group sums at most KD pairs x 64 terms of magnitude
// <= 2^14 (< 2^23): exact.
//   KD = 7: the epilogue folds the groups into one int64 W = sum_g G_g 2^(8(5-g))
//     (group 6 rounded to units of 2^8, |W| < 2^61), converts W 2^(e_i + f_c + 2 -
//     56) to FP64 by integer operations and subtracts it from T (one FP64
//     instruction per entry).  Dropped pairs (g >= 7) and digit remainders bound
//     each entry's error by about 2^-46 max_q|N(i,q)| max_q|P(q,c)| -- the order
//     of an FP64 dot product of length 64 (64 u); the fold adds at most 2^-55 of
//     that scale.
//   KD = 3: W = G_0 2^16 + G_1 2^8 + G_2 (|W| < 2^38) is rounded to FP32 once and
//     scaled by 2^(e_i + f_c + 2 - 32); dropped pairs (g >= 3) and remainders bound
//     the error by about 2^-18 max_q|N(i,q)| max_q|P(q,c)|, the order of an FP32
//     dot product of length 64.
//
//   warp 0    TMA: the row tile's digits of N once, then P's digits per column
//             tile (double-buffered)
//   warp 1    tensor memory; per K step of 16 and slice s of N one MMA (M = 128,
//             N = kBN (KD - s)) against P's planes 0 .. KD-1-s stacked along N, which
//             writes groups s .. KD-1 at once: KD x 4 MMAs per tile; the two
//             accumulator sets let a tile's MMAs run during the last tile's epilogue
//   warps 2-17 epilogue: four warps per lane quarter, 16 columns each; the
//             accumulators are read with one row per lane and released before
//             the stores, T is read (before the accumulators are ready) and
//             written coalesced, the products passing through shared memory
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {
namespace tcu {

using namespace tcx;

constexpr int kBM = 128;    // rows of T per tile
constexpr int kK = 64;      // padded K (one 128-byte swizzle row of BF16)
constexpr int kEpiWarps = 16;  // four per tensor-memory lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;

// Columns of T per tile.  The accumulators are double-buffered (the next tile's
// MMAs run while the epilogue reads the last one): two sets of KD groups x kBN
// columns, 448 (KD = 7) or 384 (KD = 3) of the 512 tensor-memory columns.
template <int KD>
__host__ __device__ constexpr int bn() {
  return KD == 7 ? 32 : 64;
}
template <int KD>
__host__ __device__ constexpr int set_cols() {
  return KD * bn<KD>();
}

template <int KD, typename TX>
struct Smem {
  alignas(1024) __nv_bfloat16 n[KD][kBM * kK];            // KD x 16 KB
  alignas(1024) __nv_bfloat16 p[2][KD][bn<KD>() * kK];    // planes back to back: one operand along N
  TX stage[kEpiWarps][32][9];  // per warp: 32 rows x 8 columns (+1 against bank conflicts)
  TX* rows[kEpiWarps][32];     // per warp: T's row of each of its 32 rows (null: not updated)
  uint64_t n_full;
  uint64_t p_full[2];
  uint64_t p_empty[2];
  uint64_t t_full[2];   // a tile's MMAs completed (accumulator set u & 1)
  uint64_t t_empty[2];  // the epilogue read accumulator set u & 1
  uint64_t drain;
  uint32_t tmem_base;
};
static_assert(sizeof(Smem<7, double>) + 1024 <= 232448, "shared memory of k_update_emu exceeds 227 KB");
static_assert(sizeof(Smem<3, float>) + 1024 <= 232448, "shared memory of k_update_emu exceeds 227 KB");
static_assert(2 * set_cols<7>() <= 512 && 2 * set_cols<3>() <= 512, "two accumulator sets exceed tensor memory");

// The folded accumulators of 8 columns of this lane's row; group g of the set
// starts at column g * bn.
template <int KD>
__device__ __forceinline__ void fold8(uint32_t taddr, long long* w) {
  constexpr int kG = bn<KD>();
  // loads issued in batches, one wait per batch (KD = 7: groups 0-3, then 4-6)
  uint32_t r[4][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = 0;
  if constexpr (KD == 7) {
#pragma unroll
    for (int g = 0; g < 4; ++g) tmem_ld8_nowait(taddr + g * kG, r[g]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      add_scaled<16>(w[i], __uint_as_float(r[0][i]));
      add_scaled<8>(w[i], __uint_as_float(r[1][i]));
      add_scaled<0>(w[i], __uint_as_float(r[2][i]));
      w[i] <<= 24;  // |w| < 2^37 before the shift
      add_scaled<16>(w[i], __uint_as_float(r[3][i]));
    }
#pragma unroll
    for (int g = 0; g < 3; ++g) tmem_ld8_nowait(taddr + (4 + g) * kG, r[g]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      add_scaled<8>(w[i], __uint_as_float(r[0][i]));
      add_scaled<0>(w[i], __uint_as_float(r[1][i]));
      w[i] += __float2int_rn(__uint_as_float(r[2][i]) * 0x1.0p-8f);
    }
  } else {
    static_assert(KD == 3, "KD is 7 or 3");
#pragma unroll
    for (int g = 0; g < 3; ++g) tmem_ld8_nowait(taddr + g * kG, r[g]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      add_scaled<16>(w[i], __uint_as_float(r[0][i]));
      add_scaled<8>(w[i], __uint_as_float(r[1][i]));
      add_scaled<0>(w[i], __uint_as_float(r[2][i]));
    }
  }
}
// unit of the fold: 2^(e_i + f_c + fold_exp)
template <int KD>
__host__ __device__ constexpr int fold_exp() {
  return KD == 7 ? 2 - 56 : 2 - 32;
}
__device__ __forceinline__ double fold_value(long long w, int ex, double) { return i64_to_double(w, ex); }
// |w| < 2^38, rounded once to FP32 without the 64-bit conversion instruction (it
// runs on GB300's FP64 pipe, about two per clock per SM): w = 2^23 h + l with
// 0 <= l < 2^23 and |h| < 2^15, both made exact floats by magic-number additions,
// then fma(h, 2^23, l) -- the exact sum rounded once, as the conversion would.  The
// power-of-two scale is exact for normal results.
__device__ __forceinline__ float fold_value(long long w, int ex, float) {
  const int h = (int)(w >> 23);
  const int l = (int)(w - ((long long)h << 23));
  const float fh = __int_as_float(0x4B400000 + h) - 12582912.0f;  // 1.5 * 2^23 + h, |h| < 2^22
  const float fl = __int_as_float(0x4B000000 | l) - 8388608.0f;   // 2^23 + l, 0 <= l < 2^23
  const float f = fmaf(fh, 8388608.0f, fl);
  if (ex >= -126 && ex <= 127) return f * __int_as_float((ex + 127) << 23);
  return ldexpf(f, ex);
}

// Tiles (row tile, column tile) in row-major order are split into one contiguous,
// balanced range per CTA (one CTA per SM): a range spans few row tiles, whose N
// digits are loaded when the range enters them.
template <int KD, typename TX>
__global__ void __launch_bounds__(kThreads, 1)
    k_update_emu(const __grid_constant__ CUtensorMap map_n, const __grid_constant__ CUtensorMap map_p, int na,
                 int tb, const int32_t* __restrict__ nexp, const int32_t* __restrict__ pexp,
                 const int32_t* __restrict__ act, const int32_t* __restrict__ pivmark, TX* __restrict__ X,
                 int64_t ldx, DevState* st, const int32_t* done) {
  constexpr int kD = KD;
  constexpr int kBN = bn<KD>();
  constexpr int kSet = set_cols<KD>();
  constexpr int kCols = kBN / 4;      // columns of a tile per epilogue warp
  constexpr int kHalves = kCols / 8;  // groups of 8 columns per warp
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem<KD, TX>& sm =
      *reinterpret_cast<Smem<KD, TX>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = (tb + kBN - 1) / kBN;
  const int rt = (na + kBM - 1) / kBM;
  const int64_t total = (int64_t)rt * ct;
  const int64_t t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
  const int my = (int)(t1 - t0);

  if (threadIdx.x == 0) {
    mbar_init(&sm.n_full, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.p_full[b], 1);
      mbar_init(&sm.p_empty[b], 1);
      mbar_init(&sm.t_full[b], 1);
      mbar_init(&sm.t_empty[b], kEpiWarps);
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
    // ---------------- TMA producer
    int issued = 0, cur = -1, segs = 0;
    bool ok = true;
    for (int u = 0; u < my && ok; ++u) {
      const int64_t t = t0 + u;
      const int row = (int)(t / ct), col = (int)(t % ct);
      const int b = u & 1;
      if (row != cur) {
        // N's tile is free once the MMAs of tile u - 1 (and all before) completed
        if (u > 0 && !mbar_wait(&sm.p_empty[(u - 1) & 1], ((u - 1) >> 1) & 1, st)) break;
        mbar_expect_tx(&sm.n_full, kD * kBM * kK * 2);
        for (int s = 0; s < kD; ++s) tma_load_3d(sm.n[s], &map_n, &sm.n_full, 0, row * kBM, s);
        cur = row;
        ++segs;
        // the copies land before this N tile is replaced (or the CTA exits)
        if (!mbar_wait(&sm.n_full, (segs - 1) & 1, st)) ok = false;
      }
      // buffer b is free once the MMAs of tile u - 2 completed
      if (!ok || (u >= 2 && !mbar_wait(&sm.p_empty[b], ((u >> 1) - 1) & 1, st))) break;
      mbar_expect_tx(&sm.p_full[b], kD * kBN * kK * 2);
      for (int q = 0; q < kD; ++q) tma_load_3d(sm.p[b][q], &map_p, &sm.p_full[b], 0, col * kBN, q);
      issued = u + 1;
    }
    for (int u = issued - 2 < 0 ? 0 : issued - 2; u < issued; ++u) mbar_wait_drain(&sm.p_full[u & 1], (u >> 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: per K step and slice s of N, one MMA against P's
    // planes 0 .. KD-1-s stacked along N writes groups s .. KD-1 at once
    int cur = -1, segs = 0;
    for (int u = 0; u < my; ++u) {
      const int64_t t = t0 + u;
      const int row = (int)(t / ct);
      const int b = u & 1;
      if (row != cur) {
        cur = row;
        ++segs;
        if (!mbar_wait(&sm.n_full, (segs - 1) & 1, st)) break;
      }
      if (u >= 2 && !mbar_wait(&sm.t_empty[b], ((u >> 1) - 1) & 1, st)) break;
      if (!mbar_wait(&sm.p_full[b], (u >> 1) & 1, st)) break;
      fence_after_sync();
      const uint64_t db = desc_sw128(sm.p[b][0]);
#pragma unroll
      for (int kk = 0; kk < kK / 16; ++kk)
#pragma unroll
        for (int s = 0; s < kD; ++s)
          mma_bf16(tmem + b * kSet + s * kBN, desc_sw128(sm.n[s]) + 2 * kk, db + 2 * kk,
                   idesc_bf16(kBM, kBN * (kD - s)), (s > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&sm.p_empty[b]);
      mma_commit(&sm.t_full[b]);
    }
    mma_commit(&sm.drain);
    mbar_wait_drain(&sm.drain, 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: each warp owns 32 rows (its tensor-memory lane
    // quarter) and kCols of the tile's columns.  The accumulators are read with
    // lane = row; T is read and written coalesced (instruction i of a group of 8
    // columns covers rows 4i .. 4i+3), the products passing through shared memory.
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int part = ew >> 2;  // 0..3
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + part * kCols;
    // rows of this lane in the coalesced layout: 4 i + (lane >> 3), i < 8
    TX* const* rowp = sm.rows[ew] + (lane >> 3);
    TX(*stage)[9] = sm.stage[ew];
    const int jc = lane & 7;
    int cur = -1, er = 0;
    auto enter_row = [&](int row) {  // this warp's 32 rows of row tile `row`
      const int r = row * kBM + quarter * 32 + lane;
      const bool live = r < na && pivmark[r] == 0;
      er = live ? nexp[r] : 0;
      __syncwarp();
      sm.rows[ew][lane] = live ? X + (int64_t)act[r] * ldx : nullptr;
      __syncwarp();
      cur = row;
    };
    // T's entries and the column exponents of tile u + 1 are loaded while tile u is
    // processed when both lie in the same row tile
    TX xn[kHalves][8];
    int pn = 0;
    auto fetch = [&](int col) {
      const int c0 = col * kBN + part * kCols;
      pn = (lane < kCols && c0 + lane < tb) ? pexp[c0 + lane] : 0;
#pragma unroll
      for (int h = 0; h < kHalves; ++h)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = c0 + 8 * h + jc;
          TX* const rp = rowp[4 * i];
          xn[h][i] = (rp != nullptr && c < tb) ? rp[c] : TX(0);
        }
    };
    bool have = false;  // xn / pn hold tile u
    for (int u = 0; u < my; ++u) {
      const int64_t t = t0 + u;
      const int row = (int)(t / ct), col = (int)(t % ct);
      const int b = u & 1;
      if (row != cur) {
        enter_row(row);
        have = false;
      }
      if (!have) fetch(col);
      const int c0 = col * kBN + part * kCols;
      TX xv[kHalves][8];
#pragma unroll
      for (int h = 0; h < kHalves; ++h)
#pragma unroll
        for (int i = 0; i < 8; ++i) xv[h][i] = xn[h][i];
      const int pe = pn;  // lane j < kCols: the exponent of column c0 + j
      have = false;
      if (u + 1 < my && (t + 1) / ct == row) {
        fetch((int)((t + 1) % ct));
        have = true;
      }
      if (!mbar_wait(&sm.t_full[b], (u >> 1) & 1, st)) break;
      fence_after_sync();
#pragma unroll
      for (int h = 0; h < kHalves; ++h) {
        long long w[8];
        fold8<KD>(lane_base + b * kSet + 8 * h, w);
        if (h == kHalves - 1) {
          // this accumulator set is free for tile u + 2
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sm.t_empty[b]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int ec = __shfl_sync(0xffffffffu, pe, 8 * h + j);
          stage[lane][j] = fold_value(w[j], er + ec + fold_exp<KD>(), TX(0));
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = c0 + 8 * h + jc;
          TX* const rp = rowp[4 * i];
          if (rp != nullptr && c < tb) rp[c] = xv[h][i] - stage[4 * i + (lane >> 3)][jc];
        }
        __syncwarp();
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

// ------------------------------------------------------------------ digit slicing
// Both slicers work on the IEEE bit patterns with integer operations: the row (or
// column) exponent from the largest pattern, then F = round(x 2^(8 KD - 1 - e)) and
// its KD balanced digits.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float x) {
  return (unsigned long long)((unsigned)__float_as_int(x) & 0x7FFFFFFFu);
}
__device__ __forceinline__ int exp_above_bits(unsigned long long b, double) { return exp_above_f64bits(b); }
__device__ __forceinline__ int exp_above_bits(unsigned long long b, float) { return exp_above_f32bits((unsigned)b); }

// N (na x bt, row stride bt): one warp per row; digits D[s][i][q] (q < 64, zero-padded).
template <typename T, int KD>
__global__ void k_slice_n(int na, int bt, const T* __restrict__ N, __nv_bfloat16* __restrict__ D,
                          int32_t* __restrict__ nexp, int64_t plane, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < na; i += nw) {
    const T a0 = lane < bt ? N[i * bt + lane] : T(0);
    const T a1 = lane + 32 < bt ? N[i * bt + lane + 32] : T(0);
    const unsigned long long mb = warp_max_u64(max(abs_bits(a0), abs_bits(a1)));
    const int e = exp_above_bits(mb, T(0));
    if (lane == 0) nexp[i] = e;
    write_digits<KD>(fixed_of<KD>(a0, e), D + i * kK + lane, plane);
    write_digits<KD>(fixed_of<KD>(a1, e), D + i * kK + lane + 32, plane);
  }
}

// P(q, c) = X(pivorig[q] row, c) for q < bt, c < tb: per column c (one warp), digits
// D[t][c][q] (q < 64, zero-padded).
template <typename T, int KD>
__global__ void k_slice_p(int bt, int tb, const T* __restrict__ X, int64_t ldx, const int32_t* __restrict__ prow,
                          __nv_bfloat16* __restrict__ D, int32_t* __restrict__ pexp, int64_t plane,
                          const int32_t* done) {
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < tb; c += nw) {
    const T a0 = lane < bt ? X[(int64_t)prow[lane] * ldx + c] : T(0);
    const T a1 = lane + 32 < bt ? X[(int64_t)prow[lane + 32] * ldx + c] : T(0);
    const unsigned long long mb = warp_max_u64(max(abs_bits(a0), abs_bits(a1)));
    const int e = exp_above_bits(mb, T(0));
    if (lane == 0) pexp[c] = e;
    write_digits<KD>(fixed_of<KD>(a0, e), D + c * kK + lane, plane);
    write_digits<KD>(fixed_of<KD>(a1, e), D + c * kK + lane + 32, plane);
  }
}

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows, int planes) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kK, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)kK * 2, (cuuint64_t)kK * rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)kK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KD, typename T>
cudaError_t update_emu(int na, int bt, int tb, const T* N, const int32_t* act, const int32_t* pivmark,
                       const int32_t* pivorig, T* X, int64_t ldx, void* ndig, int32_t* nexp, int64_t nrows, void* pdig,
                       int32_t* pexp, int64_t prows, int sms, DevState* st, const int32_t* done, cudaStream_t s) {
  if (na <= 0 || tb <= 0) return cudaSuccess;
  if (bt > kK || na > nrows || tb > prows) return cudaErrorInvalidValue;
  auto nd = static_cast<__nv_bfloat16*>(ndig);
  auto pd = static_cast<__nv_bfloat16*>(pdig);
  const int64_t nplane = nrows * kK, pplane = prows * kK;
  int64_t b1 = ((int64_t)na * 32 + 255) / 256;
  if (b1 > 4096) b1 = 4096;
  k_slice_n<T, KD><<<(int)b1, 256, 0, s>>>(na, bt, N, nd, nexp, nplane, done);
  int64_t b2 = ((int64_t)tb * 32 + 255) / 256;
  if (b2 > 4096) b2 = 4096;
  k_slice_p<T, KD><<<(int)b2, 256, 0, s>>>(bt, tb, X, ldx, pivorig, pd, pexp, pplane, done);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mn, mp;
  if (!make_map(&mn, nd, nrows, kBM, KD)) return cudaErrorInvalidValue;
  if (!make_map(&mp, pd, prows, bn<KD>(), KD)) return cudaErrorInvalidValue;
  const size_t smem = sizeof(Smem<KD, T>) + 1024;
  static SmemLimit lim;
  e = raise_smem(k_update_emu<KD, T>, smem, lim);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (int64_t)((na + kBM - 1) / kBM) * ((tb + bn<KD>() - 1) / bn<KD>());
  const int grid = (int)(tiles < sms ? tiles : sms);  // one CTA per SM, balanced tile ranges
  k_update_emu<KD, T><<<grid, kThreads, smem, s>>>(mn, mp, na, tb, nexp, pexp, act, pivmark, X, ldx, st, done);
  return cudaGetLastError();
}

}  // namespace tcu

size_t update_f64emu_digit_bytes(int64_t rows) { return (size_t)7 * rows * tcu::kK * 2; }
size_t update_f32emu_digit_bytes(int64_t rows) { return (size_t)3 * rows * tcu::kK * 2; }

cudaError_t update_f64emu(int na, int bt, int tb, const double* N, const int32_t* act, const int32_t* pivmark,
                          const int32_t* pivorig, double* X, int64_t ldx, void* ndig, int32_t* nexp, int64_t nrows,
                          void* pdig, int32_t* pexp, int64_t prows, int sms, DevState* st, const int32_t* done,
                          cudaStream_t s) {
  return tcu::update_emu<7, double>(na, bt, tb, N, act, pivmark, pivorig, X, ldx, ndig, nexp, nrows, pdig, pexp, prows,
                                    sms, st, done, s);
}

cudaError_t update_f32emu(int na, int bt, int tb, const float* N, const int32_t* act, const int32_t* pivmark,
                          const int32_t* pivorig, float* X, int64_t ldx, void* ndig, int32_t* nexp, int64_t nrows,
                          void* pdig, int32_t* pexp, int64_t prows, int sms, DevState* st, const int32_t* done,
                          cudaStream_t s) {
  return tcu::update_emu<3, float>(na, bt, tb, N, act, pivmark, pivorig, X, ldx, ndig, nexp, nrows, pdig, pexp, prows,
                                   sms, st, done, s);
}

}  // namespace rid
