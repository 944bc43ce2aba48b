// rid_tc_f64.cu -- an FP64-accurate sketch Y = Omega A on the BF16 tensor cores.
//
// GB300 executes FP64 FMAs at 1.25 TFLOP/s, so the FP64 sketch (Sec. 2.4) is
// moved onto the tensor cores by exact integer slicing:
//   * A: per column j an exponent E_j with max_i |A_ij| < 2^E_j; x = A / 2^(E_j+2)
//     (|x| < 1/4) is written as sum_{s<7} d_s 2^(-8(s+1)) + r with balanced 8-bit
//     digits, |d_0| <= 64 and d_s in [-128, 127] below, |r| <= 2^-57 -- 55 bits per
//     column.  Every digit fits a signed byte: A is stored once per call as 7 int8
//     digit planes, 7 bytes per element (the sketch reads A's 8 FP64 bytes'
//     worth of information as 7).
//   * Omega: standard normal numbers on the grid 2^-11, q = rint(2048 z) clipped to
//     |q| <= 16383, split as q = 256 q1 + q0 with |q1| <= 64, |q0| <= 128.
//   * In the kernel, converter warps widen each int8 tile to BF16 in shared memory
//     (integers exact in BF16), in the 128-byte-swizzled layout the MMA reads.
//     Products of equal weight 2^(-8g) share one FP32 accumulator group in tensor
//     memory: group g collects q1 x d_g and q0 x d_(g-1) (g = 0..7: 8 groups x 64
//     columns = the 512 columns of an SM; no product is dropped).  One MMA with
//     N = 128 (both Omega digits stacked) writes groups s and s+1 for slice s.
//     Over a chunk of 512 K a group's partial sums stay below 512 (128*128 +
//     64*128) < 2^24: the FP32 accumulation is exact.
//   * After slice g of a chunk, group g is final for that chunk; the epilogue
//     warps convert it to integers and add it, exactly, to two int64
//     accumulators per entry (groups 0..3 and 4..7 with weights 2^(8(3-g)) and
//     2^(8(7-g))), then hand the group back to the MMA issuer -- the epilogue
//     of a chunk overlaps the MMAs of the next one.  At the end
//     Y_cj = 2^(E_j - 65) (acc_hi 2^32 + acc_lo), assembled by integer operations.
// Error of an entry: the digit remainders (|r| 2^(E_j+2) <= 2^-54 max_i|A_ij| per
// term) and one final rounding: at most 2^-52 max_i|A_ij| sum_r |Omega_cr| --
// inside the worst-case rounding bound m 2^-53 sum_r |Omega_cr||A_rj| of an FP64
// dot product.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {
namespace tc64 {

constexpr int kBM = 128;         // columns of A per tile (MMA M)
constexpr int kBN = 64;          // rows of Omega per tile (MMA N per digit)
constexpr int kBK = 64;          // K per stage
constexpr int kSlices = 7;       // digits of A
constexpr int kGroups = 8;       // accumulator groups (slice s feeds groups s and s+1)
constexpr int kChunkSteps = 8;   // K stages per exact chunk (512 K)
constexpr int kChunk = kChunkSteps * kBK;
constexpr int kStages = 5;
constexpr int kEpiWarps = 8;     // two per TMEM lane quarter, 32 columns each
constexpr int kCvtWarps = 2;     // int8 -> BF16 widening of the A tiles
constexpr int kThreads = 64 + 32 * kEpiWarps + 32 * kCvtWarps;
constexpr int kMaxChunksPerSplit = 1 << 14;  // int64 accumulators: 2^14 * 2^48 < 2^63
constexpr double kQMax = 16383.0;

using namespace tcx;

// Two signed bytes of a word as a BF16 pair (low element first), without integer
// to float conversions (a quarter-rate pipe): ub is the word with every byte's sign
// bit flipped (byte = d + 128); splicing byte k under the exponent of 2^23 gives
// the float 2^23 + d + 128, and subtracting 2^23 + 128 leaves d exactly.  The
// integers are exact in BF16, whose bits are the FP32's upper half.
template <int K0>
__device__ __forceinline__ uint32_t widen2(uint32_t ub) {
  const float f0 = __uint_as_float(__byte_perm(ub, 0x4B000000u, 0x7540 | K0)) - 8388736.0f;
  const float f1 = __uint_as_float(__byte_perm(ub, 0x4B000000u, 0x7540 | (K0 + 1))) - 8388736.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// acc += v * 2^sh, exact (v an integer-valued float below 2^23 in magnitude)
struct Smem {
  alignas(1024) __nv_bfloat16 a[kStages][kBM * kBK];      // one digit slice of A, widened: 16 KB
  alignas(1024) __nv_bfloat16 w[kStages][2 * kBN * kBK];  // both digits of Omega: 128 rows, 16 KB
  alignas(1024) int8_t araw[kStages][kBM * kBK];          // the slice as loaded: 128 rows x 64 B, 8 KB
  uint64_t full[kStages];   // the TMA copies of stage b landed
  uint64_t cvt[kStages];    // the converter warps widened stage b
  uint64_t empty[kStages];  // the MMAs of stage b completed
  uint64_t ready[kGroups];  // group g of the current chunk is final
  uint64_t free_[kGroups];  // the epilogue has read group g
  uint64_t drain;
  uint32_t tmem_base;
};

// Grid: x = tiles of Omega rows (fastest, so CTAs that share an A tile run
// together and reuse it from L2), y = tiles of A's columns, z = K splits of
// kchunk (a multiple of the exact chunk).  out: FP64 partial (n x rows, row
// stride out_ld) of split blockIdx.z.
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_f64emu(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
                    const int32_t* __restrict__ colexp, int n, int rows, int K, int kchunk,
                    double* __restrict__ out, int64_t out_ld, int64_t zstride, DevState* st, const int32_t* done) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kBN;
  const int m0 = blockIdx.y * kBM;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nsteps = (kend - kbeg + kBK - 1) / kBK;  // K stages of this split
  const int nchunks = (nsteps + kChunkSteps - 1) / kChunkSteps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.cvt[s], kCvtWarps);
      mbar_init(&sm.empty[s], 1);
    }
    for (int g = 0; g < kGroups; ++g) {
      mbar_init(&sm.ready[g], 1);
      mbar_init(&sm.free_[g], kEpiWarps);
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
    // ---------------- TMA producer.  Stage order: chunk c, slice s, step j; each
    // stage holds digit slice s of A and both Omega digits at K step j.
    int it = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int s = 0; s < kSlices && ok; ++s) {
        for (int j = 0; j < steps_c; ++j, ++it) {
          const int b = it % kStages;
          if (it >= kStages && !mbar_wait(&sm.empty[b], ((it / kStages) + 1) & 1, st)) { ok = false; break; }
          mbar_expect_tx(&sm.full[b], kBM * kBK + 2 * kBN * kBK * 2);
          const int k0 = kbeg + (c * kChunkSteps + j) * kBK;
          tma_load_3d(sm.araw[b], &map_a, &sm.full[b], k0, m0, s);
          tma_load_3d(sm.w[b], &map_w, &sm.full[b], k0, n0, 0);
        }
      }
    }
    // the copies still in flight land before the CTA may exit
    for (int t = it - kStages < 0 ? 0 : it - kStages; t < it; ++t) mbar_wait_drain(&sm.full[t % kStages], (t / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t id128 = idesc_bf16(kBM, 2 * kBN), id64 = idesc_bf16(kBM, kBN);
    int it = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int s = 0; s < kSlices && ok; ++s) {
        if (c > 0) {
          // groups s and s+1 are overwritten from here on: the epilogue must have
          // read them for chunk c-1 (group s was already awaited at slice s-1)
          const uint32_t par = (c - 1) & 1;
          if (s == 0 && !mbar_wait(&sm.free_[0], par, st)) { ok = false; break; }
          if (!mbar_wait(&sm.free_[s + 1], par, st)) { ok = false; break; }
          fence_after_sync();
        }
        const uint32_t dst = tmem + s * kBN;
        for (int j = 0; j < steps_c; ++j, ++it) {
          const int b = it % kStages;
          if (!mbar_wait(&sm.full[b], (it / kStages) & 1, st)) { ok = false; break; }
          if (!mbar_wait(&sm.cvt[b], (it / kStages) & 1, st)) { ok = false; break; }
          fence_after_sync();
          const uint64_t da = desc_sw128(sm.a[b]);
          const uint64_t dq1 = desc_sw128(sm.w[b]);             // high digit of Omega (weight 1)
          const uint64_t dq0 = desc_sw128(sm.w[b] + kBN * kBK);  // low digit (weight 2^-8)
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const bool first = (j == 0 && kk == 0);
            if (first && s > 0) {
              // group s continues, group s+1 starts: two MMAs with their own flags
              mma_bf16(dst, da, dq1, id64, 1u);
              mma_bf16(dst + kBN, da, dq0, id64, 0u);
            } else {
              // groups s and s+1 at once (N = 128: q1 rows then q0 rows)
              mma_bf16(dst, da + 2 * kk, dq1 + 2 * kk, id128, (first && s == 0) ? 0u : 1u);
            }
          }
          mma_commit(&sm.empty[b]);
        }
        if (ok) {
          mma_commit(&sm.ready[s]);  // group s is final for chunk c
          if (s == kSlices - 1) mma_commit(&sm.ready[s + 1]);  // and the last group with it
        }
      }
    }
    // every MMA issued has completed before TMEM is released
    mma_commit(&sm.drain);
    mbar_wait_drain(&sm.drain, 0);
  } else if (warp >= 2 + kEpiWarps) {
    // ---------------- converters: stage b's int8 slice (128 rows x 64 K bytes, as
    // loaded) widened to BF16 in the 128-byte-swizzled K-major layout the MMA reads
    // (16-byte chunk c of row r at r * 128 + ((c ^ (r & 7)) << 4)).  Each unit is 8
    // digits: one 8-byte load, one 16-byte store.
    const int ct = threadIdx.x - 32 * (2 + kEpiWarps);  // 0 .. 32 kCvtWarps - 1
    int it = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int s = 0; s < kSlices && ok; ++s) {
        for (int j = 0; j < steps_c; ++j, ++it) {
          const int b = it % kStages;
          if (!mbar_wait(&sm.full[b], (it / kStages) & 1, st)) { ok = false; break; }
          const unsigned char* src = reinterpret_cast<const unsigned char*>(sm.araw[b]);
          unsigned char* dst = reinterpret_cast<unsigned char*>(sm.a[b]);
#pragma unroll
          for (int q = 0; q < (kBM * kBK / 8) / (32 * kCvtWarps); ++q) {
            const int u = ct + q * 32 * kCvtWarps;
            const int r = u >> 3, ch = u & 7;
            const uint2 x = *reinterpret_cast<const uint2*>(src + r * kBK + ch * 8);
            const uint32_t u0 = x.x ^ 0x80808080u, u1 = x.y ^ 0x80808080u;
            uint4 y;
            y.x = widen2<0>(u0);
            y.y = widen2<2>(u0);
            y.z = widen2<0>(u1);
            y.w = widen2<2>(u1);
            *reinterpret_cast<uint4*>(dst + r * 128 + ((ch ^ (r & 7)) << 4)) = y;
          }
          // the generic-proxy stores become visible to the tensor core's reads
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if ((threadIdx.x & 31) == 0) mbar_arrive(&sm.cvt[b]);
        }
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: exact integer accumulation of the groups
    const int ew = warp - 2;
    const int quarter = warp & 3;  // TMEM lanes this warp may read
    const int half = ew >> 2;      // columns [32 half, 32 half + 32) of the tile
    const int row = m0 + quarter * 32 + lane;
    const uint32_t base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + half * 32;
    long long hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) hi[i] = lo[i] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        if (!mbar_wait(&sm.ready[g], c & 1, st)) { ok = false; break; }
        fence_after_sync();
#pragma unroll
        for (int cb = 0; cb < 32; cb += 16) {
          float v[16];
          tmem_ld16(base + g * kBN + cb, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (g == 0) add_scaled<24>(hi[cb + i], v[i]);
            else if (g == 1) add_scaled<16>(hi[cb + i], v[i]);
            else if (g == 2) add_scaled<8>(hi[cb + i], v[i]);
            else if (g == 3) add_scaled<0>(hi[cb + i], v[i]);
            else if (g == 4) add_scaled<24>(lo[cb + i], v[i]);
            else if (g == 5) add_scaled<16>(lo[cb + i], v[i]);
            else if (g == 6) add_scaled<8>(lo[cb + i], v[i]);
            else add_scaled<0>(lo[cb + i], v[i]);
          }
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.free_[g]);
      }
    }
    if (ok && row < n) {
      const int e = colexp[row];
      double* o = out + blockIdx.z * zstride + static_cast<int64_t>(row) * out_ld + n0 + half * 32;
      const int lim = rows - n0 - half * 32;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < lim) o[i] = fixed_to_double(hi[i], lo[i], e - 65);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ digit preparation
// Column exponents: E_j with max_i |A_ij| < 2^E_j (0 for a zero column).
__global__ void k_colexp(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n, int32_t* __restrict__ E) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) mx = fmax(mx, fabs(A[i + j * lda]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, s[w]);
      int e = 0;
      if (r > 0.0) {
        frexp(r, &e);  // r = f 2^e, 0.5 <= f < 1: r < 2^e
      }
      E[j] = e;
    }
    __syncthreads();
  }
}

// Digits: D[s][j][i] (slice-major, each slice column-major m_pad x n, int8) of A(i, j),
// by integer operations on the FP64 bit patterns (x / 2^(E_j+2) = sum_s d_s 2^(-8(s+1));
// F = round(x 2^55) has |F| < 2^54, so the top digit is at most 64 in magnitude).
__global__ void k_split_digits(const double* __restrict__ A, int64_t lda, int64_t m, int64_t m_pad, int64_t n,
                               const int32_t* __restrict__ E, int8_t* __restrict__ D) {
  const int64_t total = m_pad * n;
  const int64_t slice = m_pad * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m_pad, i = e - j * m_pad;
    long long F = i < m ? fixed_of<kSlices>(A[i + j * lda], E[j] + 1) : 0ll;
    int8_t dg[kSlices];
#pragma unroll
    for (int q = kSlices - 1; q > 0; --q) {
      long long r = F & 255;
      if (r >= 128) r -= 256;  // balanced digit in [-128, 127]
      dg[q] = (int8_t)r;
      F = (F - r) >> 8;  // exact
    }
    dg[0] = (int8_t)F;  // |F| <= 64 here
#pragma unroll
    for (int q = 0; q < kSlices; ++q) D[e + q * slice] = dg[q];
  }
}

// Omega digits on the grid 2^-11: W[t][r][i], t = 0 high digit q1, t = 1 low digit q0;
// from the Philox/Box-Muller rows (gen) or a caller matrix (src != nullptr).
__global__ void k_omega_digits(uint64_t seed, int64_t row0, int64_t rows, int64_t m, int64_t ldw, int64_t rows_alloc,
                               const double* __restrict__ src, int64_t ld_src, __nv_bfloat16* __restrict__ W,
                               const int32_t* done) {
  if (done != nullptr && *done) return;
  const int64_t nq = (ldw + 3) >> 2;
  const int64_t total = rows * nq;
  const int64_t plane = rows_alloc * ldw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nq, q = e - r * nq;
    double z[4];
    if (src == nullptr) {
      uint64_t x0 = (uint64_t)q, x1 = (uint64_t)(row0 + r), x2 = 0, x3 = 0;
      philox4x64_10(x0, x1, x2, x3, seed, 0ull);
      box_muller(x0, x1, z[0], z[1]);
      box_muller(x2, x3, z[2], z[3]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = 4 * q + u;
      if (i >= ldw) break;
      double val = 0.0;
      if (i < m) val = src == nullptr ? z[u] : src[r * ld_src + i];
      double qv = rint(val * 2048.0);
      qv = fmin(fmax(qv, -kQMax), kQMax);
      const double q1 = rint(qv / 256.0);  // |q1| <= 64
      const double q0 = qv - 256.0 * q1;   // |q0| <= 128
      W[r * ldw + i] = __double2bfloat16(q1);
      W[plane + r * ldw + i] = __double2bfloat16(q0);
    }
  }
}

// ------------------------------------------------------------------ host side
// BF16 planes (Omega's digits): 128-byte swizzled boxes of 64 K x box_rows, the MMA's
// layout.  int8 planes (A's digits): plain boxes of 64 K bytes x box_rows, widened
// by the converter warps.
bool make_map_3d(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t planes, int box_rows,
                 int box_planes, bool int8) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  const cuuint64_t esz = int8 ? 1 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)inner * esz, (cuuint64_t)inner * outer * esz};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, int8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            int8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc64

// K padded to 16: the int8 planes' rows must be 16-byte multiples for TMA.
int64_t f64emu_pad(int64_t m) { return (m + 15) / 16 * 16; }
size_t f64emu_digit_bytes(int64_t m, int64_t n) { return (size_t)tc64::kSlices * f64emu_pad(m) * n; }

// Split count of the K range.  One CTA per SM holds a (column tile, split); its
// time is about its chunks (+ a fixed cost), so the launch takes
// waves x (chunks per split + c0).  The count minimising that is taken; it depends
// on (m, n) only, never on how many Omega rows a pass holds.
int f64emu_splits(int64_t m, int64_t n, int sms) {
  const int64_t tiles = (n + tc64::kBM - 1) / tc64::kBM;
  const int64_t chunks = (f64emu_pad(m) + tc64::kChunk - 1) / tc64::kChunk;
  const int64_t s_min = (chunks + tc64::kMaxChunksPerSplit - 1) / tc64::kMaxChunksPerSplit;
  const int64_t s_max = chunks < 64 ? chunks : 64;
  int best = 1;
  double best_t = 1e300;
  for (int64_t s = 1; s <= (s_max > s_min ? s_max : s_min); ++s) {
    const int64_t per = (chunks + s - 1) / s;
    const int64_t eff = (chunks + per - 1) / per;  // splits of whole chunks actually used
    if (eff < s_min || eff != s) continue;
    const int64_t waves = (tiles * eff + sms - 1) / sms;
    const double t = (double)waves * ((double)per + 0.15) + 0.01 * (double)eff;
    if (t < best_t) {
      best_t = t;
      best = (int)eff;
    }
  }
  return best;
}

cudaError_t f64emu_prepare(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* colexp, void* digits,
                           cudaStream_t s) {
  const int64_t mp = f64emu_pad(m);
  tc64::k_colexp<<<(int)(n < 4096 ? n : 4096), 256, 0, s>>>(A, lda, m, n, colexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t blocks = (mp * n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  tc64::k_split_digits<<<(int)blocks, 256, 0, s>>>(A, lda, m, mp, n, colexp, static_cast<int8_t*>(digits));
  return cudaGetLastError();
}

cudaError_t f64_colexp(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* E, cudaStream_t s) {
  tc64::k_colexp<<<(int)(n < 4096 ? n : 4096), 256, 0, s>>>(A, lda, m, n, E);
  return cudaGetLastError();
}

cudaError_t f64emu_omega(uint64_t seed, int64_t row0, int64_t rows, int64_t m, int64_t rows_alloc,
                         const double* src, int64_t ld_src, void* wdigits, const int32_t* done, cudaStream_t s) {
  const int64_t ldw = f64emu_pad(m);
  int64_t blocks = (rows * ((ldw + 3) / 4) + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  tc64::k_omega_digits<<<(int)blocks, 256, 0, s>>>(seed, row0, rows, m, ldw, rows_alloc, src, ld_src,
                                                  static_cast<__nv_bfloat16*>(wdigits), done);
  return cudaGetLastError();
}

cudaError_t f64emu_sketch(const void* digits, const int32_t* colexp, int64_t m, int64_t n, const void* wdigits,
                          int64_t rows, int64_t rows_alloc, double* out, int64_t out_ld, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s) {
  const int64_t mp = f64emu_pad(m);
  CUtensorMap ma, mw;
  if (!tc64::make_map_3d(&ma, digits, mp, n, tc64::kSlices, tc64::kBM, 1, true)) return cudaErrorInvalidValue;
  if (!tc64::make_map_3d(&mw, wdigits, mp, rows_alloc, 2, tc64::kBN, 2, false)) return cudaErrorInvalidValue;
  const int64_t chunks = (mp + tc64::kChunk - 1) / tc64::kChunk;
  const int64_t per = (chunks + splits - 1) / splits;
  const int kchunk = (int)(per * tc64::kChunk);
  const int nz = (int)((mp + kchunk - 1) / kchunk);
  if (nz != splits) return cudaErrorInvalidValue;  // the split-K reduction reads exactly `splits` partials
  const int64_t ytiles = (n + tc64::kBM - 1) / tc64::kBM;
  if (ytiles > 65535 || splits > 65535) return cudaErrorInvalidValue;
  const size_t smem = sizeof(tc64::Smem) + 1024;
  static SmemLimit lim;
  cudaError_t e = raise_smem(tc64::k_sketch_f64emu, smem, lim);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((rows + tc64::kBN - 1) / tc64::kBN), (unsigned)ytiles, (unsigned)nz);
  tc64::k_sketch_f64emu<<<grid, tc64::kThreads, smem, s>>>(ma, mw, colexp, (int)n, (int)rows, (int)mp, kchunk, out,
                                                           out_ld, zstride, st, done);
  return cudaGetLastError();
}

}  // namespace rid
