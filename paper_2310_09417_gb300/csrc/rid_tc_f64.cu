// rid_tc_f64.cu -- an FP64-accurate sketch Y = Omega A on the BF16 tensor cores.
//
// GB300 executes FP64 FMAs at 1.25 TFLOP/s, so the FP64 sketch (Sec. 2.4) is
// moved onto the tensor cores by exact integer slicing:
//   * A: per column j an exponent E_j with max_i |A_ij| < 2^E_j; x = A / 2^(E_j+1)
//     (|x| < 1/2) is written as sum_{s<7} d_s 2^(-8(s+1)) + r with balanced 8-bit
//     digits |d_s| <= 128 and |r| <= 2^-57 -- 56 bits per column.
//   * Omega: standard normal numbers on the grid 2^-11, q = rint(2048 z) clipped to
//     |q| <= 16383, split as q = 256 q1 + q0 with |q1| <= 64, |q0| <= 128.
//   * Every digit is an integer exact in BF16.  Products of equal weight
//     2^(-8g) share one FP32 accumulator group in tensor memory: group g collects
//     q1 x d_g and q0 x d_(g-1) (g = 0..7: 8 groups x 64 columns = the 512 columns
//     of an SM; no product is dropped).  One MMA with N = 128 (both Omega digits
//     stacked) writes groups s and s+1 for slice s.  Over a chunk of 512 K a
//     group's partial sums stay below 512 (128*128 + 64*128) < 2^24: the FP32
//     accumulation is exact.
//   * After slice g of a chunk, group g is final for that chunk; the epilogue
//     warps convert it to integers and add it, exactly, to two int64
//     accumulators per entry (groups 0..3 and 4..7 with weights 2^(8(3-g)) and
//     2^(8(7-g))), then hand the group back to the MMA issuer -- the epilogue
//     of a chunk overlaps the MMAs of the next one.  At the end
//     Y_cj = 2^(E_j - 66) (acc_hi 2^32 + acc_lo), assembled by integer operations.
// Error of an entry: the digit remainders (|r| 2^(E_j+1) <= 2^-55 max_i|A_ij| per
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
constexpr int kDual = 2;          // K steps per stage: one 32 KB box of A (two adjacent tiles) per barrier
constexpr int kStages = 3;        // 3 x (32 KB of A + 32 KB of Omega)
constexpr int kEpiWarps = 8;     // two per TMEM lane quarter, 32 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxChunksPerSplit = 1 << 14;  // int64 accumulators: 2^14 * 2^48 < 2^63
constexpr double kQMax = 16383.0;

using namespace tcx;

// acc += v * 2^sh, exact (v an integer-valued float below 2^23 in magnitude)
struct Smem {
  alignas(1024) __nv_bfloat16 a[kStages][kDual][kBM * kBK];      // one digit slice of A, two K steps: 32 KB
  alignas(1024) __nv_bfloat16 w[kStages][kDual][2 * kBN * kBK];  // both digits of Omega per K step: 32 KB
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t ready[kGroups];  // group g of the current chunk is final
  uint64_t free_[kGroups];  // the epilogue has read group g
  uint64_t drain;
  uint32_t tmem_base;
};
static_assert(sizeof(Smem) + 1024 <= 232448, "shared memory of k_sketch_f64emu exceeds 227 KB");
static_assert(kChunkSteps % kDual == 0, "a stage never straddles an exact chunk");

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
    // ---------------- TMA producer.  Stage order: chunk c, slice s, step pair j/2;
    // each stage holds digit slice s of A at K steps j and j+1 (one box of two
    // adjacent tiles) and both Omega digits at those steps.  Splits start and end on
    // chunk boundaries, so a step j+1 past the chunk only occurs at the end of K,
    // where the boxes read the zero fill past the tensors' extents.
    int it = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int steps_c = min(kChunkSteps, nsteps - c * kChunkSteps);
      for (int s = 0; s < kSlices && ok; ++s) {
        for (int j = 0; j < steps_c; j += kDual, ++it) {
          const int b = it % kStages;
          if (it >= kStages && !mbar_wait(&sm.empty[b], ((it / kStages) + 1) & 1, st)) { ok = false; break; }
          mbar_expect_tx(&sm.full[b], kDual * (kBM + 2 * kBN) * kBK * 2);
          const int k0 = kbeg + (c * kChunkSteps + j) * kBK;
          tma_load_4d(sm.a[b], &map_a, &sm.full[b], 0, 0, k0 / kBK, s * (int)gridDim.y + (int)blockIdx.y);
#pragma unroll
          for (int h = 0; h < kDual; ++h) tma_load_3d(sm.w[b][h], &map_w, &sm.full[b], k0 + h * kBK, n0, 0);
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
        for (int j = 0; j < steps_c; j += kDual, ++it) {
          const int b = it % kStages;
          if (!mbar_wait(&sm.full[b], (it / kStages) & 1, st)) { ok = false; break; }
          fence_after_sync();
          for (int h = 0; h < kDual && j + h < steps_c; ++h) {
            const uint64_t da = desc_sw128(sm.a[b][h]);
            const uint64_t dq1 = desc_sw128(sm.w[b][h]);             // high digit of Omega (weight 1)
            const uint64_t dq0 = desc_sw128(sm.w[b][h] + kBN * kBK);  // low digit (weight 2^-8)
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const bool first = (j + h == 0 && kk == 0);
              if (first && s > 0) {
                // group s continues, group s+1 starts: two MMAs with their own flags
                mma_bf16(dst, da, dq1, id64, 1u);
                mma_bf16(dst + kBN, da, dq0, id64, 0u);
              } else {
                // groups s and s+1 at once (N = 128: q1 rows then q0 rows)
                mma_bf16(dst, da + 2 * kk, dq1 + 2 * kk, id128, (first && s == 0) ? 0u : 1u);
              }
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
        if (i < lim) o[i] = fixed_to_double(hi[i], lo[i], e - 66);
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

// Digits of A(i, j) by integer operations on the FP64 bit patterns
// (x / 2^(E_j+1) = sum_s d_s 2^(-8(s+1))), stored tile by tile: slice s, column
// tile t (kBM columns), K block kb (kBK rows of A) is one contiguous kBM x kBK
// K-major tile, D[s][t][kb][c][k] = d_s(kb kBK + k, t kBM + c).  A TMA box is then
// one 16 KB run of memory (a column-major plane would cost kBM separate 128-byte
// segments per box), and a chunk of one slice is kChunkSteps consecutive tiles.
// Rows past m and columns past n are zero digits.
// A CTA takes whole tiles (the tile's column and K block once per tile, no 64-bit
// division per element); a thread four consecutive k of one column, its digits
// written as 8-byte runs per plane.
__global__ void k_split_digits(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n, int64_t nkb,
                               int64_t ntl, const int32_t* __restrict__ E, __nv_bfloat16* __restrict__ D) {
  constexpr int kTile = kBM * kBK;
  const int64_t tiles = nkb * ntl;
  const int64_t slice = tiles * kTile;
  for (int64_t tb = blockIdx.x; tb < tiles; tb += gridDim.x) {
    const int64_t t = tb / nkb, kb = tb - t * nkb;
    __nv_bfloat16* dt = D + tb * kTile;
    for (int w = 4 * (int)threadIdx.x; w < kTile; w += 4 * (int)blockDim.x) {
      const int64_t j = t * kBM + w / kBK, i = kb * kBK + (w % kBK);
      long long F[4];
      if (j < n) {
        const double* col = A + j * lda;
        const int e = E[j];
#pragma unroll
        for (int q = 0; q < 4; ++q) F[q] = i + q < m ? fixed_of<kSlices>(col[i + q], e) : 0ll;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) F[q] = 0ll;
      }
      write_digits4<kSlices>(F, dt + w, slice);
    }
  }
}

// Omega digits on the grid 2^-11: W[t][r][i], t = 0 high digit q1, t = 1 low digit q0,
// q = rint(2048 z) = 256 q1 + q0 (|q| <= kQMax, q1 = rint(q / 256) ties to even);
// from the Philox/Box-Muller rows (gen) or a caller matrix (src != nullptr).
// Generated rows need z to FP64 accuracy only where 2048 z is near a rounding
// boundary.  Each sample is evaluated in FP32 on the same 53-bit uniforms (a few
// FP32 ulp of z plus about 2^-23 r absolute from the FP64 value: below
// 0.0021 + 0.002 |z| in units of q); a sample whose 2048 z32 lies within
// 1/64 + |z| / 256 of a boundary n + 1/2 goes to its warp's list, and the warp's
// lanes recompute the listed samples in FP64 together.  Every q equals the FP64
// rint.  kGrid: write q / 2048 as FP64 to G (row stride ldg, columns < m) instead
// of the digit planes.
template <bool kGrid>
__device__ __forceinline__ void write_omega_q(int q, __nv_bfloat16* W, int64_t plane, int64_t at, double* G,
                                              int64_t gat) {
  if constexpr (kGrid) {
    G[gat] = (double)q * 0x1.0p-11;
  } else {
    const int t = q + 128;
    int q1 = t >> 8;                         // floor(q / 256 + 1/2)
    if ((t & 255) == 0 && (q1 & 1)) q1 -= 1;  // exact tie: to even
    W[at] = __int2bfloat16_rn(q1);            // |q1| <= 64, exact
    W[plane + at] = __int2bfloat16_rn(q - 256 * q1);  // |q0| <= 128, exact
  }
}
__device__ __forceinline__ int omega_q_f64(double val) {
  const double qv = rint(val * 2048.0);
  return (int)fmin(fmax(qv, -kQMax), kQMax);  // NaN -> -kQMax
}
__device__ __forceinline__ int omega_q_f32(float qf) {
  const int q = __float2int_rn(qf);
  const int lim = (int)kQMax;
  return q < -lim ? -lim : (q > lim ? lim : q);
}

constexpr int kOmegaThreads = 256;
constexpr int kAmbCap = 2048;  // listed samples per CTA: a flush leaves room for one more iteration (<= 1024)

// The listed samples (global element e, sample u of its four: code 4 e + u) are
// recomputed in FP64 by all the CTA's threads together, 256 at a time, so that the
// FP64 Box-Muller (GB300: about two FP64 instructions per clock per SM, a warp
// instruction costing the same whatever its active lanes) runs on full warps.
template <bool kGrid>
__device__ __forceinline__ void omega_flush(const uint64_t* list, int cnt, uint64_t seed, int64_t row0, int64_t nq,
                                            int64_t ldw, int64_t plane, __nv_bfloat16* W, double* G, int64_t ldg) {
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    const uint64_t code = list[k];
    const int u = (int)(code & 3u);
    const int64_t e = (int64_t)(code >> 2), r = e / nq, q = e - r * nq;
    uint64_t x0 = (uint64_t)q, x1 = (uint64_t)(row0 + r), x2 = 0, x3 = 0;
    philox4x64_10(x0, x1, x2, x3, seed, 0ull);
    double z0, z1;
    if (u < 2)
      box_muller(x0, x1, z0, z1);
    else
      box_muller(x2, x3, z0, z1);
    write_omega_q<kGrid>(omega_q_f64((u & 1) ? z1 : z0), W, plane, r * ldw + 4 * q + u, G, r * ldg + 4 * q + u);
  }
}

template <bool kGrid>
__global__ void __launch_bounds__(kOmegaThreads)
    k_omega_digits(uint64_t seed, int64_t row0, int64_t rows, int64_t m, int64_t ldw, int64_t rows_alloc,
                   const double* __restrict__ src, int64_t ld_src, __nv_bfloat16* __restrict__ W,
                   double* __restrict__ G, int64_t ldg, const int32_t* done) {
  if (done != nullptr && *done) return;
  __shared__ uint64_t amb_list[kAmbCap];
  __shared__ int amb_cnt;
  const int64_t nq = (ldw + 3) >> 2;
  const int64_t total = rows * nq;
  const int64_t plane = rows_alloc * ldw;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (threadIdx.x == 0) amb_cnt = 0;
  __syncthreads();
  // CTA-uniform iterations (every thread runs the same count: the flushes synchronise)
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += stride) {
    const int64_t e = base + threadIdx.x;
    const bool valid = e < total;
    const int64_t r = valid ? e / nq : 0, q = valid ? e - r * nq : 0;
    if (src != nullptr) {
      if (valid)
        for (int u = 0; u < 4; ++u) {
          const int64_t i = 4 * q + u;
          if (i >= ldw || (kGrid && i >= m)) break;
          write_omega_q<kGrid>(omega_q_f64(i < m ? src[r * ld_src + i] : 0.0), W, plane, r * ldw + i, G,
                               r * ldg + i);
        }
      continue;
    }
    unsigned amb = 0;  // bit u: sample u goes to the FP64 list
    if (valid) {
      uint64_t x0 = (uint64_t)q, x1 = (uint64_t)(row0 + r), x2 = 0, x3 = 0;
      philox4x64_10(x0, x1, x2, x3, seed, 0ull);
      float zf[4];
      box_muller_f32_53(x0, x1, zf[0], zf[1]);
      box_muller_f32_53(x2, x3, zf[2], zf[3]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = 4 * q + u;
        if (i >= ldw || (kGrid && i >= m)) break;
        if (i >= m) {
          write_omega_q<kGrid>(0, W, plane, r * ldw + i, G, 0);
          continue;
        }
        const float qf = zf[u] * 2048.0f;  // exact (a power of two)
        if (fabsf(qf - floorf(qf) - 0.5f) < 0x1.0p-6f + fabsf(qf) * 0x1.0p-19f)
          amb |= 1u << u;
        else
          write_omega_q<kGrid>(omega_q_f32(qf), W, plane, r * ldw + i, G, r * ldg + i);
      }
    }
    // append this iteration's listed samples: one shared atomic per warp
    const int mine = __popc(amb);
    int incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    int wbase = 0;
    if (lane == 31 && incl > 0) wbase = atomicAdd(&amb_cnt, incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    int at = wbase + incl - mine;
    for (int u = 0; u < 4; ++u)
      if (amb & (1u << u)) amb_list[at++] = ((uint64_t)e << 2) | (uint64_t)u;
    __syncthreads();
    const int cnt = amb_cnt;
    __syncthreads();  // every thread has read the count before the next iteration appends
    if (cnt > kAmbCap - kOmegaThreads * 4) {  // no room for another iteration: recompute now
      omega_flush<kGrid>(amb_list, cnt, seed, row0, nq, ldw, plane, W, G, ldg);
      __syncthreads();
      if (threadIdx.x == 0) amb_cnt = 0;
      __syncthreads();
    }
  }
  __syncthreads();
  omega_flush<kGrid>(amb_list, amb_cnt, seed, row0, nq, ldw, plane, W, G, ldg);
}

// ------------------------------------------------------------------ host side
bool make_map_3d(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t planes, int box_rows,
                 int box_planes) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)inner * 2, (cuuint64_t)inner * outer * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A's digit tiles as a 4-D tensor: (k within the tile, column within the tile,
// K block, slice-major tile index); a box is kDual whole kBK x kBM tiles adjacent
// along K (one contiguous run of memory).
bool make_map_tiles(CUtensorMap* map, const void* base, int64_t kblocks, int64_t tiles) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[4] = {(cuuint64_t)kBK, (cuuint64_t)kBM, (cuuint64_t)kblocks, (cuuint64_t)tiles};
  cuuint64_t strides[3] = {(cuuint64_t)kBK * 2, (cuuint64_t)kBK * kBM * 2, (cuuint64_t)kblocks * kBK * kBM * 2};
  cuuint32_t box[4] = {(cuuint32_t)kBK, (cuuint32_t)kBM, (cuuint32_t)kDual, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc64

int64_t f64emu_pad(int64_t m) { return (m + 7) / 8 * 8; }
namespace {
// Omega generator grid: at most eight 256-thread CTAs per SM, so that each CTA runs
// several iterations and its list of FP64 recomputations fills whole warps.
int64_t omega_blocks(int64_t rows, int64_t ldw) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    sms = 148;
  int64_t blocks = (rows * ((ldw + 3) / 4) + tc64::kOmegaThreads - 1) / tc64::kOmegaThreads;
  if (blocks > 8 * (int64_t)sms) blocks = 8 * (int64_t)sms;
  return blocks < 1 ? 1 : blocks;
}
}  // namespace
namespace {
int64_t digit_kblocks(int64_t m) { return (m + tc64::kBK - 1) / tc64::kBK; }
int64_t digit_tiles(int64_t n) { return (n + tc64::kBM - 1) / tc64::kBM; }
}  // namespace
size_t f64emu_digit_bytes(int64_t m, int64_t n) {
  return (size_t)tc64::kSlices * digit_kblocks(m) * digit_tiles(n) * tc64::kBM * tc64::kBK * 2;
}

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
  tc64::k_colexp<<<(int)(n < 4096 ? n : 4096), 256, 0, s>>>(A, lda, m, n, colexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nkb = digit_kblocks(m), ntl = digit_tiles(n);
  int64_t blocks = nkb * ntl;  // tiles
  if (blocks > 8192) blocks = 8192;
  tc64::k_split_digits<<<(int)blocks, 256, 0, s>>>(A, lda, m, n, nkb, ntl, colexp,
                                                   static_cast<__nv_bfloat16*>(digits));
  return cudaGetLastError();
}

cudaError_t f64_colexp(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* E, cudaStream_t s) {
  tc64::k_colexp<<<(int)(n < 4096 ? n : 4096), 256, 0, s>>>(A, lda, m, n, E);
  return cudaGetLastError();
}

cudaError_t f64emu_omega(uint64_t seed, int64_t row0, int64_t rows, int64_t m, int64_t rows_alloc,
                         const double* src, int64_t ld_src, void* wdigits, const int32_t* done, cudaStream_t s) {
  const int64_t ldw = f64emu_pad(m);
  const int64_t blocks = omega_blocks(rows, ldw);
  tc64::k_omega_digits<false><<<(int)blocks, tc64::kOmegaThreads, 0, s>>>(
      seed, row0, rows, m, ldw, rows_alloc, src, ld_src, static_cast<__nv_bfloat16*>(wdigits), nullptr, 0, done);
  return cudaGetLastError();
}

cudaError_t f64emu_omega_grid(uint64_t seed, int64_t row0, int64_t rows, int64_t m, double* out, int64_t ld,
                              cudaStream_t s) {
  const int64_t ldw = f64emu_pad(m);
  const int64_t blocks = omega_blocks(rows, ldw);
  tc64::k_omega_digits<true><<<(int)blocks, tc64::kOmegaThreads, 0, s>>>(seed, row0, rows, m, ldw, rows, nullptr, 0,
                                                                         nullptr, out, ld, nullptr);
  return cudaGetLastError();
}

cudaError_t f64emu_sketch(const void* digits, const int32_t* colexp, int64_t m, int64_t n, const void* wdigits,
                          int64_t rows, int64_t rows_alloc, double* out, int64_t out_ld, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s) {
  const int64_t mp = f64emu_pad(m);
  CUtensorMap ma, mw;
  if (!tc64::make_map_tiles(&ma, digits, digit_kblocks(m), digit_tiles(n) * tc64::kSlices))
    return cudaErrorInvalidValue;
  if (!tc64::make_map_3d(&mw, wdigits, mp, rows_alloc, 2, tc64::kBN, 2)) return cudaErrorInvalidValue;
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
