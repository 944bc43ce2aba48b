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
// The sketch, per pass: k_sparse_csr builds, once per 128-row tile of A and block
// of Omega, the tile's list for every sketch row r (the tile rows i with a nonzero
// in row r, positive ones first, each part in ascending i: a fixed order, no
// atomics on sums); k_sparse_gather stages a 128-row tile of A in shared memory
// (cp.async, double-buffered, with the next tile's lists) and sums, per sketch row
// and column of A, the listed tile entries, two columns per lane.  A is read once
// per pass; the lists (2 bytes per nonzero) are built once per pass, not once per
// column tile.  Split z of the tiles writes its own partial; the split count
// depends on (m, n) only, so the sums do not depend on how many blocks a pass holds.
//
// FP64 input is summed exactly in integers: GB300 issues about two FP64
// instructions per clock per SM, and each element of A feeds zeta sums.  A is
// converted once per call to fixed point per column (F = round(A 2^(54-e)) for
// |A| < 2^e, an error of at most 2^-55 max|A(:,j)| per term, as the digits of the
// FP64-accurate tensor-core sketch), every entry of the sketch is the exact
// integer sum of +-F (int64 within a tile, 128 bits across tiles and across the
// splits, whose 128-bit partials are added exactly), and one conversion rounds it
// to FP64 (then the scale sqrt(b/zeta), one more rounding).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {

constexpr int kSpT = 128;         // rows of A per tile (one list per tile and block)
constexpr int kSpTW = kSpT / 32;  // mask words per tile
constexpr int kSpThreads = 256;   // eight warps

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
// ------------------------------------------------------------------ per-tile lists
// Record of one (tile, block), in uint16: a head of sparse_csr_head(b) entries,
// head[r] = first list entry of sketch row r (r = 0 .. b; head[b] = the list's
// length) and head[b + 1 + r] = first negative entry of row r, then the list: for
// each tile row i (0 .. kSpT-1) with a nonzero in row r, its byte offset i * esz in
// a staged column of A (esz: bytes per staged element), positive ones first, each
// part in ascending i and padded to a multiple of four entries with kSpT * esz (a
// zero slot past the tile's rows), so the gather reads four entries at a time with
// no remainder.  Head and list are padded to 16-byte multiples.
int sparse_csr_head(int b) { return (2 * b + 1 + 7) / 8 * 8; }
int sparse_csr_rec(int b, int zeta) { return sparse_csr_head(b) + (kSpT * zeta + 6 * b + 7) / 8 * 8; }
size_t sparse_csr_bytes(int64_t m, int blocks, int b, int zeta) {
  return (size_t)((m + kSpT - 1) / kSpT) * blocks * sparse_csr_rec(b, zeta) * 2;
}

// One CTA per (tile, block): the codes of the tile's columns of Omega (Philox, the
// partial Fisher-Yates shuffle), a bit mask per key (row r, sign) over the tile's
// rows, an exclusive scan of the keys' counts, and each entry placed at its key's
// start plus the number of tile rows below it with the same key.
__global__ void __launch_bounds__(kSpThreads)
    k_sparse_csr(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, int esz, int rec, int head,
                 uint16_t* __restrict__ R, const int32_t* done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char cs_raw[];
  uint32_t* mask = reinterpret_cast<uint32_t*>(cs_raw);          // [2b][kSpTW], key = 2 r + negative
  int* woff = reinterpret_cast<int*>(mask + 2 * b * kSpTW);       // [2b][kSpTW]: first position per word
  uint8_t* codes = reinterpret_cast<uint8_t*>(woff + 2 * b * kSpTW);  // [kSpT][zeta]
  const int tid = threadIdx.x;
  const int64_t tile = blockIdx.x;
  const int q = blockIdx.y;
  const int64_t i = tile * kSpT + tid;
  uint16_t* out = R + (tile * blocks + q) * (int64_t)rec;
  for (int e = tid; e < 2 * b * kSpTW; e += kSpThreads) mask[e] = 0u;
  __syncthreads();
  if (tid < kSpT && i < m) {
    uint8_t* c = codes + tid * zeta;
    sparse_column(seed, t0 + q, i, b, zeta, c);
    for (int z = 0; z < zeta; ++z) {
      const int key = 2 * (c[z] & 127) + (c[z] >> 7);
      atomicOr(&mask[key * kSpTW + (tid >> 5)], 1u << (tid & 31));
    }
  }
  __syncthreads();
  if (tid < 32) {
    int carry = 0;
    for (int k0 = 0; k0 < 2 * b; k0 += 32) {
      const int key = k0 + tid;
      int cnt[kSpTW];
      int tot = 0;
#pragma unroll
      for (int w = 0; w < kSpTW; ++w) {
        cnt[w] = key < 2 * b ? __popc(mask[key * kSpTW + w]) : 0;
        tot += cnt[w];
      }
      const int ptot = (tot + 3) & ~3;  // the key's segment, padded to four entries
      int incl = ptot;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (tid >= off) incl += y;
      }
      int base = carry + incl - ptot;
      if (key < 2 * b) {
        out[(key & 1) ? b + 1 + (key >> 1) : (key >> 1)] = (uint16_t)base;
        for (int e = base + tot; e < base + ptot; ++e) out[head + e] = (uint16_t)(kSpT * esz);
#pragma unroll
        for (int w = 0; w < kSpTW; ++w) {
          woff[key * kSpTW + w] = base;
          base += cnt[w];
        }
      }
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (tid == 0) out[b] = (uint16_t)carry;
    for (int e = 2 * b + 1 + tid; e < head; e += 32) out[e] = 0;
  }
  __syncthreads();
  if (tid < kSpT && i < m) {
    const uint8_t* c = codes + tid * zeta;
    const uint32_t below = (1u << (tid & 31)) - 1u;
    for (int z = 0; z < zeta; ++z) {
      const int key = 2 * (c[z] & 127) + (c[z] >> 7);
      const int w = key * kSpTW + (tid >> 5);
      out[head + woff[w] + __popc(mask[w] & below)] = (uint16_t)(tid * esz);
    }
  }
}

cudaError_t sparse_csr(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, int esz, uint16_t* R,
                       const int32_t* done, cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b || blocks < 1 || m < 1) return cudaErrorInvalidValue;
  if (esz != 2 && esz != 4 && esz != 8) return cudaErrorInvalidValue;
  const int64_t tiles = (m + kSpT - 1) / kSpT;
  if (tiles > 0x7FFFFFFFll || blocks > 65535) return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * 2 * b * kSpTW * 4 + (size_t)kSpT * zeta;
  k_sparse_csr<<<dim3((unsigned)tiles, (unsigned)blocks), kSpThreads, smem, s>>>(
      seed, t0, blocks, b, m, zeta, esz, sparse_csr_rec(b, zeta), sparse_csr_head(b), R, done);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ the gather-add
// Staged element, partial-sum and accumulator types: FP32 sums for FP32 and BF16 A
// (two columns per lane); for the fixed-point copy of FP64 A, exact int64 sums
// within a tile (a sketch row takes at most one term per tile row: 128 terms below
// 2^54 each) folded into 128-bit totals (one column per lane).
template <typename TS>
struct SpT;
template <>
struct SpT<float> {
  using Part = float;
  using Acc = float;
  using Out = float;
  static constexpr int C = 2, LDT = kSpT + 1, REGS = 64;
};
template <>
struct SpT<__nv_bfloat16> {
  using Part = float;
  using Acc = float;
  using Out = float;
  static constexpr int C = 2, LDT = kSpT + 2, REGS = 64;  // element pairs stay 4-byte aligned
};
template <>
struct SpT<long long> {
  using Part = long long;
  using Acc = __int128;
  using Out = double;
  static constexpr int C = 1, LDT = kSpT + 1, REGS = 64;
};
// blocks of a pass one CTA sums (its accumulators: TG x RPW x C, at most REGS registers)
template <typename TS, int RPW>
__host__ __device__ constexpr int sp_group() {
  constexpr int per = (int)(sizeof(typename SpT<TS>::Acc) / 4) * RPW * SpT<TS>::C;
  constexpr int g = SpT<TS>::REGS / per;
  return g < 1 ? 1 : (g > 4 ? 4 : g);
}
// the staged element at byte offset o of a column, as its partial-sum type
template <typename TS>
__device__ __forceinline__ typename SpT<TS>::Part sp_val(const unsigned char* col, uint32_t o) {
  const TS x = *reinterpret_cast<const TS*>(col + o);
  if constexpr (sizeof(TS) == 2)
    return __bfloat162float(x);
  else
    return x;
}
__device__ __forceinline__ double i128_to_double(__int128 s, int ex) {
  // |s| < 2^95: s >> 32 fits 64 bits
  return tcx::fixed_to_double((long long)(s >> 32), (long long)(s & (__int128)0xFFFFFFFFll), ex);
}
// One list segment [eb, ee) (a multiple of four entries) of a sketch row, added
// (NEG: subtracted) into the partials sa / sb of the C columns whose staged copies
// start at tl (column c at c kColStride bytes): four entries per 8-byte load, the
// next load issued before the current entries are summed.
template <typename TS, int C, bool NEG>
__device__ __forceinline__ void sp_segment(const uint16_t* lst, int eb, int ee, const unsigned char* tl,
                                           typename SpT<TS>::Part (&sa)[C], typename SpT<TS>::Part (&sb)[C]) {
  using Part = typename SpT<TS>::Part;
  constexpr uint32_t kColStride = 32 * SpT<TS>::LDT * sizeof(TS);
  if (eb >= ee) return;
  uint2 w4 = *reinterpret_cast<const uint2*>(lst + eb);
  for (int e = eb; e < ee; e += 4) {
    const uint2 cur = w4;
    if (e + 4 < ee) w4 = *reinterpret_cast<const uint2*>(lst + e + 4);
    const uint32_t o0 = cur.x & 0xFFFFu, o1 = cur.x >> 16, o2 = cur.y & 0xFFFFu, o3 = cur.y >> 16;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const unsigned char* col = tl + c * kColStride;
      const Part a0 = sp_val<TS>(col, o0), a1 = sp_val<TS>(col, o1);
      const Part a2 = sp_val<TS>(col, o2), a3 = sp_val<TS>(col, o3);
      if constexpr (NEG) {
        sa[c] -= a0;
        sb[c] -= a1;
        sa[c] -= a2;
        sb[c] -= a3;
      } else {
        sa[c] += a0;
        sb[c] += a1;
        sa[c] += a2;
        sb[c] += a3;
      }
    }
  }
}

template <typename TS>
__host__ __device__ constexpr size_t sp_tile_bytes() {
  return ((size_t)2 * 32 * SpT<TS>::C * SpT<TS>::LDT * sizeof(TS) + 15) / 16 * 16;
}

// Split z (tiles [z ktiles, (z+1) ktiles) of A's rows) of the sketch rows of blocks
// [tg0, tg0 + gsize) (gsize <= TG) for the columns [j0, j0 + 32 C).  Per tile (the
// next one and its lists already in flight by cp.async into the other buffers):
// warp w sums the sketch rows r = w + 8q of each block, lane = column, the row's
// positive entries then its negative ones, four list entries per 8-byte load,
// alternately into two partials per column (a fixed order; padding entries read
// the zero slot past the tile's rows).  FP32 output: out[z zstride + j out_ld + row] = sqrt(b/zeta) * sum.
// Fixed point: with one split the rounded FP64 value goes to out; otherwise the
// exact 128-bit sum to parts[z zstride + j out_ld + row].
template <typename TS, int RPW, int TG>
__global__ void __launch_bounds__(kSpThreads, 2)
    k_sparse_gather(int64_t m, int64_t n, const TS* __restrict__ A, int64_t lda, const uint16_t* __restrict__ R,
                    int rec, int head, int b, int blocks, int gsize, int64_t rows, int ktiles,
                    typename SpT<TS>::Out* __restrict__ out, typename SpT<TS>::Acc* __restrict__ parts,
                    int64_t out_ld, int64_t zstride, typename SpT<TS>::Out v, const int32_t* __restrict__ colexp,
                    const int32_t* done) {
  using Part = typename SpT<TS>::Part;
  using Acc = typename SpT<TS>::Acc;
  constexpr int C = SpT<TS>::C, LDT = SpT<TS>::LDT, JT = 32 * C;
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char sg_raw[];
  TS* tiles = reinterpret_cast<TS*>(sg_raw);                                    // [2][JT][LDT]
  uint16_t* recs = reinterpret_cast<uint16_t*>(sg_raw + sp_tile_bytes<TS>());  // [2][gsize][rec]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * JT;
  const int tg0 = blockIdx.y * gsize;
  const int ng = min(gsize, blocks - tg0);
  const int64_t ntiles = (m + kSpT - 1) / kSpT;
  const int64_t it0 = (int64_t)blockIdx.z * ktiles;
  const int64_t it1 = min(ntiles, it0 + ktiles);
  Acc acc[TG][RPW][C];
#pragma unroll
  for (int t = 0; t < TG; ++t)
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[t][q][c] = Acc(0);

  // tile it of A (a warp per column, lanes along the rows) and the group's lists
  auto issue = [&](int64_t it, int bf) {
    const int64_t i0 = it * kSpT;
    for (int jj = wid; jj < JT; jj += kSpThreads / 32) {
      const int64_t j = j0 + jj;
      TS* dst = tiles + ((size_t)bf * JT + jj) * LDT;
      const TS* src = A + (j < n ? j : 0) * lda + i0;
      if constexpr (sizeof(TS) == 2) {  // BF16 pairs
#pragma unroll
        for (int q = 0; q < kSpT / 64; ++q) {
          const int ii = 2 * (lane + 32 * q);
          const int64_t left = j < n ? m - (i0 + ii) : 0;
          const int bytes = left >= 2 ? 4 : (left == 1 ? 2 : 0);
          cp_async<4>(dst + ii, bytes ? (const void*)(src + ii) : (const void*)A, bytes);
        }
      } else {
#pragma unroll
        for (int q = 0; q < kSpTW; ++q) {
          const int ii = lane + 32 * q;
          const bool in = j < n && i0 + ii < m;
          cp_async<sizeof(TS)>(dst + ii, in ? (const void*)(src + ii) : (const void*)A, in ? (int)sizeof(TS) : 0);
        }
      }
    }
    const uint16_t* rsrc = R + (it * blocks + tg0) * (int64_t)rec;
    uint16_t* rdst = recs + (size_t)bf * gsize * rec;
    const int pieces = ng * rec / 8;  // rec is a multiple of 8 entries (16 bytes)
    for (int e = tid; e < pieces; e += kSpThreads) cp_async<16>(rdst + 8 * e, rsrc + 8 * e, 16);
    cp_async_commit();
  };

  // the zero slot (tile row kSpT) of every staged column, which padding entries read
  if (tid < 2 * JT) tiles[(size_t)tid * LDT + kSpT] = TS(0);
  if (it0 < it1) issue(it0, 0);
  for (int64_t it = it0; it < it1; ++it) {
    const int cur = (int)((it - it0) & 1);
    if (it + 1 < it1) {
      issue(it + 1, cur ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // column lane of this buffer; column lane + 32 c at + 32 c LDT elements
    const unsigned char* tl = reinterpret_cast<const unsigned char*>(tiles + ((size_t)cur * JT + lane) * LDT);
    const uint16_t* rb = recs + (size_t)cur * gsize * rec;
#pragma unroll
    for (int t = 0; t < TG; ++t) {
      if (t < ng) {
        const uint16_t* hd = rb + t * rec;
        const uint16_t* lst = hd + head;
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          const int r = wid + 8 * q;
          if (r < b) {
            const int e0 = hd[r], em = hd[b + 1 + r], e1 = hd[r + 1];
            Part sa[C], sb[C];
#pragma unroll
            for (int c = 0; c < C; ++c) sa[c] = sb[c] = Part(0);
            sp_segment<TS, C, false>(lst, e0, em, tl, sa, sb);
            sp_segment<TS, C, true>(lst, em, e1, tl, sa, sb);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[t][q][c] += (Acc)(sa[c] + sb[c]);
          }
        }
      }
    }
    __syncthreads();
  }
  const int64_t zoff = (int64_t)blockIdx.z * zstride;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int64_t j = j0 + lane + 32 * c;
    if (j >= n) continue;
    const int ex = colexp != nullptr ? colexp[j] - 54 : 0;
#pragma unroll
    for (int t = 0; t < TG; ++t) {
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const int r = wid + 8 * q;
        const int64_t row = (int64_t)(tg0 + t) * b + r;
        if (t >= ng || r >= b || row >= rows) continue;
        if constexpr (sizeof(Acc) > 8) {
          if (parts != nullptr)
            parts[zoff + j * out_ld + row] = acc[t][q][c];
          else
            out[j * out_ld + row] = i128_to_double(acc[t][q][c], ex) * v;
        } else {
          out[zoff + j * out_ld + row] = acc[t][q][c] * v;
        }
      }
    }
  }
}

// out[j out_ld + c] = sqrt(b/zeta) * (the exact sum over splits of the 128-bit
// partials) 2^(e_j - 54), one rounding to FP64 then the scale.
__global__ void k_sparse_reduce_fixed(int64_t n, int64_t rows, int splits, const __int128* __restrict__ parts,
                                      int64_t pld, int64_t zstride, double* __restrict__ out, int64_t out_ld,
                                      const int32_t* __restrict__ colexp, double v, const int32_t* done) {
  if (done != nullptr && *done) return;
  const int64_t total = n * rows;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, c = e - j * rows;
    __int128 s = 0;
    for (int z = 0; z < splits; ++z) s += parts[z * zstride + j * pld + c];
    out[j * out_ld + c] = i128_to_double(s, colexp[j] - 54) * v;
  }
}

// Split count over A's row tiles for the kind of input (0 FP32, 1 BF16, 2 FP64 in
// fixed point): about four waves of the column tiles at the kind's occupancy;
// depends on (m, n) only.
int sparse_splits(int64_t m, int64_t n, int sms, int kind) {
  const int64_t jt = kind == 2 ? 32 : 64;
  const int64_t per_sm = kind == 2 ? 2 : (kind == 1 ? 3 : 2);
  const int64_t ctiles = (n + jt - 1) / jt;
  const int64_t ktiles = (m + kSpT - 1) / kSpT;
  int64_t s = (4 * per_sm * (int64_t)sms + ctiles - 1) / ctiles;
  if (s > 16) s = 16;
  if (s > ktiles) s = ktiles;
  if (s < 1) s = 1;
  // the count actually used: whole tiles per split
  const int64_t per = (ktiles + s - 1) / s;
  return (int)((ktiles + per - 1) / per);
}

namespace {
template <typename TS, int RPW, int TG>
cudaError_t launch_gather_tg(dim3 grid, size_t smem, int64_t m, int64_t n, const TS* A, int64_t lda,
                             const uint16_t* R, int rec, int b, int blocks, int gsize, int64_t rows, int per,
                             typename SpT<TS>::Out* out, typename SpT<TS>::Acc* parts, int64_t out_ld,
                             int64_t zstride, typename SpT<TS>::Out v, const int32_t* colexp, const int32_t* done,
                             cudaStream_t s) {
  static SmemLimit lim;
  cudaError_t e = raise_smem(k_sparse_gather<TS, RPW, TG>, smem, lim);
  if (e != cudaSuccess) return e;
  k_sparse_gather<TS, RPW, TG><<<grid, kSpThreads, smem, s>>>(m, n, A, lda, R, rec, sparse_csr_head(b), b, blocks,
                                                             gsize, rows, per, out, parts, out_ld, zstride, v, colexp,
                                                             done);
  return cudaGetLastError();
}

template <typename TS, int RPW>
cudaError_t launch_gather(int64_t m, int64_t n, const TS* A, int64_t lda, const uint16_t* R, int zeta, int b,
                          int64_t rows, int splits, typename SpT<TS>::Out* out, typename SpT<TS>::Acc* parts,
                          int64_t out_ld, int64_t zstride, const int32_t* colexp, const int32_t* done,
                          cudaStream_t s) {
  constexpr int TG = sp_group<TS, RPW>();
  constexpr int JT = 32 * SpT<TS>::C;
  const int blocks = (int)((rows + b - 1) / b);
  const int rec = sparse_csr_rec(b, zeta);
  // blocks per CTA: up to TG, while two CTAs still fit an SM (one CTA at least)
  const size_t tb = sp_tile_bytes<TS>(), per_block = (size_t)2 * rec * 2;
  const size_t budget = 113 * 1024;
  int gsize = TG;
  while (gsize > 1 && tb + gsize * per_block > budget) --gsize;
  if (gsize > blocks) gsize = blocks;
  const size_t smem = tb + gsize * per_block;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int64_t ktiles = (m + kSpT - 1) / kSpT;
  const int per = (int)((ktiles + splits - 1) / splits);
  const int64_t groups = (blocks + gsize - 1) / gsize;
  const int64_t ctiles = (n + JT - 1) / JT;
  if (groups > 65535 || splits > 65535 || ctiles > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  dim3 grid((unsigned)ctiles, (unsigned)groups, (unsigned)splits);
  const typename SpT<TS>::Out v = (typename SpT<TS>::Out)sqrt((double)b / (double)zeta);
  // one block per CTA (the usual pass) runs a variant without the group loop
  if (gsize == 1)
    return launch_gather_tg<TS, RPW, 1>(grid, smem, m, n, A, lda, R, rec, b, blocks, gsize, rows, per, out, parts,
                                        out_ld, zstride, v, colexp, done, s);
  return launch_gather_tg<TS, RPW, TG>(grid, smem, m, n, A, lda, R, rec, b, blocks, gsize, rows, per, out, parts,
                                       out_ld, zstride, v, colexp, done, s);
}

template <typename TS>
cudaError_t dispatch_gather(int64_t m, int64_t n, const TS* A, int64_t lda, const uint16_t* R, int zeta, int b,
                            int64_t rows, int splits, typename SpT<TS>::Out* out, typename SpT<TS>::Acc* parts,
                            int64_t out_ld, int64_t zstride, const int32_t* colexp, const int32_t* done,
                            cudaStream_t s) {
  if (b < 1 || b > kSparseMaxB || zeta < 1 || zeta > b || rows < 1 || splits < 1) return cudaErrorInvalidValue;
#define RID_GATHER(P) \
  launch_gather<TS, P>(m, n, A, lda, R, zeta, b, rows, splits, out, parts, out_ld, zstride, colexp, done, s)
  if (b <= 16) return RID_GATHER(2);
  if (b <= 32) return RID_GATHER(4);
  if (b <= 64) return RID_GATHER(8);
  return RID_GATHER(16);
#undef RID_GATHER
}
}  // namespace

template <typename TA>
cudaError_t sparse_sketch(int64_t m, int64_t n, const TA* A, int64_t lda, const uint16_t* R, int zeta, int b,
                          int64_t rows, int splits, float* out, int64_t out_ld, int64_t zstride, const int32_t* done,
                          cudaStream_t s) {
  // the tile is staged in A's own type; BF16 pairs need 4-byte aligned columns
  if constexpr (sizeof(TA) == 2) {
    if ((lda & 1) != 0 || (reinterpret_cast<uintptr_t>(A) & 3) != 0) return cudaErrorInvalidValue;
  }
  return dispatch_gather<TA>(m, n, A, lda, R, zeta, b, rows, splits, out, nullptr, out_ld, zstride, nullptr, done,
                             s);
}

cudaError_t sparse_sketch_fixed(int64_t m, int64_t n, const long long* F, const int32_t* colexp, const uint16_t* R,
                                int zeta, int b, int64_t rows, int splits, double* out, int64_t out_ld, void* parts,
                                int64_t pld, int64_t zstride, const int32_t* done, cudaStream_t s) {
  if (splits == 1)
    return dispatch_gather<long long>(m, n, F, m, R, zeta, b, rows, 1, out, nullptr, out_ld, 0, colexp, done, s);
  __int128* P = static_cast<__int128*>(parts);
  cudaError_t e = dispatch_gather<long long>(m, n, F, m, R, zeta, b, rows, splits, nullptr, P, pld, zstride, colexp,
                                             done, s);
  if (e != cudaSuccess) return e;
  int64_t g = (n * rows + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  k_sparse_reduce_fixed<<<(int)g, 256, 0, s>>>(n, rows, splits, P, pld, zstride, out, out_ld, colexp,
                                                sqrt((double)b / (double)zeta), done);
  return cudaGetLastError();
}

template cudaError_t sparse_sketch<float>(int64_t, int64_t, const float*, int64_t, const uint16_t*, int, int, int64_t,
                                          int, float*, int64_t, int64_t, const int32_t*, cudaStream_t);
template cudaError_t sparse_sketch<__nv_bfloat16>(int64_t, int64_t, const __nv_bfloat16*, int64_t, const uint16_t*,
                                                  int, int, int64_t, int, float*, int64_t, int64_t, const int32_t*,
                                                  cudaStream_t);
template cudaError_t sparse_dense<double>(uint64_t, int64_t, int, int, int64_t, int, double*, int64_t, cudaStream_t);
template cudaError_t sparse_dense<float>(uint64_t, int64_t, int, int, int64_t, int, float*, int64_t, cudaStream_t);

}  // namespace rid
