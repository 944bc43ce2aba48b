// rid_tc_sketch.cu -- the sketch Y = Omega A on the 5th-generation tensor cores.
//
// G (n x rows) = (Omega A)^T with A (m x n, column-major, BF16) and Omega (rows x m,
// row-major, BF16), FP32 accumulation in tensor memory (Sec. 2.4; the sampling step of Algorithm 1).
// Both operands are K-major (K = m): a column of A and a row of Omega are contiguous.
//
// One CTA computes a 128 (columns of A) x NT BN (rows of Omega) tile over a K range:
//   warp 0   one lane issues TMA loads (128B-swizzled boxes of 64 K x 128 / 64 x up to
//            256 rows of Omega)
//   warp 1   allocates tensor memory; one lane issues tcgen05.mma (M=128, K=16; N=BN
//            for one sub-tile, N=256 over four back-to-back sub-tiles), all reading the
//            same stage of A: a pass of many blocks reads each tile of A once per CTA
//            instead of once per BN rows, and every entry's sums are the same whatever
//            NT is (the same bits for any pass size, checked against one-block passes)
//   warps 2-5 drain the accumulator with tcgen05.ld and write FP32 rows of G
// A STAGES-deep ring of shared-memory stages is guarded by "full" (TMA bytes landed)
// and "empty" (the MMAs that read the stage completed) mbarriers.  Every wait is
// bounded by %globaltimer; on a timeout the CTA records kErrTimeout, waits (bounded)
// for the copies and MMAs it started, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_internal.h"
#include "rid_tc_common.cuh"

namespace rid {

namespace tc {

constexpr int kBM = 128;        // columns of A per tile (MMA M)
constexpr int kBK = 64;         // K per stage: 64 BF16 = one 128-byte swizzle row
// stages per CTA: 4 of (16 + 8 NT) KB, NT = 1 (two CTAs per SM) or 4 sub-tiles of Omega
__host__ __device__ constexpr int stages_for(int) { return 4; }
constexpr int kWBox = 256;     // rows of Omega per TMA box (the box limit)
constexpr int kThreads = 192;   // 6 warps

using namespace tcx;

template <int BN, int NT>
struct Smem {
  static constexpr int kStages = stages_for(NT);
  alignas(1024) __nv_bfloat16 a[kStages][kBM * kBK];      // 16 KB per stage
  alignas(1024) __nv_bfloat16 w[kStages][NT * BN * kBK];  // NT BN * 128 bytes per stage
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accum;
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

// Grid: x = groups of NT BN rows of Omega (fastest, so the CTAs that share a tile of
// A run together and reuse it from L2), y = tiles of A's columns, z = K splits.
template <int BN, int NT>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_tc_bf16(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w, int n,
                     int rows, int K, int kchunk, float* __restrict__ out, int64_t out_ld, int64_t zstride,
                     DevState* st, const int32_t* done) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  if (done != nullptr && *done) return;
  // dynamic shared memory is only guaranteed 16-byte aligned: align the carve-out to 1024
  Smem<BN, NT>& sm =
      *reinterpret_cast<Smem<BN, NT>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kStages = Smem<BN, NT>::kStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM;       // first column of A
  const int n0 = blockIdx.x * NT * BN;   // first row of Omega
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nkb = (kend - kbeg + kBK - 1) / kBK;
  constexpr uint32_t kTmemCols = NT * BN < 32 ? 32 : NT * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.accum, 1);
    mbar_init(&sm.drain, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
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
      mbar_expect_tx(&sm.full[s], (kBM + NT * BN) * kBK * 2);
      const int k0 = kbeg + kb * kBK;
      tma_load_2d(sm.a[s], &map_a, &sm.full[s], k0, m0);
#pragma unroll
      for (int h = 0; h < (NT * BN + kWBox - 1) / kWBox; ++h)  // boxes of at most 256 rows
        tma_load_2d(sm.w[s] + h * kWBox * kBK, &map_w, &sm.full[s], k0, n0 + h * kWBox);
      issued = kb + 1;
    }
    // copies still in flight must land before the CTA can leave
    for (int kb = issued - kStages < 0 ? 0 : issued - kStages; kb < issued; ++kb)
      mbar_wait_drain(&sm.full[kb % kStages], (kb / kStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    constexpr int kNW = NT * BN < 256 ? NT * BN : 256;       // N of one MMA over back-to-back sub-tiles
    constexpr uint32_t idesc_wide = idesc_bf16(kBM, kNW);
    int consumed = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(&sm.full[s], (kb / kStages) & 1, st)) break;
      fence_after_sync();
      const uint64_t da = desc_sw128(sm.a[s]);
      const uint64_t dw = desc_sw128(sm.w[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {  // advance 16 BF16 = 32 bytes inside the swizzle row
        if constexpr (NT > 1) {
          // the sub-tiles lie back to back (BN rows of 128 bytes each): MMAs of N = 256
          // (the same per-entry sums as one MMA per sub-tile, checked bit for bit)
#pragma unroll
          for (int h = 0; h < NT * BN / kNW; ++h)
            mma_bf16(tmem + h * kNW, da + 2 * kk, dw + (uint64_t)((h * kNW * kBK * 2) >> 4) + 2 * kk, idesc_wide,
                     (kb | kk) != 0);
        } else {
#pragma unroll
          for (int t = 0; t < NT; ++t)  // sub-tile t: BN rows of 128 bytes, 1024-byte aligned
            mma_bf16(tmem + t * BN, da + 2 * kk, dw + (uint64_t)((t * BN * kBK * 2) >> 4) + 2 * kk, idesc,
                     (kb | kk) != 0);
        }
      }
      mma_commit(&sm.empty[s]);
      consumed = kb + 1;
    }
    if (consumed == nkb) {
      mma_commit(&sm.accum);
    } else {
      sm.abort = 1;
      mma_commit(&sm.drain);  // wait for the MMAs already issued before tensor memory is freed
      mbar_wait_drain(&sm.drain, 0);
      mma_commit(&sm.accum);  // release the epilogue
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: tensor memory -> G
    const bool ok = mbar_wait(&sm.accum, 0, st);
    fence_after_sync();
    if (ok && !sm.abort) {
      const int quarter = warp & 3;  // warps 2..5 own lane quarters 2,3,0,1
      const int row = m0 + quarter * 32 + lane;
      float* o = out + blockIdx.z * zstride + static_cast<int64_t>(row) * out_ld;
#pragma unroll 1
      for (int c0 = 0; c0 < NT * BN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c0, v);
        if (row < n) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (n0 + c0 + i < rows) o[n0 + c0 + i] = v[i];
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace tc

// ------------------------------------------------------------------ host side

// The driver's cuTensorMapEncodeTiled, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

namespace tc {

// 2-D BF16 tensor map over a K-major matrix: `outer` rows of `inner` contiguous
// elements, row stride `ld` elements; box = 64 (K) x box_rows, 128-byte swizzle.
bool make_map_bf16(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t ld, int box_rows) {
  auto fn = tensor_map_encoder();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int NT>
size_t smem_bytes() {
  static_assert(sizeof(Smem<BN, NT>) + 1024 <= 232448, "shared memory of k_sketch_tc_bf16 exceeds 227 KB");
  return sizeof(Smem<BN, NT>) + 1024;  // + alignment slack
}

}  // namespace tc

bool tc_sketch_supported(const void* A, int64_t lda, const void* W, int64_t ldw) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(A), w = reinterpret_cast<uintptr_t>(W);
  return (a % 16) == 0 && (w % 16) == 0 && (lda % 8) == 0 && (ldw % 8) == 0 && tensor_map_encoder() != nullptr;
}

int tc_sketch_splits(int64_t m, int64_t n, int64_t rows, int sms) {
  const int64_t tiles = ((n + tc::kBM - 1) / tc::kBM) * ((rows + 63) / 64);
  int64_t s = (8 * (int64_t)sms + tiles - 1) / tiles;  // about eight waves of one CTA per SM
  const int64_t kmax = (m + 8 * tc::kBK - 1) / (8 * tc::kBK);  // >= 8 K-stages per CTA
  if (s > kmax) s = kmax;
  if (s > 32) s = 32;
  return (int)(s < 1 ? 1 : s);
}

cudaError_t tc_sketch_bf16(const void* A, int64_t lda, int64_t m, int64_t n, const void* W, int64_t ldw,
                           int64_t rows, float* out, int64_t out_ld, int64_t zstride, int splits, DevState* st,
                           const int32_t* done, cudaStream_t s) {
  constexpr int BN = 64;
  // passes of several blocks: four BN-row sub-tiles of Omega per CTA, and as many
  // CTAs per tile of A as groups of four blocks (they run together, x fastest, and
  // share the tile through L2).  Eight sub-tiles per CTA (two N = 256 MMAs per step,
  // two stages of 80 KB) measured slower: 11.4 against 9.4 ms of sketch per ID at
  // eight blocks per pass, 16.3 against 14.2 ms for one pass of 37 blocks.
  const int nt = rows > BN ? 4 : 1;
  CUtensorMap ma, mw;
  if (!tc::make_map_bf16(&ma, A, m, n, lda, tc::kBM)) return cudaErrorInvalidValue;
  if (!tc::make_map_bf16(&mw, W, m, rows, ldw, nt * BN < tc::kWBox ? nt * BN : tc::kWBox)) return cudaErrorInvalidValue;
  int kchunk = (int)((m + splits - 1) / splits);
  kchunk = ((kchunk + tc::kBK - 1) / tc::kBK) * tc::kBK;
  const int nz = (int)((m + kchunk - 1) / kchunk);
  const int64_t ytiles = (n + tc::kBM - 1) / tc::kBM;
  if (ytiles > 65535 || nz > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((rows + nt * BN - 1) / (nt * BN)), (unsigned)ytiles, (unsigned)nz);
  cudaError_t e;
  if (nt == 4) {
    static SmemLimit lim4;
    e = raise_smem(tc::k_sketch_tc_bf16<BN, 4>, tc::smem_bytes<BN, 4>(), lim4);
    if (e != cudaSuccess) return e;
    tc::k_sketch_tc_bf16<BN, 4><<<grid, tc::kThreads, tc::smem_bytes<BN, 4>(), s>>>(
        ma, mw, (int)n, (int)rows, (int)m, kchunk, out, out_ld, zstride, st, done);
  } else {
    static SmemLimit lim1;
    e = raise_smem(tc::k_sketch_tc_bf16<BN, 1>, tc::smem_bytes<BN, 1>(), lim1);
    if (e != cudaSuccess) return e;
    tc::k_sketch_tc_bf16<BN, 1><<<grid, tc::kThreads, tc::smem_bytes<BN, 1>(), s>>>(
        ma, mw, (int)n, (int)rows, (int)m, kchunk, out, out_ld, zstride, st, done);
  }
  return cudaGetLastError();
}

int tc_sketch_effective_splits(int64_t m, int splits) {
  int kchunk = (int)((m + splits - 1) / splits);
  kchunk = ((kchunk + tc::kBK - 1) / tc::kBK) * tc::kBK;
  return (int)((m + kchunk - 1) / kchunk);
}

}  // namespace rid
