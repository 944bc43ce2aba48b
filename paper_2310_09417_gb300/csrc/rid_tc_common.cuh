// rid_tc_common.cuh -- inline PTX shared by the tensor-core sketch kernels:
// mbarriers with bounded waits, TMA tile loads, shared-memory matrix and
// instruction descriptors for tcgen05.mma, tensor-memory loads.
//
// Every wait is bounded by %globaltimer (kWaitLimitNs).  mbar_wait gives up
// early once another thread of the launch flagged kErrTimeout; mbar_wait_drain
// ignores the flag so that copies and MMAs already issued complete before a
// CTA frees its tensor memory or exits.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rid_common.cuh"

namespace rid {
namespace tcx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false (kErrTimeout set) after
// kWaitLimitNs, or at once when another thread already flagged a timeout.
static __device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevState* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0u) {
      if (ld_acquire_u32(&st->err) & kErrTimeout) return false;
      if (globaltimer_ns() - t0 > kWaitLimitNs) {
        atomicOr(&st->err, kErrTimeout);
        return false;
      }
    }
  }
  return true;
}
// Wait for copies or MMAs in flight, even after a timeout was flagged; bounded.
static __device__ __noinline__ void mbar_wait_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0u && globaltimer_ns() - t0 > kWaitLimitNs) return;
  }
}

// TMA tile loads (x: innermost coordinate, 16-byte aligned in every caller)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile with 128-byte rows, 128-byte
// swizzle, 8-row groups 1024 bytes apart.  +2 advances 32 bytes along K.
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  const uint64_t a = smem_u32(p);
  uint64_t d = (a >> 4) & 0x3FFFull;  // start address >> 4
  d |= 1ull << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (1024ull >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= 1ull << 46;                    // descriptor version
  d |= 2ull << 61;                    // 128-byte swizzle
  return d;
}
// Instruction descriptors: FP32 accumulator, both operands K-major, M x N.
// kind::f16 with BF16 A and B.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
// kind::f8f6f4 with E4M3 A and B (format code 0 for both operands).
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on `bar` once every tcgen05 operation issued so far by this thread completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
// 16 consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive 32-bit columns of this thread's tensor-memory lane, one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 columns without waiting: the registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// (hi 2^32 + lo) 2^ex as a double, rounded to nearest even, assembled with integer
// operations (GB300 issues about two FP64 instructions per clock per SM).
// hi, lo: any int64 values; results outside the normal range take the FP64 route.
__device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int ex) {
  const __int128 V = ((__int128)hi << 32) + (__int128)lo;
  if (V == 0) return 0.0;
  const bool neg = V < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)(-V) : (unsigned __int128)V;
  const unsigned long long h = (unsigned long long)(U >> 64), l = (unsigned long long)U;
  int msb = h ? 127 - __clzll((long long)h) : 63 - __clzll((long long)l);
  const int sh = msb - 52;
  unsigned long long mant;
  if (sh > 0) {
    mant = (unsigned long long)(U >> sh);
    const unsigned __int128 rem = U & (((unsigned __int128)1 << sh) - 1);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++msb;
      }
    }
  } else {
    mant = (unsigned long long)(U << (-sh));
  }
  const int e = msb + ex + 1023;
  if (e <= 0 || e >= 2047) return ldexp((double)hi + ldexp((double)lo, -32), ex + 32);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)e << 52) |
                                          (mant & ((1ull << 52) - 1))));
}

// w 2^ex as a double, rounded to nearest even, by integer operations on the bit
// pattern (|w| < 2^63); results outside the normal range take the FP64 route.
__device__ __forceinline__ double i64_to_double(long long w, int ex) {
  if (w == 0) return 0.0;
  const unsigned long long sgn = w < 0 ? (1ull << 63) : 0ull;
  const unsigned long long u = w < 0 ? 0ull - (unsigned long long)w : (unsigned long long)w;
  const int lz = __clzll((long long)u);
  const unsigned long long nrm = u << lz;  // bit 63 set
  unsigned long long mant = nrm >> 11;     // 53 bits, leading one at bit 52
  const unsigned rem = (unsigned)(nrm & 0x7ffull);
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  const int e = 1023 + 63 - lz + ex;  // biased exponent of the leading one
  if (e <= 0 || e >= 2046) return ldexp((double)w, ex);
  // the leading one (bit 52 of mant) adds 1 to the field; a carry to 2^53 adds one more
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(e - 1) << 52) + mant)));
}

// w 2^ex as a float, rounded to nearest even, by integer operations (|w| < 2^63);
// results outside the normal range take the FP32 route.
__device__ __forceinline__ float i64_to_float(long long w, int ex) {
  if (w == 0) return 0.0f;
  const unsigned sgn = w < 0 ? 0x80000000u : 0u;
  const unsigned long long u = w < 0 ? 0ull - (unsigned long long)w : (unsigned long long)w;
  const int lz = __clzll((long long)u);
  const unsigned long long nrm = u << lz;               // bit 63 set
  unsigned mant = (unsigned)(nrm >> 40);                // 24 bits, leading one at bit 23
  const unsigned long long rem = nrm & ((1ull << 40) - 1);
  const unsigned long long half = 1ull << 39;
  mant += (rem > half || (rem == half && (mant & 1u))) ? 1u : 0u;
  const int e = 127 + 63 - lz + ex;  // biased exponent of the leading one
  if (e <= 0 || e >= 254) return ldexpf((float)w, ex);
  return __uint_as_float(sgn | (((unsigned)(e - 1) << 23) + mant));
}

// acc += v * 2^SH, exact (v an integer-valued float below 2^24 in magnitude)
template <int SH>
__device__ __forceinline__ void add_scaled(long long& acc, float v) {
  const int iv = __float2int_rn(v);
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(iv), "r"(1 << SH));
}

// ------------------------------------------------------------------ digit slicing
// Fixed-point digit slicing by integer operations on IEEE bit patterns.  For an
// exponent e with |x| < 2^e, F = round(x 2^(8 KD - 1 - e)) (|F| < 2^(8 KD - 1)) is
// written as KD balanced base-256 digits, most significant first:
// x / 2^(e+1) = sum_s d_s 2^(-8(s+1)) + r, |d_s| <= 128, |r| <= 2^(-8 KD - 1).

// e with |x| < 2^e for the largest |x| whose bit pattern (sign cleared) is `bits`; 0 for 0.
__device__ __forceinline__ int exp_above_f64bits(unsigned long long bits) {
  if (bits == 0) return 0;
  const int E = (int)(bits >> 52);
  if (E == 0) return -1074 + (64 - __clzll((long long)bits));  // subnormal: units of 2^-1074
  return E - 1022;
}
__device__ __forceinline__ int exp_above_f32bits(unsigned int bits) {
  if (bits == 0) return 0;
  const int E = (int)(bits >> 23);
  if (E == 0) return -149 + (32 - __clz((int)bits));
  return E - 126;
}

// round(m 2^sh) for m < 2^53, to nearest even; sh <= 63 - 53 keeps it in range
__device__ __forceinline__ unsigned long long scale_round(unsigned long long m, int sh) {
  if (sh >= 0) return m << sh;
  if (sh <= -64) return 0;
  const unsigned long long q = m >> (-sh);
  const unsigned long long r = m - (q << (-sh));
  const unsigned long long half = 1ull << (-sh - 1);
  return q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull);
}

template <int KD>
__device__ __forceinline__ long long fixed_of(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long frac = bits & ((1ull << 52) - 1);
  if (E == 0 && frac == 0) return 0;
  const unsigned long long m = E ? (frac | (1ull << 52)) : frac;  // x = m 2^(E' - 1075)
  const unsigned long long a = scale_round(m, (E ? E : 1) - 1075 + 8 * KD - 1 - e);
  return (bits >> 63) ? -(long long)a : (long long)a;
}
template <int KD>
__device__ __forceinline__ long long fixed_of(float x, int e) {
  const unsigned int bits = (unsigned int)__float_as_int(x);
  const int E = (int)((bits >> 23) & 0xFF);
  const unsigned long long frac = bits & ((1u << 23) - 1);
  if (E == 0 && frac == 0) return 0;
  const unsigned long long m = E ? (frac | (1ull << 23)) : frac;  // x = m 2^(E' - 150)
  const unsigned long long a = scale_round(m, (E ? E : 1) - 150 + 8 * KD - 1 - e);
  return (bits >> 31) ? -(long long)a : (long long)a;
}

// The KD digits of F at d[0], d[plane], ..., d[(KD-1) plane].
template <int KD>
__device__ __forceinline__ void write_digits(long long F, __nv_bfloat16* d, int64_t plane) {
  int dg[KD];
#pragma unroll
  for (int s = KD - 1; s > 0; --s) {
    long long r = F & 255;
    if (r >= 128) r -= 256;  // balanced digit in [-128, 127]
    dg[s] = (int)r;
    F = (F - r) >> 8;  // exact
  }
  dg[0] = (int)F;  // |F| <= 128
#pragma unroll
  for (int s = 0; s < KD; ++s) d[s * plane] = __int2bfloat16_rn(dg[s]);
}

// The KD digits of four consecutive values F[0..3] at d[0..3] of every plane, one
// 8-byte store per plane (d 8-byte aligned).
template <int KD>
__device__ __forceinline__ void write_digits4(const long long* F, __nv_bfloat16* d, int64_t plane) {
  int dg[4][KD];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    long long f = F[e];
#pragma unroll
    for (int s = KD - 1; s > 0; --s) {
      long long r = f & 255;
      if (r >= 128) r -= 256;
      dg[e][s] = (int)r;
      f = (f - r) >> 8;
    }
    dg[e][0] = (int)f;
  }
#pragma unroll
  for (int s = 0; s < KD; ++s) {
    const __nv_bfloat162 lo = __halves2bfloat162(__int2bfloat16_rn(dg[0][s]), __int2bfloat16_rn(dg[1][s]));
    const __nv_bfloat162 hi = __halves2bfloat162(__int2bfloat16_rn(dg[2][s]), __int2bfloat16_rn(dg[3][s]));
    uint2 v;
    v.x = *reinterpret_cast<const unsigned*>(&lo);
    v.y = *reinterpret_cast<const unsigned*>(&hi);
    *reinterpret_cast<uint2*>(d + s * plane) = v;
  }
}

}  // namespace tcx
}  // namespace rid
