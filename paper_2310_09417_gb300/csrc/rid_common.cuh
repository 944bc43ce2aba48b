// rid_common.cuh -- device helpers shared by the ID kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rid {

constexpr int kNumPhases = 6;

// Error bits accumulated on the device (DevState::err).
enum : unsigned {
  kErrTimeout = 1u,   // a bounded wait gave up
  kErrNonFinite = 2u, // NaN or Inf met in the input
  kErrBadIndex = 4u,  // an index argument read on the device was out of range
};

// Device-resident control block at the start of every workspace.  The host
// copies it back at synchronisation points.
struct DevState {
  double norm2_A;         // ||A||_F^2 (FP64 sum)
  double est;             // last estimate E
  double thr;             // stopping threshold tau (absolute)
  int64_t k_final;        // rank when stopped
  int64_t k_pred;         // rank proposed by the learned predictor (0: none)
  int32_t done;           // 1: stop decided -- later speculative kernels exit
  int32_t tol_not_met;    // 1: stopped at the rank cap with E > tau
  int32_t rounds;         // estimates computed
  uint32_t err;           // kErr* bits
  uint32_t zero_pivots;   // exactly zero pivot columns met
  uint32_t bar[2];        // grid-barrier arrival counters, one per launch parity
  uint32_t pad[5];
  unsigned long long pkey[2][3][2];  // LUPP panel: pivot-key maxima, [launch parity][step mod 3][key]
};
static_assert(sizeof(DevState) <= 256, "DevState must fit its 256-byte slot");

// ------------------------------------------------------------------ memory order
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Upper bound on any single device-side wait (nanoseconds).
constexpr uint64_t kWaitLimitNs = 4000000000ull;

__device__ __forceinline__ void red_max_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident) on an
// arrival counter that starts at 0 for the launch: the k-th barrier (k = 0, 1,
// ...) of the launch returns once (k+1) nblocks arrivals were counted.  Thread 0
// of each block adds its arrival with release semantics (covering the block's
// writes, ordered before it by the block barrier) and polls with acquire loads;
// no reset and no second round trip.  The wait is bounded: after kWaitLimitNs
// the block records kErrTimeout and the barrier returns false; callers then
// leave the kernel.  Returns true when every block arrived.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, DevState* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add_u32(ctr, 1u);
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

// ------------------------------------------------------------------ reductions
// (value, index) argmax: larger |value| wins, ties go to the smaller index;
// index < 0 means "no candidate".
struct ArgMax {
  double v;
  int idx;
};
__device__ __forceinline__ ArgMax argmax_pick(ArgMax a, ArgMax b) {
  if (b.idx < 0) return a;
  if (a.idx < 0) return b;
  if (b.v > a.v || (b.v == a.v && b.idx < a.idx)) return b;
  return a;
}
__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ArgMax o;
    o.v = __shfl_down_sync(0xffffffffu, a.v, off);
    o.idx = __shfl_down_sync(0xffffffffu, a.idx, off);
    a = argmax_pick(a, o);
  }
  return a;
}

// Block-wide maximum of 64-bit keys (0 = no candidate), by integer compares.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long k) {
  __shared__ unsigned long long s_k[32];
  __shared__ unsigned long long s_res64;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, k, off);
    k = o > k ? o : k;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_k[warp] = k;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long b = lane < nw ? s_k[lane] : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_down_sync(0xffffffffu, b, off);
      b = o > b ? o : b;
    }
    if (lane == 0) s_res64 = b;
  }
  __syncthreads();
  const unsigned long long r = s_res64;
  __syncthreads();
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum of one double per thread (blockDim.x multiple of 32, <= 1024);
// result valid in thread 0.
// Sum of squares in float-float: t = x * x is exact in FP32 when x has at most 12
// significant bits (BF16, E4M3) and its square is a normal FP32 number; TwoSum
// (Knuth) keeps the rounding error of hi + t in lo, so a group of a few dozen
// squares is summed to about 2^-45 relative before it is folded into FP64.
__device__ __forceinline__ void sq_twosum(float t, float& hi, float& lo) {
  const float s = __fadd_rn(hi, t);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb)));
  hi = s;
}
// x given by its FP32 bit pattern (a BF16 value widened): squares of |x| in
// [2^-63, 2^54) go to the float-float sum (below 2^108 each, so a group of 64 stays
// finite), zeros are skipped, NaN / Inf clear `finite`, the rest (subnormal,
// tiny or huge values) are added in FP64.
__device__ __forceinline__ void sq_add_bits(uint32_t bits, float& hi, float& lo, double& acc, bool& finite) {
  const uint32_t ex = (bits >> 23) & 0xFFu;
  const float x = __uint_as_float(bits);
  if (ex - 64u <= 116u) {
    sq_twosum(__fmul_rn(x, x), hi, lo);
  } else if ((bits << 1) == 0u) {
  } else if (ex == 0xFFu) {
    finite = false;
  } else {
    acc += (double)x * (double)x;
  }
}

// x^2 added to a float-float sum for an FP32 x: the square's rounding error comes
// exactly from an FMA (TwoProduct) and the sum's from TwoSum; |x| outside
// [2^-63, 2^54) (tiny, subnormal, huge) and zeros take the FP64 sum, NaN / Inf
// clear `finite`.  A few dozen squares stay within about 2^-45 relative before
// they are folded into FP64.
__device__ __forceinline__ void sq_add_f32(float x, float& hi, float& lo, double& acc, bool& finite) {
  const uint32_t bits = __float_as_uint(x);
  const uint32_t ex = (bits >> 23) & 0xFFu;
  if (ex - 64u <= 116u) {
    const float p = __fmul_rn(x, x);
    const float e = fmaf(x, x, -p);
    sq_twosum(p, hi, lo);
    lo = __fadd_rn(lo, e);
  } else if ((bits << 1) == 0u) {
  } else if (ex == 0xFFu) {
    finite = false;
  } else {
    acc += (double)x * (double)x;
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_part[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_part[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? s_part[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Block-wide argmax (every thread gets the result); blockDim.x multiple of 32.
__device__ __forceinline__ ArgMax block_argmax(ArgMax a) {
  __shared__ double s_v[32];
  __shared__ int s_i[32];
  __shared__ ArgMax s_res;
  a = warp_argmax(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_v[warp] = a.v;
    s_i[warp] = a.idx;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    ArgMax b;
    b.v = lane < nw ? s_v[lane] : -1.0;
    b.idx = lane < nw ? s_i[lane] : -1;
    b = warp_argmax(b);
    if (lane == 0) s_res = b;
  }
  __syncthreads();
  const ArgMax r = s_res;
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ Gaussian rows
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64
// -> 128-bit products whose high halves are xored into the other words and the
// round key, with the key bumped by two Weyl constants between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t& x3,
                                              uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
    const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
    const uint64_t y0 = hi1 ^ x1 ^ k0;
    const uint64_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Box-Muller on two 53-bit uniforms in (0, 1].
__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, double& z0, double& z1) {
  const double u1 = (double)((a >> 11) + 1ull) * 0x1.0p-53;
  const double u2 = (double)((b >> 11) + 1ull) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

// The same map in FP32 on the leading 24 bits, for outputs of at most 16 bits
// (BF16, E4M3), where the FP64 evaluation buys nothing.
// (float)x rounded to nearest even, for x < 2^63, with integer operations and a
// 32-bit conversion: GB300 executes 64-bit integer-to-float conversions on its
// FP64 pipe (about two per clock per SM), which made them the bottleneck of the
// Gaussian generators.  The result is the same float as the 64-bit conversion.
__device__ __forceinline__ float u64_to_f32_rn(uint64_t x) {
  if (x < (1ull << 24)) return __uint2float_rn((uint32_t)x);  // exact
  const int sh = (64 - __clzll((long long)x)) - 24;            // bits below the 24 kept
  uint64_t q = x >> sh;
  const uint64_t rem = x & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;  // q <= 2^24: exact in FP32
  return __uint2float_rn((uint32_t)q) * __int_as_float((127 + sh) << 23);  // times 2^sh, exact
}

__device__ __forceinline__ void box_muller_f32(uint64_t a, uint64_t b, float& z0, float& z1) {
  const float u1 = __uint2float_rn((uint32_t)((a >> 40) + 1ull)) * 0x1.0p-24f;  // <= 2^24: exact
  const float u2 = __uint2float_rn((uint32_t)((b >> 40) + 1ull)) * 0x1.0p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

// The same map on the same 53-bit uniforms, evaluated in FP32 for FP32 output:
// u1 = n1 2^-53 and x = 2 u2 = n2 2^-52 with n1, n2 in [1, 2^53].
//   ln u1: for u1 >= 1/2 as log1p(-d 2^-53) with d = 2^53 - n1 exact (no cancellation
//          near u1 = 1), else log(u1) (|ln u1| > 0.69, so rounding u1 costs 2^-24
//          relative);
//   the angle: x = x_hi + x_lo with x_hi = x rounded to FP32 (integer rounding of n2)
//          and the exact remainder x_lo; sincos(pi x) from sincospi(x_hi) and a
//          first-order correction (second-order terms below 2^-44).
// Against the FP64 map the result differs by a few FP32 ulp of z plus at most about
// 2^-23 r absolute (r <= 8.6) where cos or sin is near zero.
__device__ __forceinline__ void box_muller_f32_53(uint64_t a, uint64_t b, float& z0, float& z1) {
  const uint64_t n1 = (a >> 11) + 1ull;
  float ln1;
  if (n1 >= (1ull << 52)) {
    const uint64_t d = (1ull << 53) - n1;  // 0 .. 2^52
    ln1 = log1pf(-u64_to_f32_rn(d) * 0x1.0p-53f);
  } else {
    ln1 = logf(u64_to_f32_rn(n1) * 0x1.0p-53f);
  }
  const float r = sqrtf(-2.0f * ln1);
  const uint64_t n2 = (b >> 11) + 1ull;
  // n2 rounded to 24 significant bits, to nearest even, by integer operations
  const int len = 64 - __clzll((long long)n2);
  uint64_t nh = n2;
  if (len > 24) {
    const int sh = len - 24;
    const uint64_t q = n2 >> sh, rem = n2 & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    nh = (q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull)) << sh;
  }
  const float xh = u64_to_f32_rn(nh) * 0x1.0p-52f;                         // exact: nh has 24 bits
  const float t = 3.14159265358979323846f * (__int2float_rn((int32_t)(int64_t)(n2 - nh)) * 0x1.0p-52f);  // pi x_lo
  float sn, cs;
  sincospif(xh, &sn, &cs);
  z0 = r * fmaf(-t, sn, cs);
  z1 = r * fmaf(t, cs, sn);
}

template <typename T>
__device__ __forceinline__ T tabs(T x) {
  return x < T(0) ? -x : x;
}

}  // namespace rid
