// rid_batched.cu -- many independent adaptive column IDs (Algorithm 1) in one
// persistent launch.  The paper lists batched low-rank approximation as future
// work (Sec. 6, item 3); the target workload is the off-diagonal blocks of a
// hierarchical kernel matrix: thousands of problems of uneven sizes.
//
// One CTA runs one problem at a time and pulls the next one from an atomic work
// queue (problems ordered by decreasing m*n, so that the long ones start first).
// Inside a CTA every step of the method runs with CTA-local synchronisation only:
// Gaussian rows, sketch (CTA GEMM), Schur complement + FP64 norm, the stop test,
// LUPP of the panel (staged in shared memory when it fits), the inverse of the
// new unit-lower block, the interpolation-matrix update and the re-blocking of
// the index lists -- the same arithmetic as the single-problem path.
// The queue reset and the persistent kernel are replayed from a CUDA graph; the
// output-tile height of the CTA GEMM and the CTAs per SM come from a small
// autotuner that times the candidates on the largest problems of the batch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "randid.h"
#include "rid_internal.h"

namespace rid {
namespace bat {

constexpr int kNT = 512;     // threads per CTA
constexpr int kTN = 32;      // CTA GEMM tile width
constexpr int kTK = 32;      // CTA GEMM K step
constexpr int kMaxB = 32;    // largest block size of the batched path
constexpr int kMaxN = 4096;  // largest n (selection flags live in shared memory)

struct Problem {
  const void* A;
  int64_t lda;
  int64_t* J;
  void* X;
  int64_t ldx;
  double* pivots;
  int32_t m, n, cap, pad;
};

struct Result {
  int64_t k;
  double est;
  double norm_A;
  int32_t rounds;
  int32_t status;
};

struct Params {
  const Problem* probs;
  const int32_t* order;
  int count;
  int* queue;
  Result* results;
  DevState* st;
  unsigned char* slots;
  size_t slot_bytes;
  int64_t mmax, nmax;
  int b;
  double tol;
  int tol_rel;
  uint64_t seed;
  int stage_panel;  // 1: the LUPP panel is staged in shared memory
};

// Per-CTA scratch slot (one slot per resident CTA).
template <typename T>
struct Slot {
  T* omega;  // b x mmax, row-major
  T* G;      // nmax x b
  T* S;      // nmax x b
  T* N;      // nmax x b
  int32_t* act[2];
  int32_t* perm;
  int32_t* mark;
};

__host__ __device__ inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
size_t slot_bytes(int64_t mmax, int64_t nmax, int b) {
  return al(sizeof(T) * b * mmax) + 3 * al(sizeof(T) * nmax * b) + 4 * al(4 * nmax);
}

template <typename T>
__device__ Slot<T> slot_at(const Params& p) {
  unsigned char* base = p.slots + blockIdx.x * p.slot_bytes;
  Slot<T> s;
  size_t off = 0;
  s.omega = reinterpret_cast<T*>(base + off);
  off += al(sizeof(T) * p.b * p.mmax);
  s.G = reinterpret_cast<T*>(base + off);
  off += al(sizeof(T) * p.nmax * p.b);
  s.S = reinterpret_cast<T*>(base + off);
  off += al(sizeof(T) * p.nmax * p.b);
  s.N = reinterpret_cast<T*>(base + off);
  off += al(sizeof(T) * p.nmax * p.b);
  s.act[0] = reinterpret_cast<int32_t*>(base + off);
  off += al(4 * p.nmax);
  s.act[1] = reinterpret_cast<int32_t*>(base + off);
  off += al(4 * p.nmax);
  s.perm = reinterpret_cast<int32_t*>(base + off);
  off += al(4 * p.nmax);
  s.mark = reinterpret_cast<int32_t*>(base + off);
  return s;
}

// Shared memory of one CTA (dynamic): GEMM tiles, then the panel stage.
template <typename T, int BM>
struct Shared {
  T As[kTK * (BM + 1)];
  T Bs[kTK * (kTN + 1)];
  T Lp[kMaxB * kMaxB];
  T Li[kMaxB * kMaxB];
  T prow[kMaxB];
  double pdiag[kMaxB];
  int32_t piv[kMaxB];
  int32_t pivorig[kMaxB];
  unsigned char sel[kMaxN];
  int32_t warp_tot[kNT / 32];
  double red;
  int problem;
  int base;
};

// ------------------------------------------------------------------ CTA GEMM
// C (M x N) = sum_k A_r[k] B(k, c); A row r at abase + (aidx ? aidx[r] : r) * lda;
// B K-major (row c at bbase + idx*ldb + boff, contiguous in k) or N-major (row k
// contiguous in c).  mode 0: out[r*ldo + c] = acc; mode 1: out[oidx[r]*ldo + c]
// -= acc unless skip[r].  Every output accumulates over k in increasing order,
// whatever BM is, so the tile choice does not change the result.
template <typename T, int BM, bool BK>
__device__ void cta_gemm(int M, int N, int K, const T* abase, int64_t lda, const int32_t* aidx, const T* bbase,
                         int64_t ldb, const int32_t* bidx, int64_t boff, int mode, T* out, int64_t ldo,
                         const int32_t* oidx, const int32_t* skip, T* As, T* Bs) {
  constexpr int TM = BM / 16;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  for (int m0 = 0; m0 < M; m0 += BM)
    for (int n0 = 0; n0 < N; n0 += kTN) {
      T acc[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) acc[i] = T(0);
      for (int k0 = 0; k0 < K; k0 += kTK) {
        for (int e = tid; e < BM * kTK; e += kNT) {
          const int r = e / kTK, kk = e - r * kTK, row = m0 + r, k = k0 + kk;
          T v = T(0);
          if (row < M && k < K) v = abase[(int64_t)(aidx ? aidx[row] : row) * lda + k];
          As[kk * (BM + 1) + r] = v;
        }
        if (BK) {
          for (int e = tid; e < kTN * kTK; e += kNT) {
            const int c = e / kTK, kk = e - c * kTK, col = n0 + c, k = k0 + kk;
            T v = T(0);
            if (col < N && k < K) v = bbase[(int64_t)(bidx ? bidx[col] : col) * ldb + boff + k];
            Bs[kk * (kTN + 1) + c] = v;
          }
        } else {
          for (int e = tid; e < kTK * kTN; e += kNT) {
            const int kk = e / kTN, c = e - kk * kTN, col = n0 + c, k = k0 + kk;
            T v = T(0);
            if (col < N && k < K) v = bbase[(int64_t)(bidx ? bidx[k] : k) * ldb + boff + col];
            Bs[kk * (kTN + 1) + c] = v;
          }
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kTK; ++kk) {
          const T bv = Bs[kk * (kTN + 1) + tx];
#pragma unroll
          for (int i = 0; i < TM; ++i) acc[i] = fma(As[kk * (BM + 1) + ty + 16 * i], bv, acc[i]);
        }
        __syncthreads();
      }
      const int c = n0 + tx;
      if (c < N) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int r = m0 + ty + 16 * i;
          if (r >= M) continue;
          if (mode == 0) {
            out[(int64_t)r * ldo + c] = acc[i];
          } else if (skip == nullptr || skip[r] == 0) {
            out[(int64_t)(oidx ? oidx[r] : r) * ldo + c] -= acc[i];
          }
        }
      }
    }
}

template <typename T>
__device__ __forceinline__ T from_d(double x) {
  return static_cast<T>(x);
}

// ------------------------------------------------------------------ one problem
template <typename T, int BM>
__device__ void run_problem(const Params& p, const Problem& pr, Result& res, Slot<T>& sl, Shared<T, BM>& sh,
                            T* stage) {
  const int tid = threadIdx.x;
  const int m = pr.m, n = pr.n, b = p.b, cap = pr.cap;
  const T* A = static_cast<const T*>(pr.A);
  T* X = static_cast<T*>(pr.X);
  const int64_t lda = pr.lda, ldx = pr.ldx;
  // ||A||_F^2 and finiteness
  // (FP32: exact squares in float-float, folded into FP64 every 64 terms -- GB300
  // issues about two FP64 instructions per clock per SM, and per-element FP64 work
  // cost more than this kernel's FP32 arithmetic)
  double acc = 0.0;
  bool finite = true;
  if constexpr (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    int cnt = 0;
    for (int j = 0; j < n; ++j)
      for (int i = tid; i < m; i += kNT) {
        sq_add_f32(static_cast<float>(A[(int64_t)j * lda + i]), hi, lo, acc, finite);
        if (++cnt == 64) {
          acc += (double)hi + (double)lo;
          hi = lo = 0.f;
          cnt = 0;
        }
      }
    acc += (double)hi + (double)lo;
  } else {
    for (int64_t e = tid; e < (int64_t)m * n; e += kNT) {
      const int64_t j = e / m, i = e - j * m;
      const double v = static_cast<double>(A[j * lda + i]);
      finite = finite && isfinite(v);
      acc += v * v;
    }
  }
  const int bad = __syncthreads_or(!finite);
  const double n2 = block_sum(acc);
  if (tid == 0) sh.red = n2;
  __syncthreads();
  const double norm2 = sh.red;
  __syncthreads();
  if (bad) {
    if (tid == 0) {
      res.k = 0;
      res.est = 0.0;
      res.norm_A = 0.0;
      res.rounds = 0;
      res.status = ID_ERR_NONFINITE;
    }
    return;
  }
  const double thr = p.tol_rel ? p.tol * sqrt(norm2) : p.tol;
  for (int i = tid; i < n; i += kNT) {
    sl.act[0][i] = i;
    sl.mark[i] = 0;
  }
  __syncthreads();
  int tb = 0, na = n, t = 0, cur = 0, rounds = 0, status = ID_OK;
  unsigned zeros = 0;
  double est = 0.0;
  int64_t k = 0;
  for (;;) {
    // Gaussian rows [t*b, t*b + b) of Omega (same counters as the single-problem path)
    // (32-bit indices: a 64-bit division is an FP64-pipe routine on GB300)
    const int nq = (m + 3) / 4;
    for (int e = tid; e < b * nq; e += kNT) {
      const int i = e / nq, q = e - i * nq;
      uint64_t x0 = (uint64_t)q, x1 = (uint64_t)((int64_t)t * b + i), x2 = 0, x3 = 0;
      philox4x64_10(x0, x1, x2, x3, p.seed, 0ull);
      T* o = sl.omega + (int64_t)i * p.mmax + 4 * q;
      if constexpr (sizeof(T) == 4) {  // FP32: the FP32 evaluation of the same map
        float f[4];
        box_muller_f32_53(x0, x1, f[0], f[1]);
        box_muller_f32_53(x2, x3, f[2], f[3]);
        for (int j = 0; j < 4 && 4 * q + j < m; ++j) o[j] = f[j];
      } else {
        double z[4];
        box_muller(x0, x1, z[0], z[1]);
        box_muller(x2, x3, z[2], z[3]);
        for (int j = 0; j < 4 && 4 * q + j < m; ++j) o[j] = from_d<T>(z[j]);
      }
    }
    __syncthreads();
    // sketch G (n x b) = (Omega A)^T
    cta_gemm<T, BM, true>(n, b, m, A, lda, nullptr, sl.omega, p.mmax, nullptr, 0, 0, sl.G, b, nullptr, nullptr,
                          sh.As, sh.Bs);
    __syncthreads();
    // Schur complement S = G(act) - T(act, 0:tb) G(perm) and its FP64 norm
    if (tb > 0) {
      cta_gemm<T, BM, false>(na, b, tb, X, ldx, sl.act[cur], sl.G, b, sl.perm, 0, 0, sl.S, b, nullptr, nullptr,
                             sh.As, sh.Bs);
      __syncthreads();
    }
    double e2 = 0.0;
    {
      float hi = 0.f, lo = 0.f;
      bool fin = true;
      int cnt = 0;
      for (int e = tid; e < na * b; e += kNT) {
        const int i = e / b, c = e - i * b;
        T v = sl.G[(int64_t)sl.act[cur][i] * b + c];
        if (tb > 0) v -= sl.S[(int64_t)i * b + c];
        sl.S[(int64_t)i * b + c] = v;
        if constexpr (sizeof(T) == 4) {
          sq_add_f32(v, hi, lo, e2, fin);
          if (++cnt == 64) {
            e2 += (double)hi + (double)lo;
            hi = lo = 0.f;
            cnt = 0;
          }
        } else {
          e2 += static_cast<double>(v) * static_cast<double>(v);
        }
      }
      if constexpr (sizeof(T) == 4) e2 += (fin ? (double)hi + (double)lo : (double)INFINITY);
    }
    e2 = block_sum(e2);
    if (tid == 0) sh.red = e2;
    __syncthreads();
    e2 = sh.red;
    __syncthreads();
    if (t > 0) {
      est = sqrt(e2 / (double)b);
      ++rounds;
      if (est <= thr) {
        k = tb;
        break;
      }
      if (tb == cap) {
        k = tb;
        status |= ID_WARN_TOL_NOT_MET;
        break;
      }
    }
    const int bt = min(b, cap - tb);
    // LUPP of S (na x b) for bt pivots: rows are marked, not swapped
    T* R = stage != nullptr ? stage : sl.S;
    const int ldr = stage != nullptr ? b + 1 : b;
    if (stage != nullptr)
      for (int e = tid; e < na * b; e += kNT) {
        const int i = e / b, c = e - i * b;
        R[i * ldr + c] = sl.S[(int64_t)i * b + c];
      }
    for (int i = tid; i < na; i += kNT) sh.sel[i] = 0;
    __syncthreads();
    for (int c = 0; c < bt; ++c) {
      ArgMax a;
      a.v = -1.0;
      a.idx = -1;
      if constexpr (sizeof(T) == 4) {
        // FP32: keys (|v| bit pattern, ~row) compared as integers -- the same choice
        // (largest |v|, ties to the smaller row) without per-element FP64 work
        unsigned long long best = 0ull;
        for (int r = tid; r < na; r += kNT)
          if (!sh.sel[r]) {
            const unsigned long long kk = ((unsigned long long)(__float_as_uint(R[r * ldr + c]) & 0x7FFFFFFFu) << 32) |
                                          (unsigned long long)(0xFFFFFFFFu - (unsigned)r);
            best = kk > best ? kk : best;
          }
        best = block_max_u64(best);
        if (best != 0ull) {
          a.idx = (int)(0xFFFFFFFFu - (unsigned)(best & 0xFFFFFFFFull));
          a.v = (double)__uint_as_float((unsigned)(best >> 32));
        }
      } else {
        for (int r = tid; r < na; r += kNT)
          if (!sh.sel[r]) {
            ArgMax o;
            o.v = static_cast<double>(tabs(R[r * ldr + c]));
            o.idx = r;
            a = argmax_pick(a, o);
          }
        a = block_argmax(a);
      }
      const int pr_ = a.idx;
      const bool zero = !(a.v > 0.0);
      for (int cc = tid; cc < b; cc += kNT) sh.prow[cc] = R[pr_ * ldr + cc];
      if (tid == 0) {
        sh.sel[pr_] = (unsigned char)1;
        sh.piv[c] = pr_;
        sh.pdiag[c] = a.v;
      }
      if (zero) ++zeros;
      __syncthreads();
      if (!zero) {
        const T pv = sh.prow[c];
        for (int r = tid; r < na; r += kNT)
          if (!sh.sel[r]) R[r * ldr + c] = R[r * ldr + c] / pv;
        __syncthreads();
        const int wc = b - c - 1;
        for (int e = tid; e < na * wc; e += kNT) {
          const int r = e / wc, cc = c + 1 + (e - r * wc);
          if (!sh.sel[r]) R[r * ldr + cc] = fma(-R[r * ldr + c], sh.prow[cc], R[r * ldr + cc]);
        }
        __syncthreads();
      }
    }
    if (stage != nullptr)
      for (int e = tid; e < na * b; e += kNT) {
        const int i = e / b, c = e - i * b;
        sl.S[(int64_t)i * b + c] = R[i * ldr + c];
      }
    for (int i = tid; i < na; i += kNT) sl.mark[i] = sh.sel[i];
    __syncthreads();
    // inverse of the new unit-lower block L-hat(piv, 0:bt)
    for (int e = tid; e < bt * bt; e += kNT) {
      const int r = e / bt, c = e - r * bt;
      sh.Lp[e] = c < r ? sl.S[(int64_t)sh.piv[r] * b + c] : (c == r ? T(1) : T(0));
    }
    for (int e = tid; e < bt * bt; e += kNT) sh.Li[e] = (e / bt == e % bt) ? T(1) : T(0);
    __syncthreads();
    // rows in order; each column j of a row summed by 4 threads interleaved over c
    // and a shuffle -- the summation order of the single-problem driver's k_linv
    {
      const int j = tid >> 2, part = tid & 3;
      for (int i = 1; i < bt; ++i) {
        T s = T(0);
        if (j < i)
          for (int c = j + part; c < i; c += 4) s = fma(sh.Lp[i * bt + c], sh.Li[c * bt + j], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (j < i && part == 0) sh.Li[i * bt + j] = -s;
        __syncthreads();
      }
    }
    if (tid < bt) sh.pivorig[tid] = sl.act[cur][sh.piv[tid]];
    __syncthreads();
    // new block of T: N = L-hat(rest) Linv, stored in N and in X(tb:tb+bt, act)
    for (int e = tid; e < na * bt; e += kNT) {
      const int i = e / bt, c = e - i * bt;
      if (sl.mark[i]) continue;
      T s = T(0);
      for (int cp = c; cp < bt; ++cp) s = fma(sl.S[(int64_t)i * b + cp], sh.Li[cp * bt + c], s);
      sl.N[(int64_t)i * bt + c] = s;
      X[(int64_t)sl.act[cur][i] * ldx + tb + c] = s;
    }
    __syncthreads();
    // old columns: T(act, 0:tb) -= N T(piv, 0:tb)
    if (tb > 0) {
      cta_gemm<T, BM, false>(na, tb, bt, sl.N, bt, nullptr, X, ldx, sh.pivorig, 0, 1, X, ldx, sl.act[cur], sl.mark,
                             sh.As, sh.Bs);
      __syncthreads();
    }
    // re-block: append the pivots, drop them from the active list (stable)
    if (tid < bt) {
      const int32_t j = sh.pivorig[tid];
      pr.J[tb + tid] = j;
      sl.perm[tb + tid] = j;
      if (pr.pivots != nullptr) pr.pivots[tb + tid] = sh.pdiag[tid];
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) sh.base = 0;
    __syncthreads();
    for (int start = 0; start < na; start += kNT) {
      const int i = start + tid;
      const bool keep = i < na && sl.mark[i] == 0;
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) sh.warp_tot[warp] = __popc(ball);
      __syncthreads();
      int before = __popc(ball & ((1u << lane) - 1u));
      for (int w = 0; w < warp; ++w) before += sh.warp_tot[w];
      if (keep) sl.act[cur ^ 1][sh.base + before] = sl.act[cur][i];
      __syncthreads();
      if (tid == 0)
        for (int w = 0; w < kNT / 32; ++w) sh.base += sh.warp_tot[w];
      __syncthreads();
    }
    for (int i = tid; i < na; i += kNT) sl.mark[i] = 0;
    cur ^= 1;
    tb += bt;
    na -= bt;
    ++t;
    __syncthreads();
    if (tb == n) {  // every column is a skeleton
      k = n;
      est = 0.0;
      break;
    }
  }
  // X(:, J) = I
  for (int64_t e = tid; e < k * k; e += kNT) {
    const int64_t q = e / k, c = e - q * k;
    X[(int64_t)sl.perm[q] * ldx + c] = q == c ? T(1) : T(0);
  }
  if (zeros) status |= ID_WARN_ZERO_PIVOT;
  if (tid == 0) {
    res.k = k;
    res.est = est;
    res.norm_A = sqrt(norm2);
    res.rounds = rounds;
    res.status = status;
  }
  __syncthreads();
}

template <typename T, int BM, int MINB>
__global__ void __launch_bounds__(kNT, MINB) k_batched(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T, BM>& sh = *reinterpret_cast<Shared<T, BM>*>(smem_raw);
  T* stage = p.stage_panel ? reinterpret_cast<T*>(smem_raw + ((sizeof(Shared<T, BM>) + 15) & ~(size_t)15))
                           : nullptr;
  Slot<T> sl = slot_at<T>(p);
  for (;;) {
    if (threadIdx.x == 0) sh.problem = atomicAdd(p.queue, 1);
    __syncthreads();
    const int q = sh.problem;
    __syncthreads();
    if (q >= p.count) break;
    const int idx = p.order[q];
    run_problem<T, BM>(p, p.probs[idx], p.results[idx], sl, sh, stage);
  }
}

template <typename T, int BM>
size_t shared_bytes(int64_t nmax, int b, bool stage) {
  size_t s = (sizeof(Shared<T, BM>) + 15) & ~(size_t)15;
  if (stage) s += sizeof(T) * nmax * (b + 1);
  return s;
}

// ------------------------------------------------------------------ host side
struct Config {
  int bm;      // 32 or 64
  int per_sm;  // CTAs per SM: 1 or 2
};

template <typename T>
bool stage_fits(int64_t nmax, int b, const Config& c) {
  const size_t budget = c.per_sm == 1 ? 200 * 1024 : 100 * 1024;
  return (c.bm == 64 ? shared_bytes<T, 64>(nmax, b, true) : shared_bytes<T, 32>(nmax, b, true)) <= budget;
}

template <typename T>
cudaError_t launch(const Params& p0, const Config& c, int sms, cudaStream_t s) {
  Params p = p0;
  p.stage_panel = stage_fits<T>(p.nmax, p.b, c) ? 1 : 0;
  const size_t smem = c.bm == 64 ? shared_bytes<T, 64>(p.nmax, p.b, p.stage_panel)
                                 : shared_bytes<T, 32>(p.nmax, p.b, p.stage_panel);
  const int grid = sms * c.per_sm;
  cudaError_t e = cudaMemsetAsync(p.queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  // the shared-memory limit is raised once per kernel variant, device and size
  // (never inside a stream capture: the tuner launches every variant first)
#define RID_BAT_LAUNCH(BM, MINB)                                                                            \
  do {                                                                                                      \
    static SmemLimit lim;                                                                                   \
    e = raise_smem(k_batched<T, BM, MINB>, smem, lim);                                                      \
    if (e != cudaSuccess) return e;                                                                         \
    k_batched<T, BM, MINB><<<grid, kNT, smem, s>>>(p);                                                      \
  } while (0)
  if (c.bm == 64 && c.per_sm == 1) RID_BAT_LAUNCH(64, 1);
  else if (c.bm == 64) RID_BAT_LAUNCH(64, 2);
  else if (c.per_sm == 1) RID_BAT_LAUNCH(32, 1);
  else RID_BAT_LAUNCH(32, 2);
#undef RID_BAT_LAUNCH
  return cudaGetLastError();
}

}  // namespace bat
}  // namespace rid

// ====================================================================== C ABI
namespace {

using rid::bat::Config;
using rid::bat::Params;
using rid::bat::Problem;
using rid::bat::Result;

struct BatchPlan {
  int elem = 8;  // 8: FP64, 4: FP32
  int b = 32;
  int64_t mmax = 0, nmax = 0;
  int sms = 0, slots = 0;
  size_t off_state = 0, off_probs = 0, off_order = 0, off_results = 0, off_queue = 0, off_slots = 0, slot_bytes = 0,
         total = 0;
};

int sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 148;
  return v;
}

size_t alb(size_t x) { return (x + 255) & ~(size_t)255; }

int batch_plan(int64_t count, const id_matrix* A, const id_opts* o, BatchPlan* bp) {
  if (count < 1 || count > (1 << 24)) return -1;
  if (A == nullptr) return -2;
  if (o == nullptr) return -3;
  if (o->omega != nullptr) return -3;  // the batched path draws its own Gaussian rows
  const int64_t b = o->block == 0 ? 32 : o->block;
  if (b < 1 || b > rid::bat::kMaxB || !(o->tol >= 0.0) || o->k_max < 0) return -3;
  id_dtype dt = o->lu_prec;
  if (!((dt == ID_F64 || dt == ID_F32) && o->sketch_prec == dt)) return ID_ERR_UNSUPPORTED;
  bp->elem = dt == ID_F64 ? 8 : 4;
  bp->b = (int)b;
  for (int64_t i = 0; i < count; ++i) {
    const id_matrix& a = A[i];
    if (a.data == nullptr || a.dtype != dt || a.m < 1 || a.n < 1 || a.ld < a.m || a.n > rid::bat::kMaxN ||
        a.m >= ((int64_t)1 << 31))
      return -2;
    bp->mmax = std::max(bp->mmax, a.m);
    bp->nmax = std::max(bp->nmax, a.n);
  }
  bp->sms = sm_count();
  bp->slots = 2 * bp->sms;
  bp->slot_bytes = bp->elem == 8 ? rid::bat::slot_bytes<double>(bp->mmax, bp->nmax, bp->b)
                                 : rid::bat::slot_bytes<float>(bp->mmax, bp->nmax, bp->b);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = alb(off + (bytes ? bytes : 1));
    return at;
  };
  bp->off_state = take(256);
  bp->off_probs = take(sizeof(Problem) * count);
  bp->off_order = take(4 * count);
  bp->off_results = take(sizeof(Result) * count);
  bp->off_queue = take(256);
  bp->off_slots = take(bp->slot_bytes * bp->slots);
  bp->total = off;
  return ID_OK;
}

// Graph cache: the queue reset and the persistent kernel, captured once per
// (workspace, parameters, configuration) and replayed.
struct GraphEntry {
  Params p;
  Config c;
  int elem;
  int dev;
  cudaGraphExec_t exec;
};
std::vector<GraphEntry> g_graphs;
// Guards g_graphs, g_tuned and the capture streams: id_batched may be called
// from several host threads at once.  Held across a graph's capture and launch
// so that no entry is evicted (and destroyed) between its lookup and its launch.
std::mutex g_cache_mu;

bool same_params(const Params& a, const Params& b) { return memcmp(&a, &b, sizeof(Params)) == 0; }

cudaStream_t capture_stream(int dev) {
  static cudaStream_t s[64] = {nullptr};
  if (dev < 0 || dev >= 64) return nullptr;
  if (s[dev] == nullptr) cudaStreamCreateWithFlags(&s[dev], cudaStreamNonBlocking);
  return s[dev];
}

cudaError_t run_graph(const Params& p, const Config& c, int elem, int sms, cudaStream_t user) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_cache_mu);
  for (auto& g : g_graphs)
    if (g.dev == dev && g.elem == elem && g.c.bm == c.bm && g.c.per_sm == c.per_sm && same_params(g.p, p))
      return cudaGraphLaunch(g.exec, user);
  cudaStream_t cs = capture_stream(dev);
  if (cs == nullptr) return cudaErrorInvalidResourceHandle;
  cudaGraph_t graph;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = elem == 8 ? rid::bat::launch<double>(p, c, sms, cs) : rid::bat::launch<float>(p, c, sms, cs);
  e = cudaStreamEndCapture(cs, &graph);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  if (g_graphs.size() >= 16) {
    cudaGraphExecDestroy(g_graphs.front().exec);
    g_graphs.erase(g_graphs.begin());
  }
  g_graphs.push_back(GraphEntry{p, c, elem, dev, exec});
  return cudaGraphLaunch(exec, user);
}

// Autotuner: time every configuration on the largest problems of the batch
// (results of these trial runs are overwritten by the real run) and keep the
// fastest per (precision, block, size class).
struct TuneEntry {
  int elem, b, dev;
  int64_t mclass, nclass;
  Config c;
};
std::vector<TuneEntry> g_tuned;

int64_t size_class(int64_t x) {
  int64_t c = 64;
  while (c < x) c *= 2;
  return c;
}

int tune(const Params& p, int elem, int sms, int count, cudaStream_t s, Config* best) {
  int dev = 0;
  cudaGetDevice(&dev);
  // RANDID_BATCHED_CONFIG=<bm>x<per_sm> (e.g. "32x2") pins the configuration (tests)
  if (const char* env = getenv("RANDID_BATCHED_CONFIG")) {
    int bm = 0, per = 0;
    if (sscanf(env, "%dx%d", &bm, &per) == 2 && (bm == 32 || bm == 64) && (per == 1 || per == 2)) {
      *best = Config{bm, per};
      // launch once outside any capture so the variant's shared-memory limit is set
      Params q = p;
      q.count = 0;
      cudaError_t e = elem == 8 ? rid::bat::launch<double>(q, *best, sms, s) : rid::bat::launch<float>(q, *best, sms, s);
      return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
    }
  }
  const int64_t mc = size_class(p.mmax), nc = size_class(p.nmax);
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (auto& t : g_tuned)
      if (t.elem == elem && t.b == p.b && t.dev == dev && t.mclass == mc && t.nclass == nc) {
        *best = t.c;
        return ID_OK;
      }
  }
  const Config cands[4] = {{64, 1}, {64, 2}, {32, 1}, {32, 2}};
  Params q = p;
  q.count = std::min(count, 2 * sms);  // the largest problems come first in `order`
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ID_ERR_CUDA;
  float best_ms = 1e30f;
  *best = cands[0];
  for (const Config& c : cands) {
    cudaEventRecord(e0, s);
    cudaError_t e = elem == 8 ? rid::bat::launch<double>(q, c, sms, s) : rid::bat::launch<float>(q, c, sms, s);
    cudaEventRecord(e1, s);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return ID_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_cache_mu);
  g_tuned.push_back(TuneEntry{elem, p.b, dev, mc, nc, *best});  // two racing tuners may both add: harmless
  return ID_OK;
}

}  // namespace

extern "C" int id_batched_workspace_size(int64_t count, const id_matrix* A, const id_opts* opts, size_t* bytes) {
  if (bytes == nullptr) return -4;
  BatchPlan bp;
  const int rc = batch_plan(count, A, opts, &bp);
  if (rc != ID_OK) return rc;
  *bytes = bp.total;
  return ID_OK;
}

extern "C" int id_batched(int64_t count, const id_matrix* A, const id_opts* opts, void* ws, size_t ws_bytes,
                          id_result* out, void* stream) {
  BatchPlan bp;
  int rc = batch_plan(count, A, opts, &bp);
  if (rc != ID_OK) return rc;
  if (out == nullptr) return -6;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < bp.total) return ID_ERR_WORKSPACE;
  std::vector<Problem> probs(count);
  std::vector<int32_t> order(count);
  for (int64_t i = 0; i < count; ++i) {
    const id_matrix& a = A[i];
    const int64_t kmax = opts->k_max == 0 ? std::min(a.m, a.n) : opts->k_max;
    const int64_t cap = std::min(std::min(a.m, a.n), kmax);
    if (out[i].J == nullptr || out[i].X == nullptr || out[i].ldx < cap) return -6;
    probs[i] = Problem{a.data, a.ld, out[i].J, out[i].X, out[i].ldx, out[i].pivots, (int32_t)a.m, (int32_t)a.n,
                       (int32_t)cap, 0};
    order[i] = (int32_t)i;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return (int64_t)probs[x].m * probs[x].n > (int64_t)probs[y].m * probs[y].n; });
  unsigned char* w = static_cast<unsigned char*>(ws);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(w + bp.off_probs, probs.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(w + bp.off_order, order.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(w + bp.off_state, 0, 256, s) != cudaSuccess)
    return ID_ERR_CUDA;
  Params p;
  memset(&p, 0, sizeof(p));
  p.probs = reinterpret_cast<const Problem*>(w + bp.off_probs);
  p.order = reinterpret_cast<const int32_t*>(w + bp.off_order);
  p.count = (int)count;
  p.queue = reinterpret_cast<int*>(w + bp.off_queue);
  p.results = reinterpret_cast<Result*>(w + bp.off_results);
  p.st = reinterpret_cast<rid::DevState*>(w + bp.off_state);
  p.slots = w + bp.off_slots;
  p.slot_bytes = bp.slot_bytes;
  p.mmax = bp.mmax;
  p.nmax = bp.nmax;
  p.b = bp.b;
  p.tol = opts->tol;
  p.tol_rel = opts->tol_relative;
  p.seed = opts->seed;
  Config c;
  rc = tune(p, bp.elem, bp.sms, (int)count, s, &c);
  if (rc != ID_OK) return rc;
  if (run_graph(p, c, bp.elem, bp.sms, s) != cudaSuccess) return ID_ERR_CUDA;
  std::vector<Result> res(count);
  if (cudaMemcpyAsync(res.data(), w + bp.off_results, sizeof(Result) * count, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ID_ERR_CUDA;
  int worst = ID_OK;
  for (int64_t i = 0; i < count; ++i) {
    out[i].k = res[i].k;
    out[i].est_err = res[i].est;
    out[i].norm_A = res[i].norm_A;
    out[i].rounds = res[i].rounds;
    out[i].passes = res[i].rounds + 1;
    out[i].status = res[i].status;
    out[i].launches = 0;
    for (int ph = 0; ph < ID_NUM_PHASES; ++ph) {
      out[i].phase_ms[ph] = 0.0;
      out[i].phase_launches[ph] = 0;
    }
    if (res[i].status < 0) worst = worst < 0 ? std::min(worst, res[i].status) : res[i].status;
    else if (worst >= 0) worst |= res[i].status;
  }
  if (count > 0) out[0].launches = 2;  // queue reset + the persistent kernel (graph replay)
  return worst;
}
