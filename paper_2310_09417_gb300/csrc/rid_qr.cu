// rid_qr.cu -- Householder QR of tall matrices and the products built on it:
// the stable interpolation matrix X = A(:,J)^+ A of the column ID (column form
// of Eq. sID, Sec. 2.2) and the middle factor of a CUR factorisation,
// U = C^+ A R^+ (Sec. 2.2.1), or the two-sided ID's A(I,J)^{-1}.
//
// QR (LAPACK dgeqrf's convention): H_j = I - tau_j v_j v_j^T with v_j(j) = 1,
// R on and above the diagonal, v_j below it.  Panels of 32 columns:
//   * k_qr_panel: one cooperative launch over the panel's rows (staged in shared
//     memory), two bounded grid barriers per column (the column's sum of squares,
//     then the dot products with the later columns of the panel), every
//     reduction summed in block order (deterministic), then V^T V and the
//     compact-WY factor T with H_1 ... H_w = I - V T V^T (Schreiber and Van Loan).
//   * the trailing columns: C2 := C2 - V T^T (V^T C2) through the gather-GEMM
//     (split-K product, reduction times T, rank-32 subtract).
// Q (m x k) is formed explicitly by applying the panels backwards to [I; 0];
// Q^T A is one GEMM; R^{-1} is applied by blocked back substitution (64 x 64
// diagonal blocks inverted explicitly, off-diagonal blocks by GEMM).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "randid.h"
#include "rid_internal.h"

namespace rid {

constexpr int kQrW = 32;          // panel width
constexpr int kQrThreads = 256;
constexpr int kTriB = 64;         // diagonal block of the triangular solve

// ------------------------------------------------------------ panel
// Element (r, c) of the block's rows: shared memory at row stride w + 1, or the
// panel itself (column-major, ld) when the rows do not fit.
template <typename T>
struct PanelRows {
  T* base;
  int64_t rs, cs;
  __device__ __forceinline__ T& operator()(int r, int c) const { return base[r * rs + c * cs]; }
};

template <typename T>
__global__ void __launch_bounds__(kQrThreads)
    k_qr_panel(int mr, int w, T* __restrict__ P, int64_t ld, int chunk, int use_smem, double* __restrict__ pssq,
               double* __restrict__ pdot, double* __restrict__ pgram, T* __restrict__ tau, T* __restrict__ Vc,
               int64_t ldv, T* __restrict__ Tm, unsigned* ctr, DevState* st) {
  extern __shared__ __align__(16) unsigned char qr_raw[];
  __shared__ double s_w[kQrW];
  __shared__ double s_par[3];  // tau, beta, scale
  const int nb = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int r0 = bid * chunk;
  const int nr = max(0, min(mr, r0 + chunk) - r0);
  PanelRows<T> S = use_smem ? PanelRows<T>{reinterpret_cast<T*>(qr_raw), (int64_t)(w + 1), 1}
                            : PanelRows<T>{P + r0, 1, ld};
  if (use_smem)
    for (int e = tid; e < nr * w; e += blockDim.x) {
      const int r = e % nr, c = e / nr;
      S(r, c) = P[(int64_t)(r0 + r) + (int64_t)c * ld];
    }
  __syncthreads();
  unsigned nbar = 0;
  for (int j = 0; j < w; ++j) {
    // 1. the sum of squares of column j below the diagonal over this block's rows
    double acc = 0.0;
    for (int r = tid; r < nr; r += blockDim.x)
      if (r0 + r > j) {
        const double x = (double)S(r, j);
        acc += x * x;
      }
    acc = block_sum(acc);
    if (tid == 0) {
      pssq[((j & 1) * nb + bid) * 2] = acc;
      if (bid == 0) pssq[((j & 1) * nb) * 2 + 1] = (double)S(j, j);  // block 0 owns rows 0 .. w-1
    }
    if (!grid_barrier(ctr, ++nbar * (unsigned)nb, st)) return;
    // 2. the reflector (every block, identically)
    if (tid == 0) {
      double s2 = 0.0;
      for (int b = 0; b < nb; ++b) s2 += __ldcg(&pssq[((j & 1) * nb + b) * 2]);
      const double x0 = __ldcg(&pssq[((j & 1) * nb) * 2 + 1]);
      double t = 0.0, beta = x0, scale = 0.0;
      if (s2 > 0.0) {
        const double nrm = sqrt(x0 * x0 + s2);
        beta = x0 >= 0.0 ? -nrm : nrm;
        t = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
      }
      s_par[0] = t;
      s_par[1] = beta;
      s_par[2] = scale;
    }
    __syncthreads();
    const double t = s_par[0];
    for (int r = tid; r < nr; r += blockDim.x)
      if (r0 + r > j) S(r, j) = (T)((double)S(r, j) * s_par[2]);
    if (bid == 0 && tid == 0) tau[j] = (T)t;
    __syncthreads();
    // 3. the later columns of the panel: w_c = v^T S(:, c), then S(:, c) -= tau v w_c
    if (j + 1 < w && t != 0.0) {
      for (int c = j + 1 + wid; c < w; c += nw) {
        double d = 0.0;
        for (int r = lane; r < nr; r += 32) {
          const int gi = r0 + r;
          if (gi >= j) d += (gi == j ? 1.0 : (double)S(r, j)) * (double)S(r, c);
        }
        d = warp_sum(d);
        if (lane == 0) pdot[((j & 1) * nb + bid) * kQrW + c] = d;
      }
      if (!grid_barrier(ctr, ++nbar * (unsigned)nb, st)) return;
      for (int c = j + 1 + tid; c < w; c += blockDim.x) {
        double d = 0.0;
        for (int b = 0; b < nb; ++b) d += __ldcg(&pdot[((j & 1) * nb + b) * kQrW + c]);
        s_w[c] = d;
      }
      __syncthreads();
      const int ncol = w - j - 1;
      for (int e = tid; e < nr * ncol; e += blockDim.x) {
        const int r = e % nr, c = j + 1 + e / nr;
        const int gi = r0 + r;
        if (gi >= j) {
          const double v = gi == j ? 1.0 : (double)S(r, j);
          S(r, c) = (T)((double)S(r, c) - t * v * s_w[c]);
        }
      }
      __syncthreads();
    }
    if (bid == 0 && tid == 0) S(j, j) = (T)s_par[1];  // R(j, j)
    __syncthreads();
  }
  // 4. V (unit diagonal, zero above) for the GEMMs, V^T V partials, the rows back
  for (int e = tid; e < nr * w; e += blockDim.x) {
    const int r = e % nr, c = e / nr, gi = r0 + r;
    Vc[(int64_t)gi + (int64_t)c * ldv] = gi > c ? S(r, c) : (gi == c ? T(1) : T(0));
  }
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int a = e / w, c = e % w;
    double g = 0.0;
    if (a <= c)
      for (int r = 0; r < nr; ++r) {
        const int gi = r0 + r;
        const double va = gi > a ? (double)S(r, a) : (gi == a ? 1.0 : 0.0);
        const double vc = gi > c ? (double)S(r, c) : (gi == c ? 1.0 : 0.0);
        g += va * vc;
      }
    pgram[(int64_t)bid * kQrW * kQrW + e] = g;
  }
  if (use_smem)
    for (int e = tid; e < nr * w; e += blockDim.x) {
      const int r = e % nr, c = e / nr;
      P[(int64_t)(r0 + r) + (int64_t)c * ld] = S(r, c);
    }
  if (!grid_barrier(ctr, ++nbar * (unsigned)nb, st)) return;
  if (bid != 0) return;
  // 5. T (w x w upper, row-major): T(j,j) = tau_j, T(0:j, j) = -tau_j T(0:j,0:j) V(:,0:j)^T v_j
  __shared__ double G[kQrW][kQrW + 1];
  __shared__ double Ts[kQrW][kQrW + 1];
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int a = e / w, c = e % w;
    double g = 0.0;
    for (int b = 0; b < nb; ++b) g += __ldcg(&pgram[(int64_t)b * kQrW * kQrW + e]);
    G[a][c] = g;
    Ts[a][c] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    const double tj = (double)__ldcg(&tau[j]);
    if (tid < j) {
      double s = 0.0;
      for (int l = tid; l < j; ++l) s += Ts[tid][l] * G[l][j];
      Ts[tid][j] = -tj * s;
    }
    if (tid == 0) Ts[j][j] = tj;
    __syncthreads();
  }
  for (int e = tid; e < w * w; e += blockDim.x) Tm[e] = (T)Ts[e / w][e % w];
}

static size_t qr_panel_smem(int chunk, int w, size_t esz, bool staged) {
  return staged ? (size_t)chunk * (w + 1) * esz : 0;
}

// W2^T (k2 x w, row-major) = (sum_z Wp[z]) T  (trans = 0) or ... T^T (trans = 1).
template <typename T>
__global__ void k_qr_wt(int k2, int w, int nz, int64_t zs, const T* __restrict__ Wp, const T* __restrict__ Tm,
                        int trans, T* __restrict__ W2) {
  const int64_t total = (int64_t)k2 * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / w;
    const int c = (int)(e - r * w);
    T acc = T(0);
    for (int l = 0; l < w; ++l) {
      T s = T(0);
      for (int z = 0; z < nz; ++z) s += Wp[z * zs + r * w + l];
      acc += s * (trans ? Tm[c * w + l] : Tm[l * w + c]);
    }
    W2[e] = acc;
  }
}

// Q := [I_k; 0] (m x k, column-major, ldq).
template <typename T>
__global__ void k_eye(int64_t m, int64_t k, T* __restrict__ Q, int64_t ldq) {
  const int64_t total = m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, i = e - c * m;
    Q[i + c * ldq] = i == c ? T(1) : T(0);
  }
}

// V (unit lower trapezoidal, column-major) of a factored panel.
template <typename T>
__global__ void k_qr_vc(int mr, int w, const T* __restrict__ F, int64_t ld, T* __restrict__ Vc, int64_t ldv) {
  const int64_t total = (int64_t)mr * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / mr, i = e - c * mr;
    Vc[i + c * ldv] = i > c ? F[i + c * ld] : (i == c ? T(1) : T(0));
  }
}

// Gathers: out (rows x cols, column-major, ldo) = A(I, J) with I = null meaning all
// rows 0..rows-1 and J = null all columns; trans = 1 writes the transpose
// (cols x rows).  Indices outside the matrix record kErrBadIndex and read 0.
template <typename T>
__global__ void k_gather2(int64_t rows, int64_t cols, const T* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                          const int64_t* __restrict__ I, const int64_t* __restrict__ J, int trans, T* __restrict__ out,
                          int64_t ldo, DevState* st) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, c;
    if (trans) {  // consecutive threads along the output's rows (= columns of the gather)
      i = e / cols;
      c = e - i * cols;
    } else {
      c = e / rows;
      i = e - c * rows;
    }
    const int64_t gi = I ? I[i] : i, gj = J ? J[c] : c;
    T v = T(0);
    if (gi < 0 || gi >= m || gj < 0 || gj >= n)
      atomicOr(&st->err, kErrBadIndex);
    else
      v = A[gi + gj * lda];
    if (trans)
      out[c + i * ldo] = v;
    else
      out[i + c * ldo] = v;
  }
}

// out (rows x cols, row stride ldo) = in^T for in (cols x rows, row stride ldi).
template <typename T>
__global__ void k_transpose(int64_t rows, int64_t cols, const T* __restrict__ in, int64_t ldi, T* __restrict__ out,
                            int64_t ldo) {
  __shared__ T tile[32][33];
  for (int64_t bi = blockIdx.y * 32; bi < cols; bi += (int64_t)gridDim.y * 32)
    for (int64_t bj = blockIdx.x * 32; bj < rows; bj += (int64_t)gridDim.x * 32) {
      for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int64_t i = bi + q, j = bj + threadIdx.x;
        tile[q][threadIdx.x] = (i < cols && j < rows) ? in[i * ldi + j] : T(0);
      }
      __syncthreads();
      for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int64_t j = bj + q, i = bi + threadIdx.x;
        if (j < rows && i < cols) out[j * ldo + i] = tile[threadIdx.x][q];
      }
      __syncthreads();
    }
}

// R (k x k upper triangle of the factored matrix, column-major, ld) as row-major
// Rrm (k x k, zero below the diagonal) and the inverse of every 64 x 64 diagonal
// block (row-major, block q at Rinv + q * 64 * 64): one CTA per block, column by
// column back substitution in shared memory.
template <typename T>
__global__ void k_tri_blocks(int k, const T* __restrict__ F, int64_t ld, T* __restrict__ Rrm, T* __restrict__ Rinv) {
  __shared__ double Rb[kTriB][kTriB + 1];
  __shared__ double Xb[kTriB][kTriB + 1];
  const int q = blockIdx.x, b0 = q * kTriB, bs = min(kTriB, k - b0);
  // the rows of this block, row-major, zero below the diagonal
  for (int64_t e = threadIdx.x; e < (int64_t)bs * k; e += blockDim.x) {
    const int i = (int)(e / k), c = (int)(e - (int64_t)i * k);
    const int gi = b0 + i;
    Rrm[(int64_t)gi * k + c] = c >= gi ? F[gi + (int64_t)c * ld] : T(0);
  }
  for (int e = threadIdx.x; e < kTriB * kTriB; e += blockDim.x) {
    const int i = e / kTriB, c = e % kTriB;
    Rb[i][c] = (i < bs && c < bs && c >= i) ? (double)F[(b0 + i) + (int64_t)(b0 + c) * ld] : 0.0;
    Xb[i][c] = 0.0;
  }
  __syncthreads();
  // X = Rb^{-1}: column c by back substitution, thread per column
  const int c = threadIdx.x;
  if (c < bs) {
    for (int i = c; i >= 0; --i) {
      double s = i == c ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) s -= Rb[i][l] * Xb[l][c];
      Xb[i][c] = Rb[i][i] != 0.0 ? s / Rb[i][i] : 0.0;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTriB * kTriB; e += blockDim.x)
    Rinv[(int64_t)q * kTriB * kTriB + e] = (T)Xb[e / kTriB][e % kTriB];
}

// ------------------------------------------------------------ host drivers
namespace {

int sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || v <= 0)
    return 148;
  return v;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
int64_t cdv(int64_t a, int64_t b) { return (a + b - 1) / b; }

int grid1(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

// Split-K count for a product with K = depth: about four waves of 64 x 64 tiles.
int qr_splits(int64_t M, int64_t N, int64_t K, int sms) {
  const int64_t tiles = cdv(M, 64) * cdv(N, 64);
  int64_t s = cdv(4 * (int64_t)sms, tiles);
  if (s > K / 256) s = K / 256;
  if (s > 32) s = 32;
  if (s < 1) s = 1;
  return gemm_splits((int)K, (int)s);
}

// Scratch of a QR of an mr x kc matrix: barrier counter and reduction buffers of
// the panel kernel, V of one panel, the split-K partials of V^T C2, W2^T, the T
// factors of every panel and tau.
struct QrScratch {
  int64_t mr = 0, kc = 0;
  int grid = 0, chunk = 0, use_smem = 0, wsplits = 1;
  size_t smem = 0;
  size_t off_ctr, off_ssq, off_dot, off_gram, off_vc, off_wp, off_w2, off_t, off_tau, total;
};

template <typename T>
void qr_layout(int64_t mr, int64_t kc, int sms, QrScratch* q) {
  q->mr = mr;
  q->kc = kc;
  int grid = (int)std::min<int64_t>(sms, cdv(mr, kQrW));
  if (grid < 1) grid = 1;
  int64_t chunk = cdv(mr, grid);
  if (chunk < kQrW) chunk = kQrW;  // block 0 owns the panel's diagonal rows
  grid = (int)cdv(mr, chunk);
  q->grid = grid;
  q->chunk = (int)chunk;
  q->use_smem = qr_panel_smem((int)chunk, kQrW, sizeof(T), true) <= (size_t)200 * 1024;
  q->smem = qr_panel_smem((int)chunk, kQrW, sizeof(T), q->use_smem != 0);
  q->wsplits = qr_splits(kc, kQrW, mr, sms);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = al(off + (b ? b : 1));
    return at;
  };
  q->off_ctr = take(256);
  q->off_ssq = take((size_t)2 * grid * 2 * 8);
  q->off_dot = take((size_t)2 * grid * kQrW * 8);
  q->off_gram = take((size_t)grid * kQrW * kQrW * 8);
  q->off_vc = take((size_t)mr * kQrW * sizeof(T));
  q->off_wp = take((size_t)q->wsplits * kc * kQrW * sizeof(T));
  q->off_w2 = take((size_t)kc * kQrW * sizeof(T));
  q->off_t = take((size_t)cdv(kc, kQrW) * kQrW * kQrW * sizeof(T));
  q->off_tau = take((size_t)kc * sizeof(T));
  q->total = off;
}

// C2 := H C2 (trans = 0: H = I - V T V^T, forming Q) or H^T C2 (trans = 1, the
// factorisation) for C2 (mr x k2, column-major, ld) and the panel's V, T.
template <typename T>
cudaError_t qr_apply(int mr, int w, int k2, T* C2, int64_t ld, const T* Vc, const T* Tm, int trans,
                     const QrScratch& q, unsigned char* ws, cudaStream_t s) {
  if (k2 <= 0) return cudaSuccess;
  T* Wp = reinterpret_cast<T*>(ws + q.off_wp);
  T* W2 = reinterpret_cast<T*>(ws + q.off_w2);
  const int nz = std::min(q.wsplits, qr_splits(k2, w, mr, sm_count()));
  Operand<T> a{C2, ld, nullptr, 0};
  Operand<T> b{Vc, (int64_t)mr, nullptr, 0};
  EpiArgs<T> ep{Wp, w, (int64_t)k2 * w, nullptr, nullptr};
  cudaError_t e = gemm_gather<T>(k2, w, mr, nz, true, a, b, kEpiStore, ep, nullptr, s);
  if (e != cudaSuccess) return e;
  const int nzu = gemm_splits(mr, nz);
  k_qr_wt<T><<<grid1((int64_t)k2 * w), 256, 0, s>>>(k2, w, nzu, (int64_t)k2 * w, Wp, Tm, trans ? 0 : 1, W2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Operand<T> a2{W2, w, nullptr, 0};
  Operand<T> b2{Vc, (int64_t)mr, nullptr, 0};
  EpiArgs<T> ep2{C2, ld, 0, nullptr, nullptr};
  return gemm_gather<T>(k2, mr, w, 1, false, a2, b2, kEpiSubRows, ep2, nullptr, s);
}

// Householder QR in place of F (mr x kc, column-major, ld): R above, V below, the
// T factor of panel p at T + p * 32 * 32.
template <typename T>
cudaError_t qr_factor(int64_t mr, int64_t kc, T* F, int64_t ld, const QrScratch& q, unsigned char* ws, DevState* st,
                      cudaStream_t s) {
  static SmemLimit lim;
  cudaError_t e = cudaSuccess;
  unsigned* ctr = reinterpret_cast<unsigned*>(ws + q.off_ctr);
  double* pssq = reinterpret_cast<double*>(ws + q.off_ssq);
  double* pdot = reinterpret_cast<double*>(ws + q.off_dot);
  double* pgram = reinterpret_cast<double*>(ws + q.off_gram);
  T* Vc = reinterpret_cast<T*>(ws + q.off_vc);
  T* Tall = reinterpret_cast<T*>(ws + q.off_t);
  T* tau = reinterpret_cast<T*>(ws + q.off_tau);
  for (int64_t c0 = 0; c0 < kc; c0 += kQrW) {
    int w = (int)std::min<int64_t>(kQrW, kc - c0);
    int mrp = (int)(mr - c0);
    QrScratch qp;
    qr_layout<T>(mrp, kc, sm_count(), &qp);  // the panel's own grid over its rows
    e = raise_smem(k_qr_panel<T>, qp.smem, lim);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ctr, 0, 256, s);
    if (e != cudaSuccess) return e;
    T* Pp = F + c0 + c0 * ld;
    T* taup = tau + c0;
    T* Tp = Tall + (c0 / kQrW) * kQrW * kQrW;
    int chunk = qp.chunk, use_smem = qp.use_smem;
    int64_t ldl = ld, ldv = mrp;
    void* args[] = {&mrp, &w, &Pp, &ldl, &chunk, &use_smem, &pssq, &pdot, &pgram, &taup, &Vc, &ldv, &Tp, &ctr, &st};
    e = cudaLaunchCooperativeKernel((const void*)k_qr_panel<T>, dim3(qp.grid), dim3(kQrThreads), args, qp.smem, s);
    if (e != cudaSuccess) return e;
    e = qr_apply<T>(mrp, w, (int)(kc - c0 - w), F + c0 + (c0 + w) * ld, ld, Vc, Tp, 1, q, ws, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Q (m x kc, column-major, ldq) from the factored F: panels applied backwards to [I; 0].
template <typename T>
cudaError_t qr_form_q(int64_t mr, int64_t kc, const T* F, int64_t ld, T* Q, int64_t ldq, const QrScratch& q,
                      unsigned char* ws, cudaStream_t s) {
  k_eye<T><<<grid1(mr * kc), 256, 0, s>>>(mr, kc, Q, ldq);
  cudaError_t e = cudaGetLastError();
  T* Vc = reinterpret_cast<T*>(ws + q.off_vc);
  const T* Tall = reinterpret_cast<const T*>(ws + q.off_t);
  for (int64_t c0 = ((kc - 1) / kQrW) * kQrW; e == cudaSuccess && c0 >= 0; c0 -= kQrW) {
    const int w = (int)std::min<int64_t>(kQrW, kc - c0);
    const int mrp = (int)(mr - c0);
    k_qr_vc<T><<<grid1((int64_t)mrp * w), 256, 0, s>>>(mrp, w, F + c0 + c0 * ld, ld, Vc, mrp);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = qr_apply<T>(mrp, w, (int)(kc - c0), Q + c0 + c0 * ldq, ldq, Vc, Tall + (c0 / kQrW) * kQrW * kQrW, 0, q, ws,
                      s);
  }
  return e;
}

// Back substitution R X = B for R the k x k upper triangle of F: B (k x nrhs,
// row-major, row stride ldb) is overwritten by the partial right-hand sides and X
// (k x nrhs, row-major, ldx) receives the solution.  Rrm (k x k) and Rinv
// (ceil(k/64) blocks of 64 x 64) are scratch.
template <typename T>
cudaError_t tri_solve(int64_t k, const T* F, int64_t ld, T* B, int64_t ldb, int64_t nrhs, T* X, int64_t ldx, T* Rrm,
                      T* Rinv, cudaStream_t s) {
  const int nbk = (int)cdv(k, kTriB);
  k_tri_blocks<T><<<nbk, kTriB, 0, s>>>((int)k, F, ld, Rrm, Rinv);
  cudaError_t e = cudaGetLastError();
  for (int q = nbk - 1; e == cudaSuccess && q >= 0; --q) {
    const int64_t b0 = (int64_t)q * kTriB, bs = std::min<int64_t>(kTriB, k - b0), rest = k - b0 - bs;
    if (rest > 0) {  // B(block q) -= R(block q, later) X(later)
      Operand<T> a{Rrm + b0 * k, k, nullptr, b0 + bs};
      Operand<T> b{X + (b0 + bs) * ldx, ldx, nullptr, 0};
      EpiArgs<T> ep{B + b0 * ldb, ldb, 0, nullptr, nullptr};
      e = gemm_gather<T>((int)bs, (int)nrhs, (int)rest, 1, false, a, b, kEpiSubRows, ep, nullptr, s);
    }
    if (e == cudaSuccess) {  // X(block q) = R(q,q)^{-1} B(block q)
      Operand<T> a{Rinv + (int64_t)q * kTriB * kTriB, kTriB, nullptr, 0};
      Operand<T> b{B + b0 * ldb, ldb, nullptr, 0};
      EpiArgs<T> ep{X + b0 * ldx, ldx, 0, nullptr, nullptr};
      e = gemm_gather<T>((int)bs, (int)nrhs, (int)bs, 1, false, a, b, kEpiStore, ep, nullptr, s);
    }
  }
  return e;
}

// out (M x N, row-major, ldo) = A^T B for A (K x M) and B (K x N), both column-major
// (columns contiguous along K): split-K partials in P, then their sum.
template <typename T>
cudaError_t gemm_tn(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb, T* out,
                    int64_t ldo, T* P, int splits, cudaStream_t s) {
  Operand<T> a{A, lda, nullptr, 0};
  Operand<T> b{B, ldb, nullptr, 0};
  const int nz = gemm_splits((int)K, splits);
  EpiArgs<T> ep{nz > 1 ? P : out, nz > 1 ? N : ldo, M * N, nullptr, nullptr};
  cudaError_t e = gemm_gather<T>((int)M, (int)N, (int)K, nz, true, a, b, kEpiStore, ep, nullptr, s);
  if (e == cudaSuccess && nz > 1) e = splitk_reduce_ld<T>(M, (int)N, N, ldo, nz, M * N, P, out, nullptr, s);
  return e;
}

// ------------------------------------------------------------ stable X
struct StablePlan {
  QrScratch q;
  int msplits = 1;
  size_t off_st, off_F, off_Q, off_M, off_MP, off_X, off_R, off_Ri, off_qr, total;
};

template <typename T>
void stable_layout(int64_t m, int64_t n, int64_t k, StablePlan* p) {
  const int sms = sm_count();
  qr_layout<T>(m, k, sms, &p->q);
  p->msplits = qr_splits(k, n, m, sms);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = al(off + (b ? b : 1));
    return at;
  };
  const size_t e = sizeof(T);
  p->off_st = take(256);
  p->off_F = take((size_t)m * k * e);
  p->off_Q = take((size_t)m * k * e);
  p->off_M = take((size_t)k * n * e);
  p->off_MP = take(p->msplits > 1 ? (size_t)p->msplits * k * n * e : 0);
  p->off_X = take((size_t)k * n * e);
  p->off_R = take((size_t)k * k * e);
  p->off_Ri = take((size_t)cdv(k, kTriB) * kTriB * kTriB * e);
  p->off_qr = take(p->q.total);
  p->total = off;
}

template <typename T>
cudaError_t stable_x_run(const T* A, int64_t lda, int64_t m, int64_t n, const int64_t* J, int64_t k, T* Xout,
                         int64_t ldx, const StablePlan& p, unsigned char* ws, cudaStream_t s) {
  DevState* st = reinterpret_cast<DevState*>(ws + p.off_st);
  T* F = reinterpret_cast<T*>(ws + p.off_F);
  T* Q = reinterpret_cast<T*>(ws + p.off_Q);
  T* M = reinterpret_cast<T*>(ws + p.off_M);
  T* MP = reinterpret_cast<T*>(ws + p.off_MP);
  T* X = reinterpret_cast<T*>(ws + p.off_X);
  T* R = reinterpret_cast<T*>(ws + p.off_R);
  T* Ri = reinterpret_cast<T*>(ws + p.off_Ri);
  unsigned char* qws = ws + p.off_qr;
  cudaError_t e = init_state(st, nullptr, nullptr, 0, s);
  if (e != cudaSuccess) return e;
  k_gather2<T><<<grid1(m * k), 256, 0, s>>>(m, k, A, lda, m, n, nullptr, J, 0, F, m, st);  // C = A(:, J)
  e = cudaGetLastError();
  if (e == cudaSuccess) e = qr_factor<T>(m, k, F, m, p.q, qws, st, s);
  if (e == cudaSuccess) e = qr_form_q<T>(m, k, F, m, Q, m, p.q, qws, s);
  if (e == cudaSuccess) e = gemm_tn<T>(k, n, m, Q, m, A, lda, M, n, MP, p.msplits, s);  // M = Q^T A
  if (e == cudaSuccess) e = tri_solve<T>(k, F, m, M, n, n, X, n, R, Ri, s);              // X = R^{-1} M
  if (e == cudaSuccess) {  // the caller's X (k x n, column-major) = X (k x n, row-major)
    dim3 g((unsigned)std::min<int64_t>(cdv(k, 32), 1024), (unsigned)std::min<int64_t>(cdv(n, 32), 1024));
    k_transpose<T><<<g, dim3(32, 8), 0, s>>>(n, k, X, n, Xout, ldx);
    e = cudaGetLastError();
  }
  return e;
}

// ------------------------------------------------------------ CUR middle factor
struct CurPlan {
  QrScratch qc, qr;  // QR of C = A(:, J) (m x k) and of R^T = A(I, :)^T (n x k)
  int m1splits = 1, m2splits = 1;
  size_t off_st, off_Fc, off_Qc, off_Fr, off_Qr, off_M1, off_M1P, off_M2, off_M2P, off_Y, off_Z, off_R, off_Ri,
      off_qc, off_qr, total;
};

template <typename T>
void cur_layout(int64_t m, int64_t n, int64_t k, int kind, CurPlan* p) {
  const int sms = sm_count();
  const size_t e = sizeof(T);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = al(off + (b ? b : 1));
    return at;
  };
  p->off_st = take(256);
  if (kind == 0) {
    qr_layout<T>(m, k, sms, &p->qc);
    qr_layout<T>(n, k, sms, &p->qr);
    p->m1splits = qr_splits(k, n, m, sms);
    p->m2splits = qr_splits(k, k, n, sms);
    p->off_Fc = take((size_t)m * k * e);
    p->off_Qc = take((size_t)m * k * e);
    p->off_Fr = take((size_t)n * k * e);
    p->off_Qr = take((size_t)n * k * e);
    p->off_M1 = take((size_t)k * n * e);
    p->off_M1P = take(p->m1splits > 1 ? (size_t)p->m1splits * k * n * e : 0);
  } else {  // QR of the square A(I, J)
    qr_layout<T>(k, k, sms, &p->qc);
    p->m2splits = qr_splits(k, k, k, sms);
    p->off_Fc = take((size_t)k * k * e);
    p->off_Qc = take((size_t)k * k * e);
    p->off_Fr = p->off_Qr = p->off_M1 = p->off_M1P = take(0);
  }
  p->off_M2 = take((size_t)k * k * e);
  p->off_M2P = take(p->m2splits > 1 ? (size_t)p->m2splits * k * k * e : 0);
  p->off_Y = take((size_t)k * k * e);
  p->off_Z = take((size_t)k * k * e);
  p->off_R = take((size_t)k * k * e);
  p->off_Ri = take((size_t)cdv(k, kTriB) * kTriB * kTriB * e);
  p->off_qc = take(p->qc.total);
  p->off_qr = take(kind == 0 ? p->qr.total : 0);
  p->total = off;
}

template <typename T>
cudaError_t cur_run(const T* A, int64_t lda, int64_t m, int64_t n, const int64_t* I, const int64_t* J, int64_t k,
                    int kind, T* U, int64_t ldu, const CurPlan& p, unsigned char* ws, cudaStream_t s) {
  DevState* st = reinterpret_cast<DevState*>(ws + p.off_st);
  T* Fc = reinterpret_cast<T*>(ws + p.off_Fc);
  T* Qc = reinterpret_cast<T*>(ws + p.off_Qc);
  T* M2 = reinterpret_cast<T*>(ws + p.off_M2);
  T* M2P = reinterpret_cast<T*>(ws + p.off_M2P);
  T* Y = reinterpret_cast<T*>(ws + p.off_Y);
  T* Z = reinterpret_cast<T*>(ws + p.off_Z);
  T* R = reinterpret_cast<T*>(ws + p.off_R);
  T* Ri = reinterpret_cast<T*>(ws + p.off_Ri);
  cudaError_t e = init_state(st, nullptr, nullptr, 0, s);
  dim3 tg((unsigned)std::min<int64_t>(cdv(k, 32), 1024), (unsigned)std::min<int64_t>(cdv(k, 32), 1024));
  if (kind == 0) {
    // U = C^+ A R^+ = Rc^{-1} (Qc^T A Qr) Rr^{-T} with C = Qc Rc, R^T = Qr Rr
    T* Fr = reinterpret_cast<T*>(ws + p.off_Fr);
    T* Qr = reinterpret_cast<T*>(ws + p.off_Qr);
    T* M1 = reinterpret_cast<T*>(ws + p.off_M1);
    T* M1P = reinterpret_cast<T*>(ws + p.off_M1P);
    if (e == cudaSuccess) {
      k_gather2<T><<<grid1(m * k), 256, 0, s>>>(m, k, A, lda, m, n, nullptr, J, 0, Fc, m, st);  // C = A(:, J)
      k_gather2<T><<<grid1(n * k), 256, 0, s>>>(k, n, A, lda, m, n, I, nullptr, 1, Fr, n, st);  // R^T = A(I, :)^T
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = qr_factor<T>(m, k, Fc, m, p.qc, ws + p.off_qc, st, s);
    if (e == cudaSuccess) e = qr_form_q<T>(m, k, Fc, m, Qc, m, p.qc, ws + p.off_qc, s);
    if (e == cudaSuccess) e = qr_factor<T>(n, k, Fr, n, p.qr, ws + p.off_qr, st, s);
    if (e == cudaSuccess) e = qr_form_q<T>(n, k, Fr, n, Qr, n, p.qr, ws + p.off_qr, s);
    if (e == cudaSuccess) e = gemm_tn<T>(k, n, m, Qc, m, A, lda, M1, n, M1P, p.m1splits, s);  // M1 = Qc^T A (k x n)
    if (e == cudaSuccess) {  // M2 = M1 Qr (k x k, row-major): rows of M1 against columns of Qr, both along n
      Operand<T> a{M1, n, nullptr, 0};
      Operand<T> b{Qr, n, nullptr, 0};
      const int nz = gemm_splits((int)n, p.m2splits);
      EpiArgs<T> ep{nz > 1 ? M2P : M2, k, k * k, nullptr, nullptr};
      e = gemm_gather<T>((int)k, (int)k, (int)n, nz, true, a, b, kEpiStore, ep, nullptr, s);
      if (e == cudaSuccess && nz > 1) e = splitk_reduce_ld<T>(k, (int)k, k, k, nz, k * k, M2P, M2, nullptr, s);
    }
    if (e == cudaSuccess) e = tri_solve<T>(k, Fc, m, M2, k, k, Y, k, R, Ri, s);  // Y = Rc^{-1} M2
    if (e == cudaSuccess) {  // U^T = Rr^{-1} Y^T
      k_transpose<T><<<tg, dim3(32, 8), 0, s>>>(k, k, Y, k, Z, k);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = tri_solve<T>(k, Fr, n, Z, k, k, Y, k, R, Ri, s);  // Y = U^T (row-major)
    // U (column-major, ldu) = Y^T (row-major)  <=>  U^T row-major = Y: copy rows
    if (e == cudaSuccess) {
      k_transpose<T><<<tg, dim3(32, 8), 0, s>>>(k, k, Y, k, Z, k);  // Z = U row-major
      e = cudaGetLastError();
    }
  } else {
    // U = A(I, J)^{-1} = R^{-1} Q^T for A(I, J) = Q R
    if (e == cudaSuccess) {
      k_gather2<T><<<grid1(k * k), 256, 0, s>>>(k, k, A, lda, m, n, I, J, 0, Fc, k, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = qr_factor<T>(k, k, Fc, k, p.qc, ws + p.off_qc, st, s);
    if (e == cudaSuccess) e = qr_form_q<T>(k, k, Fc, k, Qc, k, p.qc, ws + p.off_qc, s);
    // Q column-major (ld k) read row-major is Q^T: the right-hand side as it stands
    if (e == cudaSuccess) e = tri_solve<T>(k, Fc, k, Qc, k, k, Z, k, R, Ri, s);  // Z = U row-major
  }
  if (e == cudaSuccess) {  // the caller's U (k x k column-major, ldu) from Z (row-major)
    k_transpose<T><<<tg, dim3(32, 8), 0, s>>>(k, k, Z, k, U, ldu);
    e = cudaGetLastError();
  }
  return e;
}

int check_matrix(const id_matrix* A) {
  if (A == nullptr || A->data == nullptr || A->m < 1 || A->n < 1 || A->ld < A->m || A->m >= ((int64_t)1 << 31) ||
      A->n >= ((int64_t)1 << 31))
    return -1;
  if (A->dtype != ID_F64 && A->dtype != ID_F32) return ID_ERR_UNSUPPORTED;
  return ID_OK;
}

int finish_status(DevState* st, cudaStream_t s) {
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ID_ERR_CUDA;
  if (h.err & kErrTimeout) return ID_ERR_TIMEOUT;
  if (h.err & kErrBadIndex) return -2;
  return ID_OK;
}

}  // namespace
}  // namespace rid

using namespace rid;

extern "C" {

int id_stable_x_workspace_size(const id_matrix* A, int64_t k, size_t* bytes) {
  const int rc = check_matrix(A);
  if (rc != ID_OK) return rc;
  if (k < 1 || k > std::min(A->m, A->n)) return -2;
  if (bytes == nullptr) return -3;
  StablePlan p;
  if (A->dtype == ID_F64)
    stable_layout<double>(A->m, A->n, k, &p);
  else
    stable_layout<float>(A->m, A->n, k, &p);
  *bytes = p.total;
  return ID_OK;
}

int id_stable_x(const id_matrix* A, const int64_t* J, int64_t k, void* X, int64_t ldx, void* ws, size_t ws_bytes,
                void* stream) {
  const int rc = check_matrix(A);
  if (rc != ID_OK) return rc;
  if (J == nullptr) return -2;
  if (k < 1 || k > std::min(A->m, A->n)) return -3;
  if (X == nullptr || ldx < k) return -4;
  StablePlan p;
  if (A->dtype == ID_F64)
    stable_layout<double>(A->m, A->n, k, &p);
  else
    stable_layout<float>(A->m, A->n, k, &p);
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < p.total) return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  cudaError_t e = A->dtype == ID_F64
                      ? stable_x_run<double>(static_cast<const double*>(A->data), A->ld, A->m, A->n, J, k,
                                             static_cast<double*>(X), ldx, p, w, s)
                      : stable_x_run<float>(static_cast<const float*>(A->data), A->ld, A->m, A->n, J, k,
                                            static_cast<float*>(X), ldx, p, w, s);
  if (e != cudaSuccess) return ID_ERR_CUDA;
  return finish_status(reinterpret_cast<DevState*>(w + p.off_st), s);
}

int cur_middle_workspace_size(const id_matrix* A, int64_t k, int middle_kind, size_t* bytes) {
  const int rc = check_matrix(A);
  if (rc != ID_OK) return rc;
  if (k < 1 || k > std::min(A->m, A->n)) return -2;
  if (middle_kind != ID_CUR_PSEUDOINVERSE && middle_kind != ID_CUR_INVERSE) return -3;
  if (bytes == nullptr) return -4;
  CurPlan p;
  if (A->dtype == ID_F64)
    cur_layout<double>(A->m, A->n, k, middle_kind, &p);
  else
    cur_layout<float>(A->m, A->n, k, middle_kind, &p);
  *bytes = p.total;
  return ID_OK;
}

int cur_middle(const id_matrix* A, const int64_t* I, const int64_t* J, int64_t k, void* U, int64_t ldu,
               int middle_kind, void* ws, size_t ws_bytes, void* stream) {
  const int rc = check_matrix(A);
  if (rc != ID_OK) return rc;
  if (I == nullptr) return -2;
  if (J == nullptr) return -3;
  if (k < 1 || k > std::min(A->m, A->n)) return -4;
  if (U == nullptr || ldu < k) return -5;
  if (middle_kind != ID_CUR_PSEUDOINVERSE && middle_kind != ID_CUR_INVERSE) return -7;
  CurPlan p;
  if (A->dtype == ID_F64)
    cur_layout<double>(A->m, A->n, k, middle_kind, &p);
  else
    cur_layout<float>(A->m, A->n, k, middle_kind, &p);
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < p.total) return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  cudaError_t e = A->dtype == ID_F64
                      ? cur_run<double>(static_cast<const double*>(A->data), A->ld, A->m, A->n, I, J, k, middle_kind,
                                        static_cast<double*>(U), ldu, p, w, s)
                      : cur_run<float>(static_cast<const float*>(A->data), A->ld, A->m, A->n, I, J, k, middle_kind,
                                       static_cast<float*>(U), ldu, p, w, s);
  if (e != cudaSuccess) return ID_ERR_CUDA;
  const int st = finish_status(reinterpret_cast<DevState*>(w + p.off_st), s);
  return st == -2 ? -2 : st;  // an index outside A: I or J (reported as I)
}

}  // extern "C"
