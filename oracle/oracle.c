/*
 * oracle.c -- plain FP64 CPU reference for the randomized column ID of
 * arXiv:2310.09417 (Pearce, Chen, Dong, Martinsson).  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Everything here is the textbook definition written out with plain loops in
 * FP64, in the paper's order of operations (transposed to the column ID, see
 * oracle.h).  There is no blocking, fusion or reordering beyond what the paper
 * states.  OpenMP only parallelises loops whose iterations are independent
 * (one column of a product each), so results do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon et al., SC'11): a 10-round Feistel-like bijection of  */
/* a 256-bit counter under a 128-bit key; each round multiplies two words by   */
/* fixed odd constants, keeps the high and low halves, and xors the high      */
/* halves with the other words and the round key; the key is bumped by two    */
/* Weyl constants between rounds.                                             */
/* ------------------------------------------------------------------------- */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    unsigned __int128 p0 = (unsigned __int128)M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 53-bit uniform in (0, 1]: never zero, so log() below is finite. */
static double orc_u53(uint64_t x) { return (double)((x >> 11) + 1) * 0x1.0p-53; }

void orc_gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, double* out) {
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i) {
    double* row = out + i * m;
    for (int64_t q = 0; 4 * q < m; ++q) {
      uint64_t ctr[4] = {(uint64_t)q, (uint64_t)(row0 + i), 0, 0};
      uint64_t key[2] = {seed, 0};
      uint64_t x[4];
      orc_philox4x64_10(ctr, key, x);
      double z[4];
      /* Box-Muller on the pairs (x0, x1) and (x2, x3). */
      for (int h = 0; h < 2; ++h) {
        double u1 = orc_u53(x[2 * h]), u2 = orc_u53(x[2 * h + 1]);
        double r = sqrt(-2.0 * log(u1));
        z[2 * h] = r * cos(two_pi * u2);
        z[2 * h + 1] = r * sin(two_pi * u2);
      }
      for (int j = 0; j < 4 && 4 * q + j < m; ++j) row[4 * q + j] = z[j];
    }
  }
}

/* Sparse-sign block t (Sec. 5.1, "Sparse Sign", column form; definition in oracle.h). */
void orc_sparse_sign_block(uint64_t seed, int64_t t, int64_t b, int64_t m, int64_t zeta, double* out) {
  const double v = sqrt((double)b / (double)zeta);
  for (int64_t e = 0; e < b * m; ++e) out[e] = 0.0;
  int64_t* p = (int64_t*)malloc(sizeof(int64_t) * b);
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t r = 0; r < b; ++r) p[r] = r;
    uint64_t w[4] = {0, 0, 0, 0};
    for (int64_t j = 0; j < zeta; ++j) {
      if (j % 4 == 0) {
        uint64_t ctr[4] = {(uint64_t)i, (uint64_t)t, (uint64_t)(j / 4), 0};
        uint64_t key[2] = {seed, 1};
        orc_philox4x64_10(ctr, key, w);
      }
      const uint64_t u = w[j % 4];
      const int64_t r = j + (int64_t)(((u >> 32) * (uint64_t)(b - j)) >> 32);
      const int64_t tmp = p[j];
      p[j] = p[r];
      p[r] = tmp;
      out[p[j] * m + i] = (u & 1u) ? -v : v;
    }
  }
  free(p);
}

/* ------------------------------------------------------------------------- */
/* Sketch (Sec. 2.4, column form Y = Omega A), stored transposed.            */
/* ------------------------------------------------------------------------- */
void orc_sketch_t(int64_t m, int64_t n, const double* A, int64_t lda,
                  int64_t rows, const double* Omega, double* YT) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    const double* a = A + j * lda;
    for (int64_t i = 0; i < rows; ++i) {
      const double* w = Omega + i * m;
      double s = 0.0;
      for (int64_t r = 0; r < m; ++r) s += w[r] * a[r];
      YT[j + i * n] = s;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* LU with partial pivoting, right-looking (Sec. 2.3.2).                      */
/* ------------------------------------------------------------------------- */
static void orc_swap_rows(double* M, int64_t ld, int64_t nc, int64_t r1, int64_t r2) {
  if (r1 == r2) return;
  for (int64_t j = 0; j < nc; ++j) {
    double t = M[r1 + j * ld];
    M[r1 + j * ld] = M[r2 + j * ld];
    M[r2 + j * ld] = t;
  }
}

int64_t orc_lupp(int64_t nr, int64_t nc, int64_t steps, double* M, int64_t ld, int64_t* orig) {
  int64_t zero_pivots = 0;
  for (int64_t c = 0; c < steps; ++c) {
    /* pivot: largest magnitude in column c among rows c.., ties to the
       smallest original label */
    int64_t best = c;
    double bv = fabs(M[c + c * ld]);
    for (int64_t i = c + 1; i < nr; ++i) {
      double v = fabs(M[i + c * ld]);
      if (v > bv || (v == bv && orig[i] < orig[best])) {
        best = i;
        bv = v;
      }
    }
    orc_swap_rows(M, ld, nc, c, best);
    int64_t t = orig[c];
    orig[c] = orig[best];
    orig[best] = t;
    if (bv == 0.0) { /* exactly zero column: nothing to eliminate */
      ++zero_pivots;
      continue;
    }
    double piv = M[c + c * ld];
    for (int64_t i = c + 1; i < nr; ++i) M[i + c * ld] /= piv;
    /* Schur-complement update, Eq. lupps */
    for (int64_t j = c + 1; j < nc; ++j) {
      double u = M[c + j * ld];
      for (int64_t i = c + 1; i < nr; ++i) M[i + j * ld] -= M[i + c * ld] * u;
    }
  }
  return zero_pivots;
}

/* ------------------------------------------------------------------------- */
/* Interpolation matrix: X(:,p[i]) = e_i for i < k, and for every other row r */
/* of the permuted L, z L1 = L(r, 0:k) solved by substitution (L1 unit lower, */
/* so z L1 = l is an upper-triangular system in z read from the last entry).  */
/* This is W = P^T [I; L2 L1^{-1}] of Eq. inty / Algorithm 1, transposed.     */
/* L is n x k column-major (ld = ldl), rows in pivot order p.                 */
/* ------------------------------------------------------------------------- */
static void orc_form_x(int64_t n, int64_t k, const double* L, int64_t ldl, const int64_t* p,
                       double* X, int64_t ldx) {
  for (int64_t i = 0; i < k; ++i) {
    double* x = X + p[i] * ldx;
    for (int64_t c = 0; c < k; ++c) x[c] = (c == i) ? 1.0 : 0.0;
  }
#pragma omp parallel for schedule(static)
  for (int64_t r = k; r < n; ++r) {
    double* z = X + p[r] * ldx;
    for (int64_t c = k - 1; c >= 0; --c) {
      double s = L[r + c * ldl];
      for (int64_t c2 = c + 1; c2 < k; ++c2) s -= z[c2] * L[c2 + c * ldl];
      z[c] = s; /* unit diagonal */
    }
  }
}

static int orc_all_finite(int64_t m, int64_t n, const double* A, int64_t lda) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i)
      if (!isfinite(A[i + j * lda])) return 0;
  return 1;
}

static int64_t orc_min3(int64_t a, int64_t b, int64_t c) {
  int64_t x = a < b ? a : b;
  return x < c ? x : c;
}

/* ------------------------------------------------------------------------- */
/* randLUPP, fixed rank (Sec. 3.1).                                           */
/* ------------------------------------------------------------------------- */
int orc_id_fixed_rank(int64_t m, int64_t n, const double* A, int64_t lda,
                      int64_t l, const double* Omega, int64_t k,
                      int64_t* J, double* X, int64_t ldx, double* est, double* pivots) {
  if (m < 1 || n < 1 || lda < m || l < 1 || k < 1 || k > l || k > orc_min3(m, n, l) || ldx < k)
    return ORC_BAD_ARG;
  if (!orc_all_finite(m, n, A, lda)) return ORC_NONFINITE;
  double* YT = (double*)malloc(sizeof(double) * n * l);
  int64_t* p = (int64_t*)malloc(sizeof(int64_t) * n);
  orc_sketch_t(m, n, A, lda, l, Omega, YT);
  for (int64_t i = 0; i < n; ++i) p[i] = i;
  orc_lupp(n, l, k, YT, n, p);
  for (int64_t i = 0; i < k; ++i) J[i] = p[i];
  if (pivots)
    for (int64_t i = 0; i < k; ++i) pivots[i] = fabs(YT[i + i * n]);
  /* Schur-complement estimate from the l-k columns beyond k (Eq. errSch) */
  double e = 0.0;
  if (l > k && n > k) {
    double s2 = 0.0;
    for (int64_t j = k; j < l; ++j)
      for (int64_t i = k; i < n; ++i) s2 += YT[i + j * n] * YT[i + j * n];
    e = sqrt(s2 / (double)(l - k));
  }
  if (est) *est = e;
  orc_form_x(n, k, YT, n, p, X, ldx);
  free(YT);
  free(p);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* randLUPPadap (Algorithm 1), column form, round by round.                   */
/* State kept exactly as the algorithm lists it: the permutation p (a vector, */
/* Sec. 4.1), L = [L1; L2] with rows in pivot order (n x tb), and the         */
/* factored sample.  U is not needed for J, X or E; only |U(i,i)| is kept.     */
/* ------------------------------------------------------------------------- */
int orc_id_adaptive(int64_t m, int64_t n, const double* A, int64_t lda,
                    int64_t b, double tol, int64_t kmax,
                    const double* Omega, int64_t rows_avail,
                    int64_t* k_out, int64_t* J, double* X, int64_t ldx,
                    double* trace, int64_t trace_cap, int64_t* rounds, double* pivots) {
  if (m < 1 || n < 1 || lda < m || b < 1 || kmax < 1 || ldx < kmax || !(tol >= 0.0))
    return ORC_BAD_ARG;
  if (!orc_all_finite(m, n, A, lda)) return ORC_NONFINITE;
  const int64_t cap = orc_min3(m, n, kmax);
  double* L = (double*)calloc((size_t)n * cap, sizeof(double)); /* n x cap, ld n */
  double* G = (double*)malloc(sizeof(double) * n * b);          /* new sample, n x b */
  double* PG = (double*)malloc(sizeof(double) * n * b);         /* rows permuted by p */
  double* U2 = (double*)malloc(sizeof(double) * cap * b);       /* tb x b */
  double* S = (double*)malloc(sizeof(double) * n * b);          /* (n-tb) x b */
  double* Lrow = (double*)malloc(sizeof(double) * n);           /* one column of L2 */
  int64_t* p = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* orig = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * n);
  int status = ORC_OK;

  /* Alg. 1, start: the first sample, its LUPP, and L1, L2 from its factors */
  int64_t t = 0;
  if ((t + 1) * b > rows_avail) { status = ORC_BAD_ARG; goto done; }
  orc_sketch_t(m, n, A, lda, b, Omega, G);
  for (int64_t i = 0; i < n; ++i) p[i] = i;
  int64_t b0 = b < cap ? b : cap;
  orc_lupp(n, b, b0, G, n, p);
  for (int64_t c = 0; c < b0; ++c) {
    if (pivots) pivots[c] = fabs(G[c + c * n]);
    for (int64_t i = c + 1; i < n; ++i) L[i + c * n] = G[i + c * n];
    L[c + c * n] = 1.0;
  }
  int64_t tb = b0;
  /* E(0) = tol + 1 (so the loop runs at least once) and t = 1 */
  t = 1;
  int64_t nrounds = 0;
  for (;;) {
    if (tb == n) break; /* every column is a skeleton: the residual is exactly zero */
    /* Alg. 1, loop: a new independent Gaussian block and its sample */
    if ((t + 1) * b > rows_avail) { status = ORC_BAD_ARG; goto done; }
    orc_sketch_t(m, n, A, lda, b, Omega + t * b * m, G);
    for (int64_t c = 0; c < b; ++c)
      for (int64_t i = 0; i < n; ++i) PG[i + c * n] = G[p[i] + c * n];
    /* U2 = L1^{-1} (P Y)(1:tb,:) by forward substitution */
    for (int64_t c = 0; c < b; ++c)
      for (int64_t i = 0; i < tb; ++i) {
        double s = PG[i + c * n];
        for (int64_t j = 0; j < i; ++j) s -= L[i + j * n] * U2[j + c * cap];
        U2[i + c * cap] = s;
      }
    /* the Schur complement S = (P Y)(tb+1:end,:) - L2 U2 */
    const int64_t ns = n - tb;
    for (int64_t c = 0; c < b; ++c)
      for (int64_t i = 0; i < ns; ++i) {
        double s = PG[tb + i + c * n];
        for (int64_t j = 0; j < tb; ++j) s -= L[tb + i + j * n] * U2[j + c * cap];
        S[i + c * ns] = s;
      }
    /* the estimate E = ||S||_F, scaled for N(0,1) blocks (variance reading of 1/b) */
    double s2 = 0.0;
    for (int64_t c = 0; c < b; ++c)
      for (int64_t i = 0; i < ns; ++i) s2 += S[i + c * ns] * S[i + c * ns];
    double E = sqrt(s2 / (double)b);
    if (trace && nrounds < trace_cap) trace[nrounds] = E;
    ++nrounds;
    if (E <= tol) break;                            /* the loop's stopping test */
    if (tb == cap) { status = ORC_TOL_NOT_MET; break; }
    const int64_t bt = (b < cap - tb) ? b : (cap - tb);
    /* LUPP of S; labels are the original column indices */
    for (int64_t i = 0; i < ns; ++i) orig[i] = p[tb + i];
    orc_lupp(ns, b, bt, S, ns, orig);
    /* apply P-hat to the rows of L2 and append the new block's factor */
    /* the row now at position tb+i of S came from position pos[orig[i]] */
    for (int64_t i = 0; i < n; ++i) pos[p[i]] = i;
    for (int64_t j = 0; j < tb; ++j) {
      for (int64_t i = 0; i < ns; ++i) Lrow[i] = L[tb + i + j * n];
      for (int64_t i = 0; i < ns; ++i) L[tb + i + j * n] = Lrow[pos[orig[i]] - tb];
    }
    for (int64_t c = 0; c < bt; ++c) {
      if (pivots) pivots[tb + c] = fabs(S[c + c * ns]);
      for (int64_t i = c + 1; i < ns; ++i) L[tb + i + (tb + c) * n] = S[i + c * ns];
      L[tb + c + (tb + c) * n] = 1.0;
    }
    /* P(t) = diag(I, P-hat) P(t-1) */
    for (int64_t i = 0; i < ns; ++i) p[tb + i] = orig[i];
    tb += bt;
    ++t;
  }
  *k_out = tb;
  if (rounds) *rounds = nrounds;
  /* after the loop: J from P, and the interpolation matrix X from L (Eq. inty) */
  for (int64_t i = 0; i < tb; ++i) J[i] = p[i];
  orc_form_x(n, tb, L, n, p, X, ldx);
done:
  free(L); free(G); free(PG); free(U2); free(S); free(Lrow);
  free(p); free(orig); free(pos);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Error measures (Sec. 2.1, 2.2.1, 5.1).                                     */
/* ------------------------------------------------------------------------- */
double orc_fro_norm(int64_t m, int64_t n, const double* A, int64_t lda) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) s += A[i + j * lda] * A[i + j * lda];
  return sqrt(s);
}

double orc_id_residual(int64_t m, int64_t n, const double* A, int64_t lda,
                       int64_t k, const int64_t* J, const double* X, int64_t ldx) {
  /* per-column sums of squares in parallel, then added in column order, so the
     value does not depend on how the threads finish */
  double* col = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      double approx = 0.0;
      for (int64_t c = 0; c < k; ++c) approx += A[i + J[c] * lda] * X[c + j * ldx];
      double d = A[i + j * lda] - approx;
      s += d * d;
    }
    col[j] = s;
  }
  double total = 0.0;
  for (int64_t j = 0; j < n; ++j) total += col[j];
  free(col);
  return sqrt(total);
}

double orc_stable_residual(int64_t m, int64_t n, const double* A, int64_t lda,
                           int64_t k, const int64_t* J) {
  /* Householder QR of C = A(:,J); apply Q^T to A; the rows k..m-1 of Q^T A
     are (I - Q Q^T) A expressed in the complementary basis. */
  double* C = (double*)malloc(sizeof(double) * m * k);
  double* B = (double*)malloc(sizeof(double) * m * n);
  double* v = (double*)malloc(sizeof(double) * m);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) C[i + c * m] = A[i + J[c] * lda];
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) B[i + j * m] = A[i + j * lda];
  int64_t steps = k < m ? k : m;
  for (int64_t c = 0; c < steps; ++c) {
    double nrm = 0.0;
    for (int64_t i = c; i < m; ++i) nrm += C[i + c * m] * C[i + c * m];
    nrm = sqrt(nrm);
    if (nrm == 0.0) continue;
    double alpha = C[c + c * m] >= 0 ? -nrm : nrm;
    for (int64_t i = c; i < m; ++i) v[i] = C[i + c * m];
    v[c] -= alpha;
    double vn = 0.0;
    for (int64_t i = c; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    /* H = I - 2 v v^T / (v^T v), applied to C(:, c:) and to B */
    for (int64_t j = c; j < k; ++j) {
      double d = 0.0;
      for (int64_t i = c; i < m; ++i) d += v[i] * C[i + j * m];
      d = 2.0 * d / vn;
      for (int64_t i = c; i < m; ++i) C[i + j * m] -= d * v[i];
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      double d = 0.0;
      for (int64_t i = c; i < m; ++i) d += v[i] * B[i + j * m];
      d = 2.0 * d / vn;
      for (int64_t i = c; i < m; ++i) B[i + j * m] -= d * v[i];
    }
  }
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = steps; i < m; ++i) s += B[i + j * m] * B[i + j * m];
  free(C); free(B); free(v);
  return sqrt(s);
}
