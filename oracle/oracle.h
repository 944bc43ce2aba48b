/*
 * oracle.h -- plain FP64 CPU reference ("the oracle") for the randomized column
 * interpolative decomposition (ID) of Pearce, Chen, Dong and Martinsson,
 * "Adaptive Parallelizable Algorithms for Interpolative Decompositions via
 * Partially Pivoted LU" (arXiv:2310.09417).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark may call this library. The GPU library shares no
 * code, header, table or helper with it.
 *
 * Orientation. The paper states everything as a row ID of A (Y = A*Omega, LUPP
 * on Y, A ~ W*A(I,:)) and notes that the column ID is the same construction on
 * A^T (Sec. 4).  This oracle computes the column ID directly:
 *     Y = Omega * A          (Omega: l x m, Y: l x n)
 *     LUPP of Y^T            (n x l; rows of Y^T are columns of A)
 *     J = first k pivots,    A ~ A(:,J) * X,  X(:,J) = I_k,
 *     X(:,J^c) = (L2 * L1^{-1})^T                        (Eq. inty, transposed)
 *
 * Conventions. A is column-major m x n with leading dimension lda >= m.
 * Omega is row-major (row i of Omega is contiguous, length m).  X is column-major
 * k x n with leading dimension ldx >= k.  Indices are 0-based int64.
 * Ties in the pivot search go to the smallest ORIGINAL row index of Y^T (i.e.
 * the smallest column index of A).  An exactly zero pivot column is skipped the
 * way LAPACK getrf does (no scaling, zero multipliers) and counted.
 *
 * Gaussian test matrices: element (i, r) of the sketching matrix is a standard
 * normal number derived from the counter-based generator Philox4x64-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11) keyed by (seed, 0) at counter (r / 4, i, 0, 0), followed by the
 * Box-Muller transform on 53-bit uniforms in (0, 1].
 *
 * Scaling of the error estimate.  The paper draws the estimation block with
 * "standard deviation 1/b" (Sec. 3.2, Sec. 5.1), which contradicts its own
 * unbiasedness statement E||S||_F^2 = ||A - WR||_F^2 (Sec. 4.2).  The oracle reads
 * it as variance 1/b: Omega has N(0,1) entries and E = ||S||_F / sqrt(b).
 */
#ifndef RANDID_ORACLE_H
#define RANDID_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status values returned by the oracle drivers */
#define ORC_OK 0
#define ORC_TOL_NOT_MET 1   /* reached the rank cap with E > tol */
#define ORC_BAD_ARG (-1)
#define ORC_NONFINITE (-2)

/* Philox4x64-10 block function (Salmon et al. 2011, Sec. 3 and Table 2). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Rows [row0, row0 + rows) of the Gaussian sketching matrix (rows x m, row-major). */
void orc_gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, double* out);

/* Block t of a sparse-sign sketching matrix (Sec. 5.1, "Sparse Sign"), column
 * form: b rows x m columns, row-major (ld = m), the rows t*b .. t*b+b-1 of Omega.
 * Every column holds zeta nonzeros (1 <= zeta <= b) at distinct rows, each
 * +-sqrt(b/zeta), so that E[Omega^T Omega] = b I as for N(0,1) entries.
 * Definition:
 *   - The words u_0, u_1, ... of column i in block t are Philox4x64-10 keyed
 *     (seed, 1) at counters (i, t, c, 0), c = 0, 1, ..., four words per
 *     counter, in order.
 *   - Rows come from a partial Fisher-Yates shuffle of p = (0, ..., b-1): for
 *     j = 0 .. zeta-1, r = j + (((u_j >> 32) * (b - j)) >> 32), swap p[j] and
 *     p[r].
 *   - Nonzero j sits at row p[j], negative if u_j is odd. */
void orc_sparse_sign_block(uint64_t seed, int64_t t, int64_t b, int64_t m, int64_t zeta, double* out);

/* Y^T = (Omega * A)^T : Omega rows x m (row-major, ld = m), A m x n col-major.
 * Output YT is n x rows, column-major with leading dimension n. */
void orc_sketch_t(int64_t m, int64_t n, const double* A, int64_t lda,
                  int64_t rows, const double* Omega, double* YT);

/* Right-looking LU with partial pivoting (Sec. 2.3.2, Eq. lupp and Eq. lupps),
 * stopped after `steps` elimination steps.  M is nr x nc column-major (ld).  On
 * exit the first `steps` columns hold L (strictly below the diagonal, unit
 * diagonal implied) and U (on and above), the trailing (nr-steps) x (nc-steps)
 * block holds the Schur complement, and rows were physically interchanged.
 * orig[i] carries the original label of the row now at position i; it must be
 * initialised by the caller (labels decide ties).  Returns the number of exactly
 * zero pivot columns met. */
int64_t orc_lupp(int64_t nr, int64_t nc, int64_t steps, double* M, int64_t ld, int64_t* orig);

/* randLUPP fixed-rank column ID (Sec. 3.1): Y = Omega(0:l,:) A, LUPP of Y^T,
 * J = first k pivots, X from L.  If l > k, *est receives the Schur-complement
 * estimate ||S||_F / sqrt(l-k) (Eq. errSch), else 0.  pivots (may be NULL)
 * receives |U(i,i)| for i < k. */
int orc_id_fixed_rank(int64_t m, int64_t n, const double* A, int64_t lda,
                      int64_t l, const double* Omega, int64_t k,
                      int64_t* J, double* X, int64_t ldx, double* est, double* pivots);

/* randLUPPadap column ID (Algorithm 1, Sec. 4), literally round by round.
 * Omega supplies all rows the run may draw, row-major (rows_avail x m); round t
 * uses rows [t*b, t*b + b).  tol is absolute (Algorithm 1 stops when E <= tol).
 * kmax caps the rank.  Outputs: *k_out, J[kmax], X (kmax x n, ldx >= kmax;
 * columns filled in rows 0..k-1), trace[t-1] = E at round t (up to
 * trace_cap entries), *rounds = number of estimates computed, pivots[kmax]
 * = |U(i,i)| (may be NULL).  Returns ORC_OK or ORC_TOL_NOT_MET. */
int orc_id_adaptive(int64_t m, int64_t n, const double* A, int64_t lda,
                    int64_t b, double tol, int64_t kmax,
                    const double* Omega, int64_t rows_avail,
                    int64_t* k_out, int64_t* J, double* X, int64_t ldx,
                    double* trace, int64_t trace_cap, int64_t* rounds, double* pivots);

/* ||A||_F with a sequential FP64 sum over column-major storage. */
double orc_fro_norm(int64_t m, int64_t n, const double* A, int64_t lda);

/* ||A - A(:,J) X||_F, the column ID error (Sec. 2.2.1). */
double orc_id_residual(int64_t m, int64_t n, const double* A, int64_t lda,
                       int64_t k, const int64_t* J, const double* X, int64_t ldx);

/* ||A - Q Q^T A||_F with Q from Householder QR of A(:,J): the stable ID error
 * (Eq. sID_row, column form; Sec. 5.1 "sID"). */
double orc_stable_residual(int64_t m, int64_t n, const double* A, int64_t lda,
                           int64_t k, const int64_t* J);

#ifdef __cplusplus
}
#endif
#endif
