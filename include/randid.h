/*
 * randid.h -- C ABI of the GB300 (sm_103a) randomized column interpolative
 * decomposition library.
 *
 * Method: Pearce, Chen, Dong, Martinsson, "Adaptive Parallelizable Algorithms
 * for Interpolative Decompositions via Partially Pivoted LU", arXiv:2310.09417.
 * Given A (m x n) the library returns a column skeleton J (|J| = k) and an
 * interpolation matrix X (k x n) with A ~ A(:,J) X, X(:,J) = I_k (Sec. 2.2.1,
 * column ID).  Skeletons come from LU with partial pivoting (Sec. 2.3.2) of the
 * transposed Gaussian sketch Y^T = (Omega A)^T (Sec. 2.4, Sec. 3.1); the
 * adaptive driver grows the sketch block by block and stops when the
 * Schur-complement estimate of Eq. errSch falls below the tolerance
 * (Algorithm 1, Sec. 4).  The paper states the method as a row ID; the
 * column ID computed here is the row ID of A^T.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major (LAPACK convention) with an explicit leading
 *     dimension.  Every data pointer is a DEVICE pointer owned by the caller,
 *     unless a field says HOST.
 *   - Indices are 0-based int64 (the paper is 1-based).
 *   - The library allocates no device memory: the caller passes a workspace of
 *     at least the size the matching *_workspace_size query returns, aligned to
 *     256 bytes.  The workspace may be reused between calls, not shared by calls
 *     that run concurrently.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every entry
 *     point enqueues its work on `stream` and returns after that work has
 *     finished (the adaptive driver needs the stop decision on the host), so
 *     outputs are ready when the call returns.
 *   - Return value: ID_OK (0), a positive warning bit set, or a negative error.
 *     -i means argument i (1-based) is invalid; nothing was launched.
 *   - Ties in the pivot search go to the smallest column index of A.  An
 *     exactly zero pivot column is skipped as LAPACK getrf does (zero
 *     multipliers) and reported with ID_WARN_ZERO_PIVOT.
 *   - The error estimate uses N(0,1) sketch rows and E = ||S||_F / sqrt(b):
 *     the paper's "standard deviation 1/b" (Sec. 3.2, Sec. 5.1) is read as
 *     variance 1/b, the scaling under which E^2 is unbiased for
 *     ||A - A(:,J) X||_F^2 (Sec. 4.2).
 */
#ifndef RANDID_H
#define RANDID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define ID_OK 0
#define ID_WARN_TOL_NOT_MET 1  /* rank cap (k_max or min(m,n)) reached with E > tol */
#define ID_WARN_ZERO_PIVOT 2   /* an exactly zero pivot column was met */
#define ID_ERR_NONFINITE (-101) /* A holds NaN or Inf (checked before factoring) */
#define ID_ERR_CUDA (-102)      /* a CUDA runtime call failed */
#define ID_ERR_TIMEOUT (-103)   /* a bounded device-side wait gave up */
#define ID_ERR_WORKSPACE (-104) /* workspace NULL, misaligned or too small */
#define ID_ERR_UNSUPPORTED (-105) /* dtype / precision combination not built */

/* ---------------------------------------------------------------- types */
typedef enum {
  ID_F64 = 0,
  ID_F32 = 1,
  ID_BF16 = 2,
  ID_FP8_E4M3 = 3,
  /* sketch_prec only, with F64 A and lu_prec F64: the sketch computed to FP64
     accuracy on the BF16 tensor cores by exact integer slicing.  A is split once
     per call into 7 digit slices of 8 bits with per-column exponents (56 bits);
     Omega is the Gaussian on the grid 2^-11 (|q| <= 16383), split into 2 digits;
     every digit product is kept and summed exactly in FP32 over chunks of 512
     and in int64 across chunks.  Entry error <= 2^-52 max_i|A_ij|
     sum_r |Omega_cr|.  The Schur GEMM and the block update of X run on the
     tensor cores the same way (7 digits of 8 bits per operand).  A caller omega
     (F64) is rounded to the same grid.  Extra workspace: 14 bytes per element
     of A plus 14 bytes per element of T(act, 0:k). */
  ID_F64_EMU = 4,
  /* sketch_prec only, with F32 A and lu_prec F32: the sketch on the BF16 tensor
     cores with A and Omega each split into 3 digits of 8 bits (per-column /
     per-row exponents); the 6 leading digit products are summed exactly in
     FP32 over chunks of 320 and in int64 across chunks.  FP32-level accuracy;
     Omega is the FP32 Gaussian (not rounded to a grid).  Extra workspace:
     6 bytes per element of A. */
  ID_F32_EMU = 5
} id_dtype;

/* An input matrix: DEVICE data, column-major m x n, leading dimension ld >= m. */
typedef struct {
  const void* data;
  id_dtype dtype;
  int64_t m, n, ld;
  /* ID_FP8_E4M3 only: one FP32 scale per 128-row block of each column,
     column-major ceil(m/128) x n (ld = ceil(m/128)); the value of entry (i,j)
     is fp8(i,j) * block_scale[i/128 + j*ceil(m/128)].  NULL otherwise. */
  const float* block_scale;
} id_matrix;

typedef struct {
  /* Precision triples (A->dtype, sketch_prec, lu_prec) built; others return
     ID_ERR_UNSUPPORTED:
       F64 / F64 / F64            FP64 throughout (FP64 FMA sketch)
       F64 / F64_EMU / F64        FP64-accurate sketch on the tensor cores
       F32 / F32 / F32            FP32 throughout
       F32 / F32_EMU / F32        FP32-accurate sketch on the tensor cores
       BF16 / BF16 / F32          tensor-core sketch, FP32 LU and X
       FP8_E4M3 / FP8_E4M3 / F32  tensor-core sketch with block scales, FP32 LU and X
     ||A||_F and the estimate's sum of squares are FP64 on every path. */
  id_dtype sketch_prec; /* inputs of the sketch GEMM */
  id_dtype lu_prec;     /* Schur complement, LUPP and X */
  int64_t block;        /* b, rows of each sketch block (Algorithm 1); default 64 */
  double tol;           /* tau */
  int tol_relative;     /* 1: stop when E <= tol * ||A||_F; 0: E <= tol (Algorithm 1) */
  int64_t k_max;        /* capacity of J and X; rank never exceeds min(m, n, k_max) */
  int64_t k0;           /* rows of the first sketch pass (a rank guess, e.g. from the
                           learned predictor); 0 = one block.  Same J, X, k as k0 = 0. */
  int64_t blocks_per_pass; /* sketch blocks drawn per later pass over A; 0 = automatic:
                              2 on the ID_F64_EMU tensor-core sketch, 4 on
                              ID_F32_EMU and on the FP32 sparse-sign sketch, 8 on the
                              BF16 and FP8 tensor-core sketches, 1 elsewhere (J, X and
                              k do not depend on it) */
  uint64_t seed;        /* key of the Philox4x64-10 generator of Omega */
  /* Optional caller-supplied sketching matrix: DEVICE, row-major omega_rows x m
     with row stride ld_omega >= m, dtype sketch_prec.  Block t uses rows
     [t*b, t*b+b); omega_rows must cover every row the run may draw.
     NULL = generate from `seed`. */
  const void* omega;
  int64_t ld_omega, omega_rows;
  int profile;          /* 1: time each phase with CUDA events (id_result.phase_ms) */
  /* Optional learned rank predictor (DEVICE, id_mlp_param_count() floats, see
     id_mlp_forward).  When set, id_adaptive evaluates it on the pivots of the
     first block and sketches the blocks up to the predicted rank in as few
     passes over A as max_pass_rows allows.  J, X and k are those of the plain
     loop (the rows are counter-based and LUPP pivots do not depend on later
     columns); only the number of passes over A changes. */
  const float* predictor;
  int64_t max_pass_rows;  /* rows per pass the predictor may request; 0 = 16 b */
  /* The condition of L1 (the k x k unit-lower factor on the skeleton rows) and the
     precision of the solve X^T(J^c,:) = L2 L1^{-1} (Eq. inty):
       0  no estimate; X as computed in lu_prec;
       1  compute kappa_1(L1) = ||L1||_1 ||L1^{-1}||_1 into id_result.cond_L1 and,
          with lu_prec F32, re-solve X in FP64 from the stored LU multipliers when
          kappa_1(L1) > ID_COND_SWITCH (an FP32 X would keep fewer than half of
          its digits);
       2  as 1, and always re-solve in FP64 with lu_prec F32.
     Modes 1 and 2 add n x k_max multipliers (lu_prec) to the workspace, and with
     lu_prec F32 the FP64 solve's k_max x k_max and n x k_max FP64 buffers. */
  int x_solve_f64;
  /* The sketching matrix the library generates (omega = NULL):
       ID_OMEGA_GAUSSIAN    N(0,1) rows (Philox4x64-10 + Box-Muller, see id_gaussian_rows);
       ID_OMEGA_SPARSE_SIGN the sparse-sign matrix of Sec. 5.1: every column of every
                            b-row block holds zeta entries +-sqrt(b/zeta) at distinct
                            rows (see id_sparse_sign_rows), so the sketch is a
                            gather-add that reads A once per pass, in A's own
                            precision (FP32 sums for BF16).  Built for A F64, F32 and
                            BF16; with sketch_prec F64_EMU / F32_EMU the gather-add
                            replaces the digit-sliced sketch and the tensor-core
                            Schur GEMM and block update remain.  b <= 128. */
  int omega_kind;
  int64_t zeta;   /* nonzeros per column of a sparse-sign block, 1 <= zeta <= b; 0 = 8 */
} id_opts;

#define ID_OMEGA_GAUSSIAN 0
#define ID_OMEGA_SPARSE_SIGN 1

/* kappa_1(L1) above which x_solve_f64 = 1 re-solves an FP32 X in FP64 (2^12). */
#define ID_COND_SWITCH 4096.0

/* Phases reported in id_result.phase_ms / phase_launches. */
enum {
  ID_PHASE_OMEGA = 0,  /* generate Gaussian rows */
  ID_PHASE_SKETCH = 1, /* Y = Omega A (GEMM) and its split-K reduction */
  ID_PHASE_SCHUR = 2,  /* S = (PY)_2 - L2 L1^{-1} (PY)_1 and ||S||_F^2 */
  ID_PHASE_LU = 3,     /* LUPP of S */
  ID_PHASE_UPDATE = 4, /* interpolation-matrix update, re-blocking */
  ID_PHASE_OTHER = 5,  /* norm, checks, finalisation */
  ID_NUM_PHASES = 6
};

typedef struct {
  int64_t k;        /* HOST out: rank of the ID */
  int64_t* J;       /* DEVICE out: int64[k_max] (k used) column skeletons in pivot order */
  void* X;          /* DEVICE out: lu_prec, k_max x n column-major, leading dim ldx >= k_max;
                       rows 0..k-1 hold X, X(:,J) = I_k; rows >= k are unspecified */
  int64_t ldx;
  double* pivots;   /* optional DEVICE out: double[k_max], |U(i,i)| of the LUPP */
  double* est_trace;/* optional HOST out: E^(t) for t = 1, 2, ... (trace_cap entries) */
  int64_t trace_cap;
  double est_err;   /* HOST out: last estimate E (0 when k = n) */
  double norm_A;    /* HOST out: ||A||_F */
  int32_t rounds;   /* HOST out: estimates computed (Algorithm 1 loop trips) */
  int32_t passes;   /* HOST out: sketch passes over A */
  int64_t launches; /* HOST out: kernels launched by this call */
  double phase_ms[ID_NUM_PHASES];      /* HOST out when opts->profile */
  int64_t phase_launches[ID_NUM_PHASES];
  int32_t status;   /* HOST out: this problem's status (id_batched: per problem; otherwise
                       equal to the return value) */
  double cond_L1;   /* HOST out (x_solve_f64 != 0): kappa_1(L1) = ||L1||_1 ||L1^{-1}||_1, else 0 */
  int32_t x_f64;    /* HOST out: 1 if X was re-solved in FP64 */
} id_result;

/* ---------------------------------------------------------------- entry points */

/* Workspace bytes for id_fixed_rank (l > 0: sketch rows) or id_adaptive (l = 0).
   Returns ID_OK or -i for an invalid argument. */
int id_workspace_size(const id_matrix* A, const id_opts* opts, int64_t l, size_t* bytes);

/* randLUPP, fixed rank (Sec. 3.1; dong2022 Algorithm 2 as the paper cites it):
   Y = Omega(0:l,:) A, LUPP of Y^T, J = the first k pivots, X = [I, (L2 L1^{-1})^T]
   permuted back (Eq. inty).  If l > k the l-k extra rows give the Schur estimate
   E = ||S||_F / sqrt(l-k) of the rank-k ID (Eq. errSch) in out->est_err.
   Requires 1 <= k <= min(m, n, l); out->X needs ldx >= k. */
int id_fixed_rank(const id_matrix* A, int64_t k, int64_t l, const id_opts* opts,
                  void* ws, size_t ws_bytes, id_result* out, void* stream);

/* randLUPPadap (Algorithm 1, Sec. 4): blocks of b sketch rows; each round forms
   S = (P Y)(tb+1:,:) - L2 L1^{-1} (P Y)(1:tb,:) for a fresh block, stops when
   E = ||S||_F / sqrt(b) <= tau (returning k = tb, the rank E certifies), else
   factors S by LUPP and re-blocks.  The minimum rank is min(b, cap); at
   k = min(m, n, k_max) with E > tau it returns ID_WARN_TOL_NOT_MET. */
int id_adaptive(const id_matrix* A, const id_opts* opts, void* ws, size_t ws_bytes,
                id_result* out, void* stream);

/* Batched adaptive IDs (the paper's future-work item 3, Sec. 6): `count`
   independent problems A[i] (HOST array of descriptors, DEVICE data, one dtype:
   F64 or F32 with sketch_prec = lu_prec = that dtype, n <= 4096 each) run
   Algorithm 1 with the shared options in ONE persistent kernel launch replayed
   from a CUDA graph: each CTA takes problems from a work queue (largest m*n
   first) and runs every step of the method for it with CTA-local
   synchronisation.  opts->block defaults to 32 here and is at most 32;
   opts->omega must be NULL (Gaussian rows come from opts->seed, the same
   counters as id_adaptive); k0 and blocks_per_pass are ignored.  out is a HOST
   array of `count` results with caller-owned J / X per problem (ldx >= the
   problem's rank cap); per-problem k, est_err, norm_A, rounds and status are
   filled.  The return value is the most severe per-problem status.  The CTA
   GEMM tile height and CTAs per SM are picked by a built-in autotuner on the
   first call for a size class (the environment variable
   RANDID_BATCHED_CONFIG=<32|64>x<1|2> pins them); results do not depend on the
   choice. */
int id_batched_workspace_size(int64_t count, const id_matrix* A, const id_opts* opts,
                              size_t* bytes);
int id_batched(int64_t count, const id_matrix* A, const id_opts* opts, void* ws,
               size_t ws_bytes, id_result* out, void* stream);

/* Two-sided ID from a column skeleton (Sec. 2.2.1 "Two-sided ID", Sec. 3.1):
   LUPP of C = A(:,J) (m x k, the columns J gathered on the device) picks the row
   skeletons I (k, DEVICE int64, pivot order), and W (m x k, column-major, ldw >= m,
   dtype of A) = P^T [I; L2 L1^{-1}] (Eq. inty) satisfies C = W C(I,:), W(I,:) = I_k,
   so that A ~ W A(I,J) X with the column ID's X.  The paper derives the row
   skeletons of a CUR factorisation the same way (LUPP on the selected columns,
   Sec. 3.1).  A: F64 or F32.  J: DEVICE int64[k]; an entry outside [0, n) returns
   -2.  ws: id_cur_workspace_size bytes, 256-aligned. */
int id_cur_workspace_size(const id_matrix* A, int64_t k, size_t* bytes);
int cur_from_id(const id_matrix* A, const int64_t* J, int64_t k, int64_t* I, void* W,
                int64_t ldw, void* ws, size_t ws_bytes, void* stream);

/* A-posteriori certificate of a column ID (the certificate Remark 1 points to,
   Sec. 3.2; its square is unbiased by Sec. 4.2):
     E_post = || Omega' A - (Omega' A)(:,J) X ||_F / sqrt(q)
   with q fresh Gaussian rows Omega' drawn after J was fixed.  A: any input the
   sketch supports, with sketch_prec as for id_sketch (F64 / F64_EMU for F64 A,
   F32 / F32_EMU for F32 A, BF16, FP8_E4M3 with block scales).  J: DEVICE int64[k]
   (an entry outside [0, n) returns -2).  X: DEVICE, k x n column-major (ldx >= k),
   FP64 for F64 A and FP32 otherwise (the X an ID of this library returns).
   Omega': omega = NULL draws rows [row0, row0 + q) of the Philox generator keyed
   by `seed` (pass a seed, or rows, the ID did not use); else omega is DEVICE,
   row-major q x m (row stride ld_omega >= m) in the sketch's input type.
   est: HOST out.  ws: id_certificate_workspace_size bytes, 256-aligned.
   Synchronises the stream. */
int id_certificate_workspace_size(const id_matrix* A, int64_t k, int64_t q, id_dtype sketch_prec, size_t* bytes);
int id_certificate(const id_matrix* A, const int64_t* J, const void* X, int64_t ldx, int64_t k, int64_t q,
                   id_dtype sketch_prec, uint64_t seed, int64_t row0, const void* omega, int64_t ld_omega,
                   double* est, void* ws, size_t ws_bytes, void* stream);

/* The residual block U_r of Remark 1 (Sec. 3.2), column form: the fixed-rank
   ID of rank k from l = k + p sketch rows (as id_fixed_rank, results in out),
   then LUPP of the transposed sketch continued for p more steps, so that
   P Y^T = [L1; L2 L_r][U1 U2; 0 U_r] with U_r the trailing p x p block.
   U_r: DEVICE out, p x p column-major (ldu >= p), lu_prec, zero below the
   diagonal.  J_extra: optional DEVICE out, int64[p], the columns of A picked by
   the p extra pivots.  stats (HOST out): u_fro = ||U_r||_F, u_max = max|U_r(i,j)|,
   est = ||L_r U_r||_F / sqrt(p) (the Schur estimate of Eq. errSch for rank k),
   bound = sqrt(n-k) ||U_r||_F (the remark's bound, from |L_r| <= 1).  Eq. normUest
   and Eq. maxUest multiply u_fro and u_max by (4 log k / k) sqrt(n-k); the paper
   supports that factor only with a figure, so it is left to the caller.
   Requires 1 <= p <= 128 and k + p <= min(m, n).  ws: id_workspace_size(A, opts,
   k + p) bytes.  Argument codes: A -1, k -2, p -3, opts -4, ws/ws_bytes
   ID_ERR_WORKSPACE, out -7, U_r/ldu -8, stats -11. */
typedef struct {
  double u_fro, u_max, est, bound;
} id_ur_stats;
int id_ur_estimates(const id_matrix* A, int64_t k, int64_t p, const id_opts* opts, void* ws, size_t ws_bytes,
                    id_result* out, void* U_r, int64_t ldu, int64_t* J_extra, id_ur_stats* stats, void* stream);

/* The stable interpolation matrix of a column skeleton (Eq. sID in column form,
   Sec. 2.2; the stable-ID error of Sec. 5.1): X = A(:,J)^+ A, the least-squares
   coefficients of every column of A on the skeleton columns, through a
   Householder QR of C = A(:,J) = Q R on the device (LAPACK dgeqrf's reflectors,
   panels of 32 columns): X = R^{-1} Q^T A.  ||A - A(:,J) X||_F is the stable
   ID error, at most the ID's.  A: F64 or F32 (computed in A's precision).
   J: DEVICE int64[k] (an entry outside [0, n) returns -2).  X: DEVICE out,
   k x n column-major (ldx >= k), A's dtype.  ws: id_stable_x_workspace_size
   bytes (2 m k + 2 k n elements and the QR's scratch), 256-aligned.
   Synchronises the stream. */
int id_stable_x_workspace_size(const id_matrix* A, int64_t k, size_t* bytes);
int id_stable_x(const id_matrix* A, const int64_t* J, int64_t k, void* X, int64_t ldx, void* ws, size_t ws_bytes,
                void* stream);

/* The middle factor of a CUR or two-sided ID from row skeletons I and column
   skeletons J (Sec. 2.2.1; Sec. 3.1 derives I by LUPP of A(:,J), which
   cur_from_id computes):
     middle_kind ID_CUR_PSEUDOINVERSE  U = C^+ A R^+ with C = A(:,J), R = A(I,:),
                                       the Frobenius-optimal middle factor of CUR,
                                       through Householder QRs of C and R^T:
                                       U = Rc^{-1} (Qc^T A Qr) Rr^{-T};
     middle_kind ID_CUR_INVERSE        U = A(I,J)^{-1} (the two-sided ID's middle
                                       matrix inverted: C U R interpolates A on the
                                       rows I and the columns J), through a QR of
                                       A(I,J).
   A: F64 or F32.  I, J: DEVICE int64[k] (entries outside A return -2).  U: DEVICE
   out, k x k column-major (ldu >= k), A's dtype.  ws: cur_middle_workspace_size
   bytes, 256-aligned.  Synchronises the stream. */
#define ID_CUR_PSEUDOINVERSE 0
#define ID_CUR_INVERSE 1
int cur_middle_workspace_size(const id_matrix* A, int64_t k, int middle_kind, size_t* bytes);
int cur_middle(const id_matrix* A, const int64_t* I, const int64_t* J, int64_t k, void* U, int64_t ldu,
               int middle_kind, void* ws, size_t ws_bytes, void* stream);

/* Rows [row0, row0+rows) of the Gaussian sketching matrix (row-major, row
   stride ld >= m, dtype F64, F32, BF16 or FP8_E4M3): entry (i, r) is a standard
   normal from Philox4x64-10 (Salmon et al. 2011) keyed (seed, 0) at counter
   (r/4, i, 0, 0) and Box-Muller on 53-bit uniforms in FP64 (Sec. 2.4, Sec. 5.1);
   for BF16 and FP8_E4M3 output Box-Muller runs in FP32 on the leading 24 bits of
   the same counters.  Rounded to nearest-even in the output type (E4M3
   saturating at +-448).  dtype ID_F64_EMU: the rows the FP64-accurate sketch
   uses, rint(2^11 z) / 2^11 with |rint(2^11 z)| clamped to 16383 (z the FP64
   value above), written as F64 by the generator that path runs (FP32 Box-Muller,
   FP64 recomputation of the samples near a rounding boundary).
   Synchronises the stream. */
int id_gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, id_dtype dtype,
                     void* out, int64_t ld, void* stream);

/* Blocks t0 .. t0+blocks-1 of the sparse-sign sketching matrix (Sec. 5.1,
   "Sparse Sign"; zeta = 8 in the paper) as dense rows: block t0+q occupies rows
   q*b .. q*b+b-1 of out (DEVICE, row-major, row stride ld >= m, dtype F64 or F32).
   Column i of block t holds zeta nonzeros +-sqrt(b/zeta) at distinct rows:
   the words u_0, u_1, ... are Philox4x64-10 (Salmon et al. 2011) keyed (seed, 1)
   at counters (i, t, c, 0), four words per counter; a partial Fisher-Yates
   shuffle of (0..b-1) puts nonzero j at row p[j] after swapping p[j] with
   p[j + ((u_j >> 32) (b - j)) >> 32], negative when u_j is odd.  The scale makes
   E[Omega^T Omega] = b I, as for N(0,1) rows, so the estimator keeps its scale.
   Requires 1 <= zeta <= b <= 128.  Synchronises the stream. */
int id_sparse_sign_rows(uint64_t seed, int64_t t0, int64_t blocks, int64_t b, int64_t m, int64_t zeta,
                        id_dtype dtype, void* out, int64_t ld, void* stream);

/* The sparse-sign sketch alone: G = (Omega A)^T for rows [t0*b, t0*b + rows) of
   the sparse-sign matrix above (n x rows, row-major, row stride ldg >= rows; FP64
   for F64 A, FP32 for F32 and BF16 A), summed in a fixed order (deterministic).
   F64 A is summed exactly: each column in 55-bit fixed point (error <= 2^-55
   max|A(:,j)| per term, as the FP64-accurate tensor-core sketch), exact integer
   sums, one rounding to FP64 and one for the scale.  BF16 A needs an
   even leading dimension and a 4-byte aligned base (else ID_ERR_UNSUPPORTED).
   At most 65535 blocks (rows <= 65535 b).
   ws: id_sparse_sketch_workspace_size bytes, 256-aligned. */
int id_sparse_sketch_workspace_size(const id_matrix* A, int64_t rows, int64_t b, int64_t zeta, size_t* bytes);
int id_sparse_sketch(const id_matrix* A, uint64_t seed, int64_t t0, int64_t rows, int64_t b, int64_t zeta, void* G,
                     int64_t ldg, void* ws, size_t ws_bytes, void* stream);

/* FP8 storage of a matrix for the FP8 sketch: A (F64, F32 or BF16, column-major)
   -> Q (E4M3 bytes, column-major, ld ldq >= m) and one FP32 scale per 128-row
   block of each column (block_scale, column-major ceil(m/128) x n, the id_matrix
   layout).  scale = amax/448 of the block, or with pow2 != 0 the power of two
   >= amax/448 (a UE8M0-representable scale); a zero block has scale 1, a block
   holding a NaN a NaN scale.  Q(i,j) = E4M3 of A(i,j)/scale rounded to nearest
   even, saturating at +-448 (FP64 input divided in FP64, others in FP32).
   Asynchronous on `stream`.  Returns -1 (A), -2 (Q/ldq), -4 (block_scale). */
int id_quantize_fp8(const id_matrix* A, void* Q, int64_t ldq, float* block_scale, int pow2, void* stream);

/* The sketch alone (Sec. 2.4; the sampling step of Algorithm 1): G = (Omega A)^T, n x rows,
   row-major with row stride ldg >= rows (row j holds the sketch of column j).
   omega: DEVICE, row-major rows x m, row stride ld_omega >= m, dtype sketch_prec.
   Paths: A F64 / sketch F64 (FP64 FMA, G in FP64); A F32 / F32 (FP32 FMA, G in
   FP32); A BF16 / BF16 (tcgen05 tensor cores fed by TMA, FP32 accumulation, G in
   FP32; A->ld and ld_omega multiples of 8, 16-byte aligned bases, else
   ID_ERR_UNSUPPORTED); A FP8_E4M3 / FP8_E4M3 (block scales in A->block_scale,
   tcgen05 kind::f8f6f4, FP32 accumulation per 128-row block, G in FP32; A->ld
   and ld_omega multiples of 16); A F64 / ID_F64_EMU (omega F64, rounded to the grid 2^-11,
   then the FP64-accurate digit-sliced product on the tensor cores, G in FP64).
   ws: at least id_sketch_workspace_size bytes, 256-aligned. */
int id_sketch_workspace_size(const id_matrix* A, int64_t rows, id_dtype sketch_prec, size_t* bytes);
int id_sketch(const id_matrix* A, const void* omega, int64_t ld_omega, int64_t rows, id_dtype sketch_prec,
              void* G, int64_t ldg, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- learned rank predictor
   A 35 -> 128 -> 128 -> 1 MLP with tanh hidden layers, FP32.  Parameter block
   (id_mlp_param_count() floats): W1 [128 x 35] row-major, b1 [128], W2 [128 x 128],
   b2 [128], w3 [128], b3, then the input standardisation mu [35], sigma [35] and
   the output scale y_mu, y_sigma.  Inputs (id_rank_features): log10 of the first
   32 LUPP pivot magnitudes of the first sketch block relative to the first
   (Remark 1 ties them to the spectrum), log10 m, log10 n, log10 of the relative
   tolerance.  Output: log2 of the rank of the adaptive loop.  The trainable
   parameters are the first 21249 entries. */
#define ID_MLP_IN 35
#define ID_MLP_HIDDEN 128
int64_t id_mlp_param_count(void);
/* y[i] = predicted log2 rank for the feature row x[i*35 .. i*35+34] (DEVICE). */
int id_mlp_forward(const float* params, int64_t batch, const float* x, float* y, void* stream);
/* loss = mean_i (yhat_i - t_i)^2 on the standardised output (t_i = (target_i - y_mu)
   / y_sigma) and its gradient w.r.t. the 21249 trainable parameters (DEVICE).
   Deterministic (one CTA, fixed summation order). */
int id_mlp_loss_grad(const float* params, int64_t batch, const float* x, const float* target, float* grad,
                     float* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step counts from 1) on the
   trainable parameters; m1, m2: DEVICE moment buffers of 21249 floats. */
int id_mlp_adam(float* params, const float* grad, float* m1, float* m2, int64_t step, float lr, void* stream);
/* The 35 features from the pivots |U(i,i)| of the first block (DEVICE doubles). */
int id_rank_features(const double* pivots, int64_t npiv, int64_t m, int64_t n, double rel_tol, float* x,
                     void* stream);

/* Human-readable text for a status value. */
const char* id_status_string(int status);

/* Self-test of the failure handling; the paper has no counterpart.  Every
   device-side wait of the library gives up after a bounded time (4 s of the
   GPU's global timer).  That covers the grid barrier of the cooperative LUPP
   panel and the mbarrier waits of the tensor-core kernels.  The wait records a
   timeout and lets its kernel exit, so the call returns ID_ERR_TIMEOUT and the
   CUDA context stays usable.  This entry runs, with the same device helpers,
   one wait that nothing can satisfy: which = 0 the grid barrier, which = 1 an
   mbarrier wait.
   ws: DEVICE scratch of at least 256 bytes, 256-aligned, owned by the caller.
   Synchronises the stream and takes about 4 s.  Returns ID_ERR_TIMEOUT when
   the wait gave up as designed.  ID_OK would mean the wait was satisfied.
   Other returns: -1 for another `which`, ID_ERR_WORKSPACE, ID_ERR_CUDA. */
int id_selftest_timeout(int which, void* ws, size_t ws_bytes, void* stream);

/* Bytes of the library-owned device buffer behind id_fixed_rank_noalloc. */
#define ID_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* id_fixed_rank for callers that cannot allocate device memory.  The paper has
   no counterpart: this is a deployment variant of id_fixed_rank.

   Some callers may not call cudaMalloc at all, or not at the moment they need
   an ID.  Examples: a host application that reserved the GPU's memory up front
   for its own pool, or a loop with latency or certification rules that forbid
   device allocation after start-up, since cudaMalloc and cudaFree can block the
   device.  They still own and pass A, J and X; the scratch the method needs
   comes from one buffer of ID_NOALLOC_SCRATCH_BYTES that the library defines as
   a static device array.

   When the buffer exists on a device: it belongs to the library's device code,
   which CUDA loads into each device's context.  Under CUDA's default lazy
   module loading that happens on the first call of this function on the
   device (the buffer's address lookup), and that load allocates the
   ID_NOALLOC_SCRATCH_BYTES.  So make the first call on each device at
   start-up: before the caller reserves its memory pool or forbids
   allocation, and before any stream capture.  (With CUDA_MODULE_LOADING=EAGER
   the buffer is allocated when the context is created.)  From then on the
   device holds the buffer until the process exits, and later calls allocate
   nothing.

   Arguments and results are those of id_fixed_rank without ws / ws_bytes, so
   a negative argument code -i counts this function's own positions: A = -1,
   k = -2, l = -3, opts = -4, out = -5 (id_fixed_rank reports a bad out as -7).
   opts->profile is ignored (no timing events are created).  A problem whose
   scratch (the id_workspace_size value for the same A, opts and l) exceeds
   ID_NOALLOC_SCRATCH_BYTES is rejected with ID_ERR_WORKSPACE before anything
   runs.  Calls share the buffer and each call re-initialises what it reads,
   but calls that overlap on the GPU (other streams, other host threads) race
   on it: serialise them.  Nothing here calls cudaMalloc, cudaFree or an
   allocating library routine. */
int id_fixed_rank_noalloc(const id_matrix* A, int64_t k, int64_t l, const id_opts* opts,
                          id_result* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RANDID_H */
