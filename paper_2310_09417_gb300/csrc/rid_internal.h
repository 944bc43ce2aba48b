// rid_internal.h -- launchers shared between the kernel files and the C-ABI
// driver.  Every launcher enqueues on `s`, returns the launch error, and does
// nothing when *done (a device flag) is already set, so rounds enqueued past
// the stopping point cost only their launch.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "rid_common.cuh"

namespace rid {

// The dynamic shared-memory limit of a kernel (cudaFuncSetAttribute), set to
// what its launches use before the first one and raised when a launch needs
// more.  By default the limit is 48 KB minus the kernel's static shared memory,
// so it is set whatever the size.  The attribute belongs to each device's
// context, so the size already set is kept per device.  The check is an atomic
// load; the call runs under a lock, so that concurrent callers never lower a
// limit another one relies on.
constexpr int kMaxDevices = 64;
struct SmemLimit {
  std::atomic<size_t> raised[kMaxDevices];
};
inline std::mutex& smem_limit_mutex() {
  static std::mutex m;
  return m;
}
template <typename K>
inline cudaError_t raise_smem(K* func, size_t bytes, SmemLimit& lim) {
  if (bytes == 0) return cudaSuccess;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool keep = dev >= 0 && dev < kMaxDevices;
  if (keep && lim.raised[dev].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
  std::lock_guard<std::mutex> guard(smem_limit_mutex());
  if (keep && lim.raised[dev].load(std::memory_order_relaxed) >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(reinterpret_cast<const void*>(func), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes);
  if (e == cudaSuccess && keep) lim.raised[dev].store(bytes, std::memory_order_release);
  return e;
}

// Operand of the gather-GEMM: row r lives at base + (idx ? idx[r] : r) * ld + off.
template <typename T>
struct Operand {
  const T* base;
  int64_t ld;
  const int32_t* idx;
  int64_t off;
};

// Epilogues of the gather-GEMM.
enum GemmEpi : int {
  kEpiStore = 0,    // out[z*zstride + r*out_ld + c] = acc          (split-K partials)
  kEpiSubRows = 1,  // out[out_idx[r]*out_ld + c] -= acc, rows with skip[r] != 0 left alone
};

template <typename T>
struct EpiArgs {
  T* out;
  int64_t out_ld;
  int64_t zstride;
  const int32_t* out_idx;
  const int32_t* skip;
};

// C (M x N) = sum_k A_r[k] * B(k, c).  A rows are contiguous along K.  B is
// K-major (b_kmajor: row c contiguous along K) or N-major (row k contiguous
// along N).  The K range is split across gridDim.z in chunks of `kchunk`.
// The split count actually used (<= requested) is what gemm_splits() returns.
int gemm_splits(int K, int splits);
template <typename T>
cudaError_t gemm_gather(int M, int N, int K, int splits, bool b_kmajor, Operand<T> a, Operand<T> b,
                        int epi, EpiArgs<T> ep, const int32_t* done, cudaStream_t s);

template <typename T>
cudaError_t gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, T* out, int64_t ld,
                          const int32_t* done, cudaStream_t s);

// ||A||_F^2 partial sums (one per block, fixed partition) + finiteness check.
template <typename T>
cudaError_t norm2_partial(int64_t m, int64_t n, const T* A, int64_t lda, double* part, int nparts,
                          DevState* st, cudaStream_t s);
cudaError_t norm2_final(const double* part, int nparts, DevState* st, cudaStream_t s);

// G[j*ldg + c] = sum_z P[z*zs + j*ldg + c]
template <typename T>
cudaError_t splitk_reduce(int64_t n, int rows, int64_t ldg, int nz, int64_t zs, const T* P, T* G,
                          const int32_t* done, cudaStream_t s);
// the same with partials of row stride ldp: G[j*ldg + c] = sum_z P[z*zs + j*ldp + c]
template <typename T>
cudaError_t splitk_reduce_ld(int64_t n, int rows, int64_t ldp, int64_t ldg, int nz, int64_t zs, const T* P, T* G,
                             const int32_t* done, cudaStream_t s);

// S[i*lds + c] = G[act[i]*ldg + col0 + c] - sum_z P[z*zs + i*lds + c]; e2part[blk] = sum S^2
template <typename T>
cudaError_t schur_finish(int na, int w, const int32_t* act, const T* G, int64_t ldg, int64_t col0,
                         int nz, int64_t zs, const T* P, T* S, int64_t lds, double* e2part, int nparts,
                         const int32_t* done, cudaStream_t s);

// E = sqrt(sum e2part / w); stop test against tau (absolute or relative to ||A||_F).
cudaError_t decide(const double* e2part, int nparts, int w, double tol, int tol_rel, int64_t tb,
                   int last, double* trace, int round, DevState* st, cudaStream_t s);

// Cooperative LUPP of S (na x w, row-major, ld lds) for `steps` pivots.
struct PanelCfg {
  int grid;
  int chunk;
  int use_smem;
  size_t smem;
};
template <typename T>
PanelCfg panel_config(int na, int w, int num_sms);
// Rows per block and shared memory of the panel kernel for a given block count.
template <typename T>
PanelCfg panel_layout(int na, int w, int grid);
template <typename T>
cudaError_t panel_lupp(const PanelCfg& cfg, int na, int w, int steps, int par, T* S, int64_t lds,
                       int32_t* piv, int32_t* pivmark, double* pivdiag, double* cand_v,
                       int32_t* cand_i, T* cand_rows, DevState* st, cudaStream_t s);

// Inverse of the unit-lower block L-hat(piv, 0:bt) (bt x bt, row-major).
template <typename T>
cudaError_t linv(int bt, const T* S, int64_t lds, const int32_t* piv, T* Linv, const int32_t* done,
                 cudaStream_t s);

// N = L-hat(rest) * Linv; X(tb:tb+bt, act[i]) = N(i,:) for non-pivot rows; pivorig = act[piv].
template <typename T>
cudaError_t make_n(int na, int bt, const T* S, int64_t lds, const T* Linv, const int32_t* pivmark,
                   const int32_t* act, T* Nbuf, T* X, int64_t ldx, int64_t tb, const int32_t* piv,
                   int32_t* pivorig, const int32_t* done, cudaStream_t s);

// Drop the new pivots from the active list (stable), append them to J / perm32.
cudaError_t compact(int na, int bt, const int32_t* act_in, int32_t* act_out, int32_t* pivmark,
                    const int32_t* piv, int64_t* J, int32_t* perm32, int64_t tb, double* pivots_out,
                    const double* pivdiag, const int32_t* done, cudaStream_t s);

// X(:, perm32[q]) = e_q for q < k.
template <typename T>
cudaError_t finalize_x(int64_t k, const int32_t* perm32, T* X, int64_t ldx, cudaStream_t s);

cudaError_t init_state(DevState* st, int32_t* act, int32_t* pivmark, int64_t n, cudaStream_t s);

// G (m x k row-major) = A(:, J); W (m x k column-major) = X^T.
template <typename T>
cudaError_t gather_panel(const T* A, int64_t lda, int64_t m, int64_t n, const int64_t* J, int64_t k, T* G,
                         DevState* st, cudaStream_t s);
template <typename T>
cudaError_t transpose_w(const T* X, int64_t ldx, int64_t m, int64_t k, T* W, int64_t ldw, cudaStream_t s);

// ---- condition of L1 and the FP64 solve for X (rid_cond.cu).  Blocks are at most
// kMaxBlockCond wide.  L: the LUPP multipliers by original row (row stride ldl), columns
// in pivot order; Linv_all: the inverse diagonal blocks, block t at t*b*b (row-major bt x bt).
constexpr int kMaxBlockCond = 128;
template <typename T>
cudaError_t store_l(int na, int bt, const T* S, int64_t lds, const int32_t* piv, const int32_t* pivmark,
                    const int32_t* act, T* L, int64_t ldl, int64_t tb, const int32_t* done, cudaStream_t s);
// column sums of |L1| (skipped when L is null) and of |L1^{-1}| (from the pivots' rows of T in X)
template <typename T>
cudaError_t cond_colsums(int64_t k, int b, const int32_t* perm, const T* L, int64_t ldl, const T* X, int64_t ldx,
                         const T* Linv_all, double* colsum_l1, double* colsum_inv, cudaStream_t s);
// X(0:k, act[r]) = (L2 L1^{-1})(r, :) solved in FP64 from L; L1 (k x k), T64 (na x k),
// Linv64 (b x b) FP64 and iota (k) are scratch.
template <typename T>
cudaError_t resolve_x_f64(int64_t k, int b, int64_t na, const int32_t* perm, const int32_t* act, const T* L,
                          int64_t ldl, double* L1, double* T64, double* Linv64, int32_t* iota, T* X, int64_t ldx,
                          cudaStream_t s, int* launches);

// ---- learned rank predictor (rid_mlp.cu): features of the first block's pivots, one
// forward pass, ceil(2^output) written to st->k_pred.
cudaError_t mlp_predict_rank(const float* params, const double* piv, int npiv, int64_t m, int64_t n, double tol,
                             int tol_rel, DevState* st, cudaStream_t s);

// ---- FP64-accurate sketch on the tensor cores (rid_tc_f64.cu).  A is split once into
// 7 BF16 digit slices (slice-major; each slice stored as contiguous 128-column x 64-row
// K-major tiles, f64emu_digit_bytes in all) with column exponents; Omega rows are quantised to the grid 2^-11 and split into
// 2 digit planes (each rows_alloc x f64emu_pad(m)); out[z] (n x rows, FP64) holds split z
// of (Omega A)^T.
int64_t f64emu_pad(int64_t m);
size_t f64emu_digit_bytes(int64_t m, int64_t n);
int f64emu_splits(int64_t m, int64_t n, int sms);
cudaError_t f64emu_prepare(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* colexp, void* digits,
                           cudaStream_t s);
cudaError_t f64emu_omega(uint64_t seed, int64_t row0, int64_t rows, int64_t m, int64_t rows_alloc,
                         const double* src, int64_t ld_src, void* wdigits, const int32_t* done, cudaStream_t s);
// Omega's grid values rint(2048 z) / 2048 (|.| <= 16383 / 2048) from the same
// generator as f64emu_omega, as FP64 rows (row stride ld >= m).
cudaError_t f64emu_omega_grid(uint64_t seed, int64_t row0, int64_t rows, int64_t m, double* out, int64_t ld,
                              cudaStream_t s);
cudaError_t f64emu_sketch(const void* digits, const int32_t* colexp, int64_t m, int64_t n, const void* wdigits,
                          int64_t rows, int64_t rows_alloc, double* out, int64_t out_ld, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s);

// ---- FP8 sketch (rid_tc_fp8.cu): A E4M3 (m x n, column-major, ld multiple of 16) with
// FP32 scales per 128-row block of each column (column-major ceil(m/128) x n), Omega E4M3
// (rows x m, row-major, ld multiple of 16); out[z] (n x rows, FP32) holds split z of (W A)^T.
bool tc_fp8_supported(const void* A, int64_t lda, const void* W, int64_t ldw);
int tc_fp8_splits(int64_t m, int64_t n, int64_t rows, int sms);
int tc_fp8_effective_splits(int64_t m, int splits);
cudaError_t tc_sketch_fp8(const void* A, int64_t lda, int64_t m, int64_t n, const float* scale, const void* W,
                          int64_t ldw, int64_t rows, float* out, int64_t out_ld, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s);
cudaError_t norm2_fp8(int64_t m, int64_t n, const void* A, int64_t lda, const float* scale, double* part, int nparts,
                      DevState* st, cudaStream_t s);
// Q (E4M3) and the block scales of A (dtype ID_F64, ID_F32 or ID_BF16).
cudaError_t quantize_fp8(int dtype, int64_t m, int64_t n, const void* A, int64_t lda, void* Q, int64_t ldq,
                         float* scale, int pow2, cudaStream_t s);

// ---- FP64 block update of T on the tensor cores (rid_tc_update.cu): X(act[i], 0:tb) -=
// N(i, :) X(pivorig[:], 0:tb) for rows with pivmark[i] == 0; N is na x bt (row stride bt,
// bt <= 64).  ndig / pdig hold update_f64emu_digit_bytes(nrows / prows) bytes, nexp / pexp
// nrows / prows exponents.
size_t update_f64emu_digit_bytes(int64_t rows);
size_t update_f32emu_digit_bytes(int64_t rows);
// The same for FP32 T with 3 digits per operand (FP32-accurate).
cudaError_t update_f32emu(int na, int bt, int tb, const float* N, const int32_t* act, const int32_t* pivmark,
                          const int32_t* pivorig, float* X, int64_t ldx, void* ndig, int32_t* nexp, int64_t nrows,
                          void* pdig, int32_t* pexp, int64_t prows, int sms, DevState* st, const int32_t* done,
                          cudaStream_t s);
cudaError_t update_f64emu(int na, int bt, int tb, const double* N, const int32_t* act, const int32_t* pivmark,
                          const int32_t* pivorig, double* X, int64_t ldx, void* ndig, int32_t* nexp, int64_t nrows,
                          void* pdig, int32_t* pexp, int64_t prows, int sms, DevState* st, const int32_t* done,
                          cudaStream_t s);

// ---- FP64-accurate GEMM on the tensor cores (rid_tc_gemm64.cu): out[z] (M x N, row stride
// ldo) = split z of A B with A(m, k) = A[aidx[m] * lda + k] and B(k, n) = B[bidx[k] * ldb +
// boff + n], N <= 64, K <= kmax.  adig / bdig hold gemm_f64emu_digit_bytes(arows / brows,
// kmax) bytes, aexp / bexp arows / brows exponents, colmax N words.
int64_t gemm_f64emu_kpad(int64_t K);
size_t gemm_f64emu_digit_bytes(int64_t rows, int64_t Kmax);
int gemm_f64emu_splits(int64_t M, int64_t N, int64_t K, int sms);
cudaError_t gemm_f64emu(int M, int N, int K, const double* A, int64_t lda, const int32_t* aidx, const double* B,
                        int64_t ldb, int64_t boff, const int32_t* bidx, void* adig, int64_t arows, int32_t* aexp,
                        void* bdig, int64_t brows, int32_t* bexp, unsigned long long* colmax, int64_t kmax,
                        double* out, int64_t ldo, int64_t zstride, int splits, DevState* st, const int32_t* done,
                        cudaStream_t s);

// ---- FP32 sketch on the tensor cores (rid_tc_gemm64.cu, 3 digits of 8 bits per operand):
// sketch_f32emu_slice writes the digits of `rows` rows of length K (row stride lds) into
// `dig` (3 planes of rows_alloc x kpad(K)) with per-row exponents; sketch_f32emu forms
// out[z] (n x rows, FP32) = split z of (W A)^T from A's digits (rows = A's n columns)
// and W's digits.
size_t sketch_f32emu_digit_bytes(int64_t rows, int64_t K);
int sketch_f32emu_splits(int64_t m, int64_t n, int64_t unit_rows, int sms);
cudaError_t sketch_f32emu_slice(int rows, int K, const float* src, int64_t lds, void* dig, int64_t rows_alloc,
                                int32_t* ex, unsigned long long* rowmax, const int32_t* done, cudaStream_t s);
cudaError_t sketch_f32emu(int64_t m, int64_t n, int64_t rows, const void* adig, const int32_t* aexp, const void* wdig,
                          int64_t wrows, const int32_t* wexp, float* out, int64_t ldo, int64_t zstride, int splits,
                          DevState* st, const int32_t* done, cudaStream_t s);

// ---- after the ID (rid_post.cu): index conversion for gathered operands, an
// identity list, and U_r of Remark 1 from the factored extra rows.
cudaError_t index32(const int64_t* J, int64_t k, int64_t n, int32_t* out, DevState* st, cudaStream_t s);
cudaError_t iota32(int32_t* a, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t ur_extract(int p, int na, const T* S, int64_t lds, const int32_t* piv, const int32_t* act, T* U,
                       int64_t ldu, int64_t* Jx, double* stats, cudaStream_t s);

// ---- sparse-sign sketch (rid_sparse.cu; Sec. 5.1 "Sparse Sign").  Blocks of b <=
// kSparseMaxB rows with zeta nonzeros +-sqrt(b/zeta) per column.  sparse_csr writes,
// for `blocks` blocks from block t0 on, one list record per 128-row tile of A and
// block (sparse_csr_bytes in all); sparse_sketch forms split z of (Omega A)^T
// (n x rows, row stride out_ld) in out + z zstride from those lists for rows = the
// pass's rows (the last block may be cut short); sparse_dense writes the blocks as
// dense rows (row-major, row stride ld).  Split counts: sparse_splits, kind 0 for
// FP32 A, 1 for BF16, 2 for FP64 (fixed point).
constexpr int kSparseMaxB = 128;
int sparse_splits(int64_t m, int64_t n, int sms, int kind);
int sparse_csr_head(int b);
int sparse_csr_rec(int b, int zeta);
size_t sparse_csr_bytes(int64_t m, int blocks, int b, int zeta);
// esz: bytes per staged element of A in the gather (4 FP32, 2 BF16, 8 FP64 fixed point)
cudaError_t sparse_csr(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, int esz, uint16_t* R,
                       const int32_t* done, cudaStream_t s);
template <typename TA>
cudaError_t sparse_sketch(int64_t m, int64_t n, const TA* A, int64_t lda, const uint16_t* R, int zeta, int b,
                          int64_t rows, int splits, float* out, int64_t out_ld, int64_t zstride, const int32_t* done,
                          cudaStream_t s);
template <typename T>
cudaError_t sparse_dense(uint64_t seed, int64_t t0, int blocks, int b, int64_t m, int zeta, T* out, int64_t ld,
                         cudaStream_t s);
// FP64 input: column exponents and the 64-bit fixed-point copy F (m x n, ld m) made
// once per call; the sketch's entries are exact integer sums rounded once to FP64.
// With splits > 1 the 128-bit partials go to parts (16 bytes each, split z at
// z zstride, row stride pld) and are summed exactly into out.
cudaError_t sparse_fixed_prepare(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* colexp, long long* F,
                                 cudaStream_t s);
cudaError_t sparse_sketch_fixed(int64_t m, int64_t n, const long long* F, const int32_t* colexp, const uint16_t* R,
                                int zeta, int b, int64_t rows, int splits, double* out, int64_t out_ld, void* parts,
                                int64_t pld, int64_t zstride, const int32_t* done, cudaStream_t s);
// e_j with |A(:, j)| < 2^e_j (0 for a zero column), by a reduction over each column.
cudaError_t f64_colexp(const double* A, int64_t lda, int64_t m, int64_t n, int32_t* E, cudaStream_t s);

// ---- the driver's cuTensorMapEncodeTiled (nullptr when unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// ---- tensor-core sketch (rid_tc_sketch.cu): out[z] (n x rows, FP32, row stride out_ld)
// holds split z of (W A)^T for BF16 A (m x n, column-major) and W (rows x m, row-major).
// TMA needs 16-byte aligned bases and leading dimensions that are multiples of 8.
bool tc_sketch_supported(const void* A, int64_t lda, const void* W, int64_t ldw);
int tc_sketch_splits(int64_t m, int64_t n, int64_t rows, int sms);
int tc_sketch_effective_splits(int64_t m, int splits);
cudaError_t tc_sketch_bf16(const void* A, int64_t lda, int64_t m, int64_t n, const void* W, int64_t ldw,
                           int64_t rows, float* out, int64_t out_ld, int64_t zstride, int splits, DevState* st,
                           const int32_t* done, cudaStream_t s);

}  // namespace rid
