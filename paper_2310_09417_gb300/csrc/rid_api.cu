// rid_api.cu -- C ABI (include/randid.h) over the ID kernels.
//
// The drivers below walk Algorithm 1 of arXiv:2310.09417 (column form) and
// the fixed-rank randLUPP of Sec. 3.1.  Per factored block:
//   Schur      S = G(act, blk) - T(act, 0:tb) G(perm, blk)      (T = L2 L1^{-1})
//   estimate   E = ||S||_F / sqrt(w), stop test on the device
//   LUPP       of S, rows marked instead of swapped
//   re-block   N = L-hat(rest) L-hat(piv)^{-1};  T(act, tb:tb+bt) = N;
//              T(act, 0:tb) -= N T(piv, 0:tb);  act, J updated
// T is the caller's X buffer (column j of X is row j of T), so X is complete
// when the loop ends except for the identity columns at J.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "randid.h"
#include "rid_internal.h"

using namespace rid;

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kMaxBlock = 128;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

// Split-K factor of the 64 x 64 gather-GEMM (FP64 Schur products): enough blocks
// for about four waves, at least 256 K per split.
int choose_splits_gather(int64_t M, int64_t N, int64_t K, int sms, int cap) {
  const int64_t tiles = cdiv(M, 64) * cdiv(N, 64);
  int64_t s = cdiv(4 * (int64_t)sms, tiles);
  s = imin(s, imax(1, K / 256));
  s = imin(s, cap);
  return (int)imax(1, s);
}

// Split-K factor for the store GEMM (k_sgemm_gather: 128 x 64 tiles, two blocks per
// SM in FP32, one in FP64): the count (at most cap, at least 128 K per split)
// minimising waves x (K per split + a fixed cost).
int choose_splits_sgemm(int64_t M, int64_t N, int64_t K, int sms, int cap, int per_sm) {
  const int64_t tiles = cdiv(M, 128) * cdiv(N, 64);
  const int64_t slots = (int64_t)per_sm * sms;
  int best = 1;
  double best_t = 1e300;
  for (int64_t s = 1; s <= cap && (s == 1 || K / s >= 128); ++s) {
    const double t = (double)cdiv(tiles * s, slots) * ((double)cdiv(K, s) + 128.0);
    if (t < best_t * (1.0 - 1e-9)) {
      best_t = t;
      best = (int)s;
    }
  }
  return best;
}

// Input kind of the sparse-sign gather on path `path`: 1 for BF16 A, 2 for FP64 A
// (its fixed-point copy), 0 for FP32 A.
int sparse_kind(int path) { return path == 16 ? 1 : (path == 64 || path == 65 ? 2 : 0); }

// Every size and offset of one call's workspace.
struct Plan {
  int64_t m = 0, n = 0, b = 0, cap = 0, k = 0, l = 0;
  int64_t rows_first = 0, rows_pass = 0, ldg = 0, wmax = 0, max_rounds = 0;
  int64_t rows_pred = 0;  // largest pass the learned predictor may request
  int s1_cap = 1;         // largest split-K count any pass uses (sizes the partials)
  int s1_first = 1, s1_pass = 1, s2max = 8, nparts = 0, maxg = 0, sms = 0;
  bool gen_omega = true;
  size_t esz = 0;
  int path = 0;          // 64, 32 (SIMT), 16 (BF16 tensor cores), 8 (FP8 tensor cores), 65 / 33 (FP64 / FP32 by
                         // digit slicing on the tensor cores)
  int64_t ldw = 0;       // row stride of the generated Omega
  size_t wsz = 0;        // bytes per Omega element
  size_t off_state = 0, off_omega = 0, off_G = 0, off_Gpart = 0, off_S = 0, off_Spart = 0, off_N = 0,
         off_Linv = 0, off_act0 = 0, off_act1 = 0, off_pivmark = 0, off_perm32 = 0, off_piv = 0,
         off_pivorig = 0, off_pivdiag = 0, off_cand_v = 0, off_cand_i = 0, off_cand_rows = 0, off_e2 = 0,
         off_normp = 0, off_trace = 0, off_digits = 0, off_colexp = 0, total = 0;
  // condition of L1 / FP64 solve for X (opts->x_solve_f64)
  int64_t ldl = 0;
  size_t off_L = 0, off_L1 = 0, off_T64 = 0, off_Linv64 = 0, off_iota = 0, off_csum = 0;
  // path 65: digit slices of N and T(piv, old) for the tensor-core block update
  size_t off_ndig = 0, off_nexp = 0, off_pdig = 0, off_pexp = 0;
  // path 65: digit slices of T(act, 0:tb) and G(perm, cols) for the tensor-core Schur GEMM
  size_t off_adig = 0, off_aexp = 0, off_bdig = 0, off_bexp = 0, off_colmax = 0;
  size_t off_f32a = 0, off_f32ae = 0, off_f32w = 0, off_f32we = 0, off_f32rmax = 0;
  bool schur_tc = false;
  bool update_tc = false;
  bool sparse = false;  // sparse-sign sketching matrix (Sec. 5.1), generated
  int64_t zeta = 8;
  size_t off_sfix = 0, off_scol = 0;  // FP64 A in 64-bit fixed point for the exact gather-add
  bool keep_l = false, f64_solve = false;
};

// Which (input, sketch, LU) precision triples are built.
int precision_path(const id_matrix* A, const id_opts* o) {
  if (A->dtype == ID_F64 && o->sketch_prec == ID_F64 && o->lu_prec == ID_F64) return 64;
  if (A->dtype == ID_F32 && o->sketch_prec == ID_F32 && o->lu_prec == ID_F32) return 32;
  // FP32 input: FP32-accurate sketch on the tensor cores, LU and X in FP32
  if (A->dtype == ID_F32 && o->sketch_prec == ID_F32_EMU && o->lu_prec == ID_F32) return 33;
  // BF16 input: sketch on the tensor cores (FP32 accumulation), LU and X in FP32
  if (A->dtype == ID_BF16 && o->sketch_prec == ID_BF16 && o->lu_prec == ID_F32) return 16;
  // FP8 input with block scales: E4M3 sketch on the tensor cores, LU and X in FP32
  if (A->dtype == ID_FP8_E4M3 && o->sketch_prec == ID_FP8_E4M3 && o->lu_prec == ID_F32) return 8;
  // FP64 input: FP64-accurate sketch on the tensor cores, LU and X in FP64
  if (A->dtype == ID_F64 && o->sketch_prec == ID_F64_EMU && o->lu_prec == ID_F64) return 65;
  return 0;
}

// make_plan failures, mapped to argument positions by each entry point.
constexpr int kBadA = -1, kBadOpts = -2, kBadK = -3, kBadL = -4;

// Validate A and opts; on success fill the plan.  l > 0: fixed rank with k.
int make_plan(const id_matrix* A, const id_opts* o, int64_t k, int64_t l, Plan* p) {
  if (A == nullptr || A->data == nullptr) return kBadA;
  if (o == nullptr) return kBadOpts;
  if (A->m < 1 || A->n < 1 || A->ld < A->m || A->m >= (int64_t)1 << 31 || A->n >= (int64_t)1 << 30) return kBadA;
  const int path = precision_path(A, o);
  if (path == 0) return ID_ERR_UNSUPPORTED;
  // the tensor-core path reads A and Omega with TMA: 16-byte aligned rows
  if (path == 16 && ((A->ld % 8) != 0 || (reinterpret_cast<uintptr_t>(A->data) % 16) != 0))
    return ID_ERR_UNSUPPORTED;
  if (path == 16 && o->omega != nullptr &&
      ((o->ld_omega % 8) != 0 || (reinterpret_cast<uintptr_t>(o->omega) % 16) != 0))
    return ID_ERR_UNSUPPORTED;
  // FP8: block scales required; rows of A and Omega 16-byte aligned for TMA
  if (path == 8 && A->block_scale == nullptr) return kBadA;
  if (path == 8 && ((A->ld % 16) != 0 || (reinterpret_cast<uintptr_t>(A->data) % 16) != 0))
    return ID_ERR_UNSUPPORTED;
  if (path == 8 && o->omega != nullptr &&
      ((o->ld_omega % 16) != 0 || (reinterpret_cast<uintptr_t>(o->omega) % 16) != 0))
    return ID_ERR_UNSUPPORTED;
  const int64_t b = o->block == 0 ? 64 : o->block;
  if (b < 1 || b > kMaxBlock) return kBadOpts;
  if (!(o->tol >= 0.0) || o->k_max < 0 || o->k0 < 0 || o->blocks_per_pass < 0) return kBadOpts;
  if (o->x_solve_f64 < 0 || o->x_solve_f64 > 2) return kBadOpts;
  if (o->omega_kind != ID_OMEGA_GAUSSIAN && o->omega_kind != ID_OMEGA_SPARSE_SIGN) return kBadOpts;
  p->sparse = o->omega_kind == ID_OMEGA_SPARSE_SIGN && o->omega == nullptr;
  if (p->sparse) {
    // the gather-add sketch reads A in its own type: FP64, FP32 or BF16 input (on the
    // digit-sliced paths only their tensor-core Schur GEMM and block update remain)
    if (path == 8) return ID_ERR_UNSUPPORTED;
    const int64_t z = o->zeta == 0 ? 8 : o->zeta;
    if (z < 1 || z > b || b > kSparseMaxB) return kBadOpts;
    p->zeta = z;
  }
  p->m = A->m;
  p->n = A->n;
  p->b = b;
  p->sms = num_sms();
  p->esz = o->lu_prec == ID_F64 ? 8 : 4;
  p->path = path;
  p->ldw = path == 16 ? cdiv(A->m, 8) * 8 : (path == 65 ? f64emu_pad(A->m) : (path == 8 ? cdiv(A->m, 16) * 16 : A->m));
  p->wsz = path == 16 || path == 65 ? 2 : (path == 8 ? 1 : p->esz);
  p->gen_omega = (o->omega == nullptr);
  if (l > 0) {  // fixed rank; sizes do not depend on k (estimate block sized for k = 1)
    if (l > ((int64_t)1 << 20)) return kBadL;
    if (k < 1 || k > l || k > imin(A->m, A->n)) return kBadK;
    p->k = k;
    p->l = l;
    p->cap = k;
    p->rows_first = l;
    p->rows_pass = 0;
    p->wmax = imax(b, l);
    p->max_rounds = 2;
  } else {
    const int64_t kmax = o->k_max == 0 ? imin(A->m, A->n) : o->k_max;
    p->cap = imin(imin(A->m, A->n), kmax);
    const int64_t max_blocks = cdiv(p->cap, b) + 1;  // blocks that can ever be used
    int64_t first = o->k0 > 0 ? (cdiv(o->k0, b) + 1) : 1;
    p->rows_first = imin(first, max_blocks) * b;
    // 0 = automatic: two blocks per pass on the FP64-accurate tensor-core sketch (the
    // CTAs of a pass's two blocks read each tile of A's digits together, the second
    // from L2), eight on the BF16 and FP8 tensor-core sketches (a CTA runs the MMAs
    // of four 64-row blocks on each stage of A, and the two CTAs of a tile of A share
    // it through L2: A is read once per eight blocks), four on the FP32-accurate sketch
    // (its CTAs of a pass share each tile of A's digits through L2) and on the FP32
    // sparse-sign gather (its tiles of A staged once for four blocks' lists), one
    // elsewhere (the FP64 sparse gather's exact sums measured slower at two and four)
    const int64_t per = o->blocks_per_pass > 0
                            ? o->blocks_per_pass
                            : (p->sparse ? (sparse_kind(path) == 0 ? 4 : 1)
                                         : (path == 65 ? 2 : ((path == 16 || path == 8) ? 8 : (path == 33 ? 4 : 1))));
    p->rows_pass = imin(per, max_blocks) * b;
    p->wmax = b;
    p->max_rounds = max_blocks + 1;
    if (o->predictor != nullptr) {
      const int64_t cap_rows = o->max_pass_rows > 0 ? cdiv(o->max_pass_rows, b) * b : 16 * b;
      p->rows_pred = imin(cap_rows, max_blocks * b);
    }
  }
  if (!p->gen_omega) {
    if (o->ld_omega < A->m) return kBadOpts;
    const int64_t need = l > 0 ? l : (cdiv(p->cap, b) + 1) * b;
    if (o->omega_rows < need) return kBadOpts;
  }
  const int64_t rows_max = imax(imax(p->rows_first, p->rows_pass), p->rows_pred);
  if (p->sparse && cdiv(rows_max, b) > 65535) return ID_ERR_UNSUPPORTED;  // blocks of one sparse pass
  p->ldg = rows_max;
  // one split-K count for every pass (see Engine::splits_for): that of a pass of
  // one block (adaptive) or of the l rows (fixed rank)
  const int64_t unit = l > 0 ? l : b;
  const int s1 = p->sparse ? sparse_splits(p->m, p->n, p->sms, sparse_kind(path))
                 : path == 16 ? tc_sketch_effective_splits(p->m, tc_sketch_splits(p->m, p->n, unit, p->sms))
                 : path == 8  ? tc_fp8_effective_splits(p->m, tc_fp8_splits(p->m, p->n, unit, p->sms))
                 : path == 65 ? f64emu_splits(p->m, p->n, p->sms)
                 : path == 33 ? sketch_f32emu_splits(p->m, p->n, unit, p->sms)
                 : path == 32 ? gemm_splits((int)p->m, choose_splits_sgemm(p->n, unit, p->m, p->sms, 16, 2))
                              : gemm_splits((int)p->m, choose_splits_sgemm(p->n, unit, p->m, p->sms, 16, 1));
  p->s1_first = p->s1_pass = p->s1_cap = s1;
  // Schur split-K partials: FP32 products may split K 32 ways (late rounds: few rows of
  // S, thousands of earlier pivots); FP64 ones 8 (the FP64-accurate digit GEMM caps at 8)
  p->s2max = p->esz == 4 ? 32 : 8;
  p->nparts = 2 * p->sms;
  p->maxg = p->sms;
  const size_t e = p->esz;
  // regions that grow with the rank are sized for l >= k in fixed rank (the
  // workspace query plans with k = 1) and for the rank cap in adaptive runs
  const int64_t kcap = l > 0 ? l : p->cap;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + (bytes == 0 ? 1 : bytes));
    return at;
  };
  p->off_state = take(256);
  // path 65 keeps two digit planes of Omega, also for a caller Omega (rounded to its grid)
  // (sparse sign: the zeta codes of every column of the pass's blocks)
  p->off_omega = take(path == 65 ? 2 * (size_t)rows_max * p->ldw * p->wsz
                                 : (p->sparse ? sparse_csr_bytes(p->m, (int)cdiv(rows_max, b), (int)b, (int)p->zeta)
                                              : (p->gen_omega ? (size_t)rows_max * p->ldw * p->wsz : 0)));
  p->off_G = take((size_t)p->n * rows_max * e);
  // (the fixed-point sparse sketch of FP64 A keeps exact 128-bit split partials)
  const bool sfix_parts = p->sparse && (path == 64 || path == 65);
  p->off_Gpart = take(s1 > 1 ? (size_t)s1 * p->n * rows_max * (sfix_parts ? 16 : e) : 0);
  p->off_S = take((size_t)p->n * p->wmax * e);
  p->off_Spart = take((size_t)p->s2max * p->n * p->wmax * e);
  p->off_N = take((size_t)p->n * b * e);
  p->off_Linv = take((size_t)(cdiv(kcap, b) + 1) * b * b * e);  // every block's inverse diagonal block
  p->off_act0 = take((size_t)p->n * 4);
  p->off_act1 = take((size_t)p->n * 4);
  p->off_pivmark = take((size_t)p->n * 4);
  p->off_perm32 = take((size_t)p->n * 4);
  p->off_piv = take((size_t)kMaxBlock * 4);
  p->off_pivorig = take((size_t)kMaxBlock * 4);
  p->off_pivdiag = take((size_t)kMaxBlock * 8);
  p->off_cand_v = take((size_t)2 * p->maxg * 8);
  p->off_cand_i = take((size_t)2 * p->maxg * 4);
  p->off_cand_rows = take((size_t)2 * p->maxg * p->wmax * e);
  p->off_e2 = take((size_t)p->nparts * 8);
  p->off_normp = take((size_t)p->nparts * 8);
  p->off_trace = take((size_t)p->max_rounds * 8);
  // path 65: the 8 digit slices of A and its column exponents
  const bool sfix = p->sparse && (path == 64 || path == 65);
  p->off_sfix = take(sfix ? (size_t)p->m * p->n * 8 : 0);
  p->off_scol = take(sfix ? (size_t)p->n * 4 : 0);
  p->off_digits = take(path == 65 && !p->sparse ? f64emu_digit_bytes(p->m, p->n) : 0);
  p->off_colexp = take(path == 65 && !p->sparse ? (size_t)p->n * 4 : 0);
  // the Schur complement and the block update on the tensor cores: 7 digits for the
  // FP64-emulated path, 3 for every FP32 LU (panels and blocks of width <= 64)
  const bool emu7 = path == 65, emu3 = e == 4;
  p->update_tc = (emu7 || emu3) && b <= 64;
  const size_t udig = emu7 ? update_f64emu_digit_bytes(1) : update_f32emu_digit_bytes(1);
  p->off_ndig = take(p->update_tc ? udig * (size_t)p->n : 0);
  p->off_nexp = take(p->update_tc ? (size_t)p->n * 4 : 0);
  p->off_pdig = take(p->update_tc ? udig * (size_t)kcap : 0);
  p->off_pexp = take(p->update_tc ? (size_t)kcap * 4 : 0);
  // The Schur GEMM's K runs over every earlier pivot: per-row fixed point keeps the
  // FP64 accuracy with 7 digits, but with 3 it loses FP32's relative accuracy on
  // the small late pivot rows, so FP32 LUs keep the SIMT GEMM there.
  p->schur_tc = emu7;  // used for panels of width <= 64
  // path 33: digits of A (n rows of length m) and of each pass's Omega rows
  const bool slice32 = path == 33 && !p->sparse;
  p->off_f32a = take(slice32 ? sketch_f32emu_digit_bytes(p->n, p->m) : 0);
  p->off_f32ae = take(slice32 ? (size_t)p->n * 4 : 0);
  p->off_f32w = take(slice32 ? sketch_f32emu_digit_bytes(rows_max, p->m) : 0);
  p->off_f32we = take(slice32 ? (size_t)rows_max * 4 : 0);
  p->off_f32rmax = take(slice32 ? (size_t)rows_max * 8 : 0);
  p->off_adig = take(p->schur_tc ? gemm_f64emu_digit_bytes(p->n, kcap) : 0);
  p->off_aexp = take(p->schur_tc ? (size_t)p->n * 4 : 0);
  p->off_bdig = take(p->schur_tc ? gemm_f64emu_digit_bytes(64, kcap) : 0);
  p->off_bexp = take(p->schur_tc ? (size_t)64 * 4 : 0);
  p->off_colmax = take(p->schur_tc ? (size_t)64 * 8 : 0);
  // x_solve_f64: the multipliers (n x cap), column sums, and for an FP32 LU the FP64 solve's buffers
  p->keep_l = o->x_solve_f64 != 0;
  p->f64_solve = p->keep_l && e == 4;
  p->ldl = kcap;
  p->off_L = take(p->keep_l ? (size_t)p->n * kcap * e : 0);
  p->off_csum = take(p->keep_l ? (size_t)2 * kcap * 8 : 0);
  p->off_L1 = take(p->f64_solve ? (size_t)kcap * kcap * 8 : 0);
  p->off_T64 = take(p->f64_solve ? (size_t)p->n * kcap * 8 : 0);
  p->off_Linv64 = take(p->f64_solve ? (size_t)b * b * 8 : 0);
  p->off_iota = take(p->f64_solve ? (size_t)kcap * 4 : 0);
  p->total = off;
  return ID_OK;
}

#define RID_TRY(expr)             \
  do {                            \
    int rid_rc_ = (expr);         \
    if (rid_rc_ != 0) return rid_rc_; \
  } while (0)

// One call's state and the steps of the method.
template <typename T>
class Engine {
 public:
  Engine(const Plan& p, const id_matrix* A, const id_opts* o, void* ws, id_result* out, cudaStream_t s)
      : p_(p), o_(*o), out_(out), s_(s) {
    A_ = static_cast<const T*>(A->data);
    Araw_ = A->data;
    scale_ = A->block_scale;
    lda_ = A->ld;
    unsigned char* w = static_cast<unsigned char*>(ws);
    st_ = reinterpret_cast<DevState*>(w + p.off_state);
    omega_ = reinterpret_cast<T*>(w + p.off_omega);
    G_ = reinterpret_cast<T*>(w + p.off_G);
    Gpart_ = reinterpret_cast<T*>(w + p.off_Gpart);
    S_ = reinterpret_cast<T*>(w + p.off_S);
    Spart_ = reinterpret_cast<T*>(w + p.off_Spart);
    N_ = reinterpret_cast<T*>(w + p.off_N);
    Linv_ = reinterpret_cast<T*>(w + p.off_Linv);
    act_[0] = reinterpret_cast<int32_t*>(w + p.off_act0);
    act_[1] = reinterpret_cast<int32_t*>(w + p.off_act1);
    pivmark_ = reinterpret_cast<int32_t*>(w + p.off_pivmark);
    perm32_ = reinterpret_cast<int32_t*>(w + p.off_perm32);
    piv_ = reinterpret_cast<int32_t*>(w + p.off_piv);
    pivorig_ = reinterpret_cast<int32_t*>(w + p.off_pivorig);
    pivdiag_ = reinterpret_cast<double*>(w + p.off_pivdiag);
    cand_v_ = reinterpret_cast<double*>(w + p.off_cand_v);
    cand_i_ = reinterpret_cast<int32_t*>(w + p.off_cand_i);
    cand_rows_ = reinterpret_cast<T*>(w + p.off_cand_rows);
    e2_ = reinterpret_cast<double*>(w + p.off_e2);
    normp_ = reinterpret_cast<double*>(w + p.off_normp);
    trace_ = reinterpret_cast<double*>(w + p.off_trace);
    digits_ = w + p.off_digits;
    colexp_ = reinterpret_cast<int32_t*>(w + p.off_colexp);
    L_ = p.keep_l ? reinterpret_cast<T*>(w + p.off_L) : nullptr;
    csum_ = reinterpret_cast<double*>(w + p.off_csum);
    L1_64_ = reinterpret_cast<double*>(w + p.off_L1);
    T64_ = reinterpret_cast<double*>(w + p.off_T64);
    Linv64_ = reinterpret_cast<double*>(w + p.off_Linv64);
    iota_ = reinterpret_cast<int32_t*>(w + p.off_iota);
    ndig_ = w + p.off_ndig;
    nexp_ = reinterpret_cast<int32_t*>(w + p.off_nexp);
    pdig_ = w + p.off_pdig;
    pexp_ = reinterpret_cast<int32_t*>(w + p.off_pexp);
    adig_ = w + p.off_adig;
    aexp_ = reinterpret_cast<int32_t*>(w + p.off_aexp);
    bdig_ = w + p.off_bdig;
    bexp_ = reinterpret_cast<int32_t*>(w + p.off_bexp);
    colmax_ = reinterpret_cast<unsigned long long*>(w + p.off_colmax);
    f32a_ = w + p.off_f32a;
    f32ae_ = reinterpret_cast<int32_t*>(w + p.off_f32ae);
    f32w_ = w + p.off_f32w;
    f32we_ = reinterpret_cast<int32_t*>(w + p.off_f32we);
    f32rmax_ = reinterpret_cast<unsigned long long*>(w + p.off_f32rmax);
    sfix_ = reinterpret_cast<long long*>(w + p.off_sfix);
    sfix_col_ = reinterpret_cast<int32_t*>(w + p.off_scol);
    X_ = static_cast<T*>(out->X);
    ldx_ = out->ldx;
    done_ = &st_->done;
    for (int i = 0; i < kNumPhases; ++i) {
      phase_ms_[i] = 0.0;
      phase_launches_[i] = 0;
    }
  }
  ~Engine() {
    for (cudaEvent_t e : events_) cudaEventDestroy(e);
  }

  int run_adaptive() {
    RID_TRY(start());
    int64_t tb = 0, na = p_.n, t = 0, sketched = 0, gstart = 0;
    const int64_t b = p_.b;
    bool full = false;
    for (;;) {
      if (t >= sketched) {
        const int64_t max_blocks = cdiv(p_.cap, b) + 1;
        int64_t rows = t == 0 ? p_.rows_first : p_.rows_pass;
        if (t > 0 && pred_blocks_ > t)  // blocks t .. pred_blocks_ certify the predicted rank
          rows = imax(rows, imin((pred_blocks_ - t + 1) * b, p_.rows_pred));
        rows = imin(rows, (max_blocks - t) * b);
        RID_TRY(sketch(t * b, rows, splits_for(rows)));
        gstart = t;
        sketched = t + rows / b;
      }
      RID_TRY(schur((t - gstart) * b, b, tb, na));
      if (t > 0) {
        RID_TRY(decide(b, tb, tb == p_.cap, (int)(t - 1)));
        RID_TRY(sync_state());
        if (h_.err) break;
        if (h_.done) break;
      }
      const int64_t bt = imin(b, p_.cap - tb);
      RID_TRY(factor(b, bt, tb, na));
      if (t == 0 && o_.predictor != nullptr) {
        // learned rank guess from the first block's pivots: it only sets how many
        // blocks the next pass over A sketches
        RID_TRY(tbegin(ID_PHASE_OTHER));
        RID_TRY(cuda(mlp_predict_rank(o_.predictor, pivdiag_, (int)imin(bt, 32), p_.m, p_.n, o_.tol,
                                      o_.tol_relative, st_, s_)));
        RID_TRY(tend(1));
        RID_TRY(sync_state());
        pred_blocks_ = imin(cdiv(imax(h_.k_pred, 1), b), cdiv(p_.cap, b));
        predicted_ = h_.k_pred;
      }
      tb += bt;
      na -= bt;
      ++t;
      if (tb == p_.n) {  // every column is a skeleton: X is a permutation, the residual is 0
        full = true;
        break;
      }
    }
    const int64_t k = full ? p_.n : (h_.done ? h_.k_final : tb);
    est_zero_ = full;  // k = n: no columns left, the ID is exact
    return finish(k);
  }

  int run_fixed() {
    RID_TRY(start());
    RID_TRY(sketch(0, p_.l, splits_for(p_.l)));
    int64_t tb = 0, na = p_.n;
    while (tb < p_.k) {
      const int64_t w = imin(p_.b, p_.k - tb);
      RID_TRY(schur(tb, w, tb, na));
      RID_TRY(factor(w, w, tb, na));
      tb += w;
      na -= w;
    }
    if (p_.l > p_.k && p_.n > p_.k) {
      RID_TRY(schur(p_.k, p_.l - p_.k, tb, na));
      RID_TRY(decide(p_.l - p_.k, tb, 0, 0));
    }
    est_zero_ = !(p_.l > p_.k && p_.n > p_.k);  // no estimation rows: report 0
    return finish(p_.k);
  }

  // Remark 1 (Sec. 3.2): the rank-k fixed-rank ID from l = k + p sketch rows, then
  // the LUPP of the p extra rows' Schur complement S ((n-k) x p) continued for p
  // steps.  S = L_r U_r; U_r is read from the pivot rows, and the columns of the
  // extra pivots (the skeleton's continuation) go to Jx.
  int run_ur(int64_t p, T* U, int64_t ldu, int64_t* Jx, double* stats) {
    const int status = run_fixed();
    if (status < 0) return status;
    const int64_t na = p_.n - p_.k;
    RID_TRY(tbegin(ID_PHASE_LU));
    // the fixed-rank estimate set the stop flag; the extra steps must run
    RID_TRY(cuda(cudaMemsetAsync(&st_->done, 0, sizeof(int32_t), s_)));
    PanelCfg cfg = panel_config<T>((int)na, (int)p, p_.maxg);
    RID_TRY(cuda(panel_lupp<T>(cfg, (int)na, (int)p, (int)p, panel_par_, S_, p_.wmax, piv_, pivmark_, pivdiag_,
                               cand_v_, cand_i_, cand_rows_, st_, s_)));
    panel_par_ ^= 1;
    RID_TRY(cuda(ur_extract<T>((int)p, (int)na, S_, p_.wmax, piv_, act_[cur_], U, ldu, Jx, e2_, s_)));
    RID_TRY(tend(2));
    RID_TRY(cuda(cudaMemcpyAsync(stats, e2_, 2 * sizeof(double), cudaMemcpyDeviceToHost, s_)));
    RID_TRY(sync_state());
    if (h_.err & kErrTimeout) return ID_ERR_TIMEOUT;
    out_->launches = launches_;
    return status;
  }

  // LUPP of a given panel instead of a sketch: G (p_.n rows x p_.k columns) is
  // gathered from the columns J of `src` (m_src x n_src, ld_src), its rows are
  // pivoted for k steps, and the interpolation coefficients land in the X buffer.
  int run_panel(const T* src, int64_t m_src, int64_t n_src, int64_t ld_src, const int64_t* J) {
    RID_TRY(tbegin(ID_PHASE_OTHER));
    RID_TRY(cuda(init_state(st_, act_[0], pivmark_, p_.n, s_)));
    panel_par_ = 0;  // both barrier counters were cleared
    RID_TRY(cuda(gather_panel<T>(src, ld_src, m_src, n_src, J, p_.k, G_, st_, s_)));
    RID_TRY(tend(2));
    int64_t tb = 0, na = p_.n;
    while (tb < p_.k) {
      const int64_t w = imin(p_.b, p_.k - tb);
      RID_TRY(schur(tb, w, tb, na));
      RID_TRY(factor(w, w, tb, na));
      tb += w;
      na -= w;
    }
    est_zero_ = true;
    RID_TRY(sync_state());
    if (h_.err & kErrBadIndex) return -2;
    return finish(p_.k);
  }

 private:
  int cuda(cudaError_t e) { return e == cudaSuccess ? 0 : ID_ERR_CUDA; }

  // ---- phase timing (CUDA events on the launching stream) and launch counts
  int tbegin(int ph) {
    cur_phase_ = ph;
    if (!o_.profile) return 0;
    cudaEvent_t e;
    RID_TRY(cuda(cudaEventCreate(&e)));
    events_.push_back(e);
    RID_TRY(cuda(cudaEventRecord(e, s_)));
    return 0;
  }
  int tend(int launches) {
    launches_ += launches;
    phase_launches_[cur_phase_] += launches;
    if (!o_.profile) return 0;
    cudaEvent_t e;
    RID_TRY(cuda(cudaEventCreate(&e)));
    events_.push_back(e);
    RID_TRY(cuda(cudaEventRecord(e, s_)));
    pending_.push_back(cur_phase_);
    return 0;
  }
  void collect_times() {
    for (size_t i = 0; i < pending_.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, events_[2 * i], events_[2 * i + 1]) == cudaSuccess)
        phase_ms_[pending_[i]] += ms;
    }
    for (cudaEvent_t e : events_) cudaEventDestroy(e);
    events_.clear();
    pending_.clear();
  }

  int start() {
    RID_TRY(tbegin(ID_PHASE_OTHER));
    RID_TRY(cuda(init_state(st_, act_[0], pivmark_, p_.n, s_)));
    panel_par_ = 0;  // both barrier counters were cleared
    if (p_.path == 8)
      RID_TRY(cuda(norm2_fp8(p_.m, p_.n, Araw_, lda_, scale_, normp_, p_.nparts, st_, s_)));
    else if (p_.path == 16)
      RID_TRY(cuda(norm2_partial<__nv_bfloat16>(p_.m, p_.n, static_cast<const __nv_bfloat16*>(Araw_), lda_, normp_,
                                                p_.nparts, st_, s_)));
    else
      RID_TRY(cuda(norm2_partial<T>(p_.m, p_.n, A_, lda_, normp_, p_.nparts, st_, s_)));
    RID_TRY(cuda(norm2_final(normp_, p_.nparts, st_, s_)));
    RID_TRY(tend(3));
    RID_TRY(sync_state());
    if (h_.err & kErrNonFinite) return ID_ERR_NONFINITE;
    if (p_.path == 33 && !p_.sparse) {  // digits of A's columns, once per call
      RID_TRY(tbegin(ID_PHASE_SKETCH));
      RID_TRY(cuda(sketch_f32emu_slice((int)p_.n, (int)p_.m, reinterpret_cast<const float*>(Araw_), lda_, f32a_, p_.n,
                                       f32ae_, nullptr, nullptr, s_)));
      RID_TRY(tend(1));
    }
    if (p_.sparse && sizeof(T) == 8) {  // FP64 A in 64-bit fixed point, once per call
      RID_TRY(tbegin(ID_PHASE_SKETCH));
      RID_TRY(cuda(sparse_fixed_prepare(reinterpret_cast<const double*>(Araw_), lda_, p_.m, p_.n, sfix_col_,
                                        sfix_, s_)));
      RID_TRY(tend(2));
    }
    if (p_.path == 65 && !p_.sparse) {  // column exponents and digit slices of A, once per call
      RID_TRY(tbegin(ID_PHASE_SKETCH));
      RID_TRY(cuda(f64emu_prepare(reinterpret_cast<const double*>(Araw_), lda_, p_.m, p_.n, colexp_, digits_, s_)));
      RID_TRY(tend(2));
    }
    return 0;
  }

  int sync_state() {
    RID_TRY(cuda(cudaMemcpyAsync(&h_, st_, sizeof(DevState), cudaMemcpyDeviceToHost, s_)));
    RID_TRY(cuda(cudaStreamSynchronize(s_)));
    collect_times();
    return 0;
  }

  // G(:, 0:rows) = (Omega rows [row0, row0+rows)) A, stored n x rows (row-major, ld ldg).
  // Split-K count of every sketch pass.  It depends on the problem and the block
  // size only -- never on how many blocks a pass draws -- so each entry of the
  // sketch is summed in the same order whatever the pass size, and a rank guess
  // (k0, blocks_per_pass, the learned predictor) leaves J, X and k bit-identical.
  int splits_for(int64_t /*rows*/) {
    const int64_t unit = p_.l > 0 ? p_.l : p_.b;
    if (p_.sparse) return sparse_splits(p_.m, p_.n, p_.sms, sparse_kind(p_.path));
    if (p_.path == 16) return tc_sketch_effective_splits(p_.m, tc_sketch_splits(p_.m, p_.n, unit, p_.sms));
    if (p_.path == 8) return tc_fp8_effective_splits(p_.m, tc_fp8_splits(p_.m, p_.n, unit, p_.sms));
    if (p_.path == 65) return f64emu_splits(p_.m, p_.n, p_.sms);
    if (p_.path == 33) return sketch_f32emu_splits(p_.m, p_.n, unit, p_.sms);
    if (p_.path == 32) return gemm_splits((int)p_.m, choose_splits_sgemm(p_.n, unit, p_.m, p_.sms, 16, 2));
    return gemm_splits((int)p_.m, choose_splits_sgemm(p_.n, unit, p_.m, p_.sms, 16, 1));
  }

  int sketch(int64_t row0, int64_t rows, int splits) {
    if (p_.sparse) return sketch_sparse(row0, rows, splits);
    if (p_.path == 16) return sketch_tc(row0, rows, splits);
    if (p_.path == 8) return sketch_fp8(row0, rows, splits);
    if (p_.path == 65) return sketch_emu(row0, rows, splits);
    if (p_.path == 33) return sketch_f32emu_pass(row0, rows, splits);
    const T* Om;
    int64_t ldo;
    if (p_.gen_omega) {
      RID_TRY(tbegin(ID_PHASE_OMEGA));
      RID_TRY(cuda(gaussian_rows<T>(o_.seed, row0, rows, p_.m, omega_, p_.m, done_, s_)));
      RID_TRY(tend(1));
      Om = omega_;
      ldo = p_.m;
    } else {
      Om = static_cast<const T*>(o_.omega) + row0 * o_.ld_omega;
      ldo = o_.ld_omega;
    }
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    Operand<T> a{A_, lda_, nullptr, 0};
    Operand<T> bop{Om, ldo, nullptr, 0};
    EpiArgs<T> ep{splits > 1 ? Gpart_ : G_, p_.ldg, (int64_t)p_.n * p_.ldg, nullptr, nullptr};
    splits = gemm_splits((int)p_.m, splits);
    ep.out = splits > 1 ? Gpart_ : G_;
    RID_TRY(cuda(gemm_gather<T>((int)p_.n, (int)rows, (int)p_.m, splits, true, a, bop, kEpiStore, ep, done_, s_)));
    if (splits > 1)
      RID_TRY(cuda(splitk_reduce<T>(p_.n, (int)rows, p_.ldg, splits, (int64_t)p_.n * p_.ldg, Gpart_, G_, done_, s_)));
    RID_TRY(tend(splits > 1 ? 2 : 1));
    ++passes_;
    return 0;
  }

  // Sparse-sign rows [row0, row0+rows) (Sec. 5.1): the lists of the pass's blocks
  // per 128-row tile of A, then the gather-add G = Omega A (FP32 sums for FP32 and
  // BF16 A, exact integer sums of the fixed-point copy of FP64 A).
  int sketch_sparse(int64_t row0, int64_t rows, int splits) {
    const int64_t b = p_.b;
    uint16_t* R = reinterpret_cast<uint16_t*>(omega_);
    RID_TRY(tbegin(ID_PHASE_OMEGA));
    const int esz = p_.path == 16 ? 2 : (int)sizeof(T);  // staged bytes: BF16, FP32 or the FP64 fixed point
    RID_TRY(cuda(sparse_csr(o_.seed, row0 / b, (int)cdiv(rows, b), (int)b, p_.m, (int)p_.zeta, esz, R, done_, s_)));
    RID_TRY(tend(1));
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    const int64_t zs = (int64_t)p_.n * p_.ldg;
    if constexpr (std::is_same<T, float>::value) {
      T* out = splits > 1 ? Gpart_ : G_;
      if (p_.path == 16)
        RID_TRY(cuda(sparse_sketch<__nv_bfloat16>(p_.m, p_.n, static_cast<const __nv_bfloat16*>(Araw_), lda_, R,
                                                  (int)p_.zeta, (int)b, rows, splits, out, p_.ldg, zs, done_, s_)));
      else
        RID_TRY(cuda(sparse_sketch<float>(p_.m, p_.n, A_, lda_, R, (int)p_.zeta, (int)b, rows, splits, out, p_.ldg, zs,
                                          done_, s_)));
      if (splits > 1) RID_TRY(cuda(splitk_reduce<T>(p_.n, (int)rows, p_.ldg, splits, zs, Gpart_, G_, done_, s_)));
    } else {  // exact integer sums of the fixed-point copy (128-bit split partials)
      RID_TRY(cuda(sparse_sketch_fixed(p_.m, p_.n, sfix_, sfix_col_, R, (int)p_.zeta, (int)b, rows, splits, G_, p_.ldg,
                                       Gpart_, p_.ldg, zs, done_, s_)));
    }
    RID_TRY(tend(splits > 1 ? 2 : 1));
    ++passes_;
    return 0;
  }

  // BF16 operands on the tensor cores: G = (Omega rows [row0, row0+rows)) A in FP32.
  int sketch_tc(int64_t row0, int64_t rows, int splits) {
    const void* W;
    int64_t ldw;
    if (p_.gen_omega) {
      RID_TRY(tbegin(ID_PHASE_OMEGA));
      RID_TRY(cuda(gaussian_rows<__nv_bfloat16>(o_.seed, row0, rows, p_.m, reinterpret_cast<__nv_bfloat16*>(omega_),
                                                p_.ldw, done_, s_)));
      RID_TRY(tend(1));
      W = omega_;
      ldw = p_.ldw;
    } else {
      W = static_cast<const __nv_bfloat16*>(o_.omega) + row0 * o_.ld_omega;
      ldw = o_.ld_omega;
    }
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    float* out = reinterpret_cast<float*>(splits > 1 ? Gpart_ : G_);
    RID_TRY(cuda(tc_sketch_bf16(Araw_, lda_, p_.m, p_.n, W, ldw, rows, out, p_.ldg, (int64_t)p_.n * p_.ldg, splits,
                                st_, done_, s_)));
    if (splits > 1)
      RID_TRY(cuda(splitk_reduce<float>(p_.n, (int)rows, p_.ldg, splits, (int64_t)p_.n * p_.ldg,
                                        reinterpret_cast<const float*>(Gpart_), reinterpret_cast<float*>(G_), done_,
                                        s_)));
    RID_TRY(tend(splits > 1 ? 2 : 1));
    ++passes_;
    return 0;
  }

  // FP8 operands on the tensor cores: G = (Omega rows [row0, row0+rows)) A in FP32,
  // A's block scales applied per 128-row block.
  int sketch_fp8(int64_t row0, int64_t rows, int splits) {
    const void* W;
    int64_t ldw;
    if (p_.gen_omega) {
      RID_TRY(tbegin(ID_PHASE_OMEGA));
      RID_TRY(cuda(gaussian_rows<__nv_fp8_e4m3>(o_.seed, row0, rows, p_.m, reinterpret_cast<__nv_fp8_e4m3*>(omega_),
                                                p_.ldw, done_, s_)));
      RID_TRY(tend(1));
      W = omega_;
      ldw = p_.ldw;
    } else {
      W = static_cast<const uint8_t*>(o_.omega) + row0 * o_.ld_omega;
      ldw = o_.ld_omega;
    }
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    float* out = reinterpret_cast<float*>(splits > 1 ? Gpart_ : G_);
    RID_TRY(cuda(tc_sketch_fp8(Araw_, lda_, p_.m, p_.n, scale_, W, ldw, rows, out, p_.ldg, (int64_t)p_.n * p_.ldg,
                               splits, st_, done_, s_)));
    if (splits > 1)
      RID_TRY(cuda(splitk_reduce<float>(p_.n, (int)rows, p_.ldg, splits, (int64_t)p_.n * p_.ldg,
                                        reinterpret_cast<const float*>(Gpart_), reinterpret_cast<float*>(G_), done_,
                                        s_)));
    RID_TRY(tend(splits > 1 ? 2 : 1));
    ++passes_;
    return 0;
  }

  // FP32 A on the tensor cores: the pass's Omega rows (FP32 Gaussian) sliced into 3
  // digits, then G = Omega A from the digits of A and Omega.
  int sketch_f32emu_pass(int64_t row0, int64_t rows, int splits) {
    const float* Om;
    int64_t ldo;
    if (p_.gen_omega) {
      RID_TRY(tbegin(ID_PHASE_OMEGA));
      RID_TRY(cuda(gaussian_rows<float>(o_.seed, row0, rows, p_.m, reinterpret_cast<float*>(omega_), p_.m, done_, s_)));
      RID_TRY(tend(1));
      Om = reinterpret_cast<const float*>(omega_);
      ldo = p_.m;
    } else {
      Om = static_cast<const float*>(o_.omega) + row0 * o_.ld_omega;
      ldo = o_.ld_omega;
    }
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    RID_TRY(cuda(sketch_f32emu_slice((int)rows, (int)p_.m, Om, ldo, f32w_, p_.ldg, f32we_, f32rmax_, done_, s_)));
    float* out = reinterpret_cast<float*>(splits > 1 ? Gpart_ : G_);
    RID_TRY(cuda(sketch_f32emu(p_.m, p_.n, rows, f32a_, f32ae_, f32w_, p_.ldg, f32we_, out, p_.ldg,
                               (int64_t)p_.n * p_.ldg, splits, st_, done_, s_)));
    if (splits > 1)
      RID_TRY(cuda(splitk_reduce<float>(p_.n, (int)rows, p_.ldg, splits, (int64_t)p_.n * p_.ldg,
                                        reinterpret_cast<const float*>(Gpart_), reinterpret_cast<float*>(G_), done_,
                                        s_)));
    RID_TRY(tend(splits > 1 ? 3 : 2));
    ++passes_;
    return 0;
  }

  // FP64 A on the tensor cores: Omega rows [row0, row0+rows) on the grid 2^-11 as
  // two digit planes, then G = Omega A from the digit slices of A (FP64 accurate).
  int sketch_emu(int64_t row0, int64_t rows, int splits) {
    RID_TRY(tbegin(ID_PHASE_OMEGA));
    const double* src = p_.gen_omega ? nullptr : static_cast<const double*>(o_.omega) + row0 * o_.ld_omega;
    RID_TRY(cuda(f64emu_omega(o_.seed, row0, rows, p_.m, p_.ldg, src, o_.ld_omega, omega_, done_, s_)));
    RID_TRY(tend(1));
    RID_TRY(tbegin(ID_PHASE_SKETCH));
    double* out = reinterpret_cast<double*>(splits > 1 ? Gpart_ : G_);
    RID_TRY(cuda(f64emu_sketch(digits_, colexp_, p_.m, p_.n, omega_, rows, p_.ldg, out, p_.ldg,
                               (int64_t)p_.n * p_.ldg, splits, st_, done_, s_)));
    if (splits > 1)
      RID_TRY(cuda(splitk_reduce<double>(p_.n, (int)rows, p_.ldg, splits, (int64_t)p_.n * p_.ldg,
                                         reinterpret_cast<const double*>(Gpart_), reinterpret_cast<double*>(G_),
                                         done_, s_)));
    RID_TRY(tend(splits > 1 ? 2 : 1));
    ++passes_;
    return 0;
  }

  // S = G(act, col0:col0+w) - T(act, 0:tb) G(perm, col0:col0+w) and ||S||^2 partials.
  int schur(int64_t col0, int64_t w, int64_t tb, int64_t na) {
    RID_TRY(tbegin(ID_PHASE_SCHUR));
    int nz = 0, nl = 0;
    const int64_t lds = p_.wmax;
    if (tb > 0) {
      bool done_tc = false;
      if constexpr (std::is_same<T, double>::value) {
        if (p_.schur_tc && w <= 64) {  // FP64-accurate on the tensor cores
          nz = gemm_f64emu_splits(na, w, tb, p_.sms);
          RID_TRY(cuda(gemm_f64emu((int)na, (int)w, (int)tb, X_, ldx_, act_[cur_], G_, p_.ldg, col0, perm32_, adig_,
                                   p_.n, aexp_, bdig_, 64, bexp_, colmax_, p_.ldl, Spart_, lds, (int64_t)p_.n * lds,
                                   nz, st_, done_, s_)));
          nl += 4;
          done_tc = true;
        }
      }
      if (!done_tc) {
        // FP64 Schur products run on the 64 x 64 kernel: about four blocks per SM
        nz = gemm_splits((int)tb, sizeof(T) == 4 ? choose_splits_sgemm(na, w, tb, p_.sms, p_.s2max, 2)
                                                 : choose_splits_gather(na, w, tb, p_.sms, p_.s2max));
        Operand<T> a{X_, ldx_, act_[cur_], 0};
        Operand<T> bop{G_, p_.ldg, perm32_, col0};
        EpiArgs<T> ep{Spart_, lds, (int64_t)p_.n * lds, nullptr, nullptr};
        RID_TRY(cuda(gemm_gather<T>((int)na, (int)w, (int)tb, nz, false, a, bop, kEpiStore, ep, done_, s_)));
        ++nl;
      }
    }
    RID_TRY(cuda(schur_finish<T>((int)na, (int)w, act_[cur_], G_, p_.ldg, col0, nz, (int64_t)p_.n * lds, Spart_,
                                 S_, lds, e2_, p_.nparts, done_, s_)));
    RID_TRY(tend(nl + 1));
    return 0;
  }

  int decide(int64_t w, int64_t tb, int last, int round) {
    RID_TRY(tbegin(ID_PHASE_OTHER));
    const double tol = p_.l > 0 ? INFINITY : o_.tol;  // fixed rank: estimate only
    RID_TRY(cuda(rid::decide(e2_, p_.nparts, (int)w, tol, p_.l > 0 ? 0 : o_.tol_relative, tb, last, trace_,
                             round, st_, s_)));
    RID_TRY(tend(1));
    return 0;
  }

  // LUPP of S (na x w) for bt pivots, then re-blocking.
  int factor(int64_t w, int64_t bt, int64_t tb, int64_t na) {
    const int64_t lds = p_.wmax;
    RID_TRY(tbegin(ID_PHASE_LU));
    PanelCfg cfg = panel_config<T>((int)na, (int)w, p_.maxg);
    RID_TRY(cuda(panel_lupp<T>(cfg, (int)na, (int)w, (int)bt, panel_par_, S_, lds, piv_, pivmark_, pivdiag_,
                               cand_v_, cand_i_, cand_rows_, st_, s_)));
    panel_par_ ^= 1;
    RID_TRY(tend(1));
    RID_TRY(tbegin(ID_PHASE_UPDATE));
    int nl = 3;
    T* Linv_t = Linv_ + (tb / p_.b) * p_.b * p_.b;  // kept per block for the condition of L1
    RID_TRY(cuda(linv<T>((int)bt, S_, lds, piv_, Linv_t, done_, s_)));
    if (L_ != nullptr) {
      RID_TRY(cuda(store_l<T>((int)na, (int)bt, S_, lds, piv_, pivmark_, act_[cur_], L_, p_.ldl, tb, done_, s_)));
      ++nl;
    }
    RID_TRY(cuda(make_n<T>((int)na, (int)bt, S_, lds, Linv_t, pivmark_, act_[cur_], N_, X_, ldx_, tb, piv_,
                           pivorig_, done_, s_)));
    if (tb > 0) {
      bool done_tc = false;
      if (p_.update_tc) {  // FP64- or FP32-accurate on the tensor cores
        if constexpr (std::is_same<T, double>::value)
          RID_TRY(cuda(update_f64emu((int)na, (int)bt, (int)tb, N_, act_[cur_], pivmark_, pivorig_, X_, ldx_, ndig_,
                                     nexp_, p_.n, pdig_, pexp_, p_.ldl, p_.sms, st_, done_, s_)));
        else
          RID_TRY(cuda(update_f32emu((int)na, (int)bt, (int)tb, N_, act_[cur_], pivmark_, pivorig_, X_, ldx_, ndig_,
                                     nexp_, p_.n, pdig_, pexp_, p_.ldl, p_.sms, st_, done_, s_)));
        nl += 3;
        done_tc = true;
      }
      if (!done_tc) {
        Operand<T> a{N_, bt, nullptr, 0};
        Operand<T> bop{X_, ldx_, pivorig_, 0};
        EpiArgs<T> ep{X_, ldx_, 0, act_[cur_], pivmark_};
        RID_TRY(cuda(gemm_gather<T>((int)na, (int)tb, (int)bt, 1, false, a, bop, kEpiSubRows, ep, done_, s_)));
        ++nl;
      }
    }
    RID_TRY(cuda(compact((int)na, (int)bt, act_[cur_], act_[cur_ ^ 1], pivmark_, piv_, out_->J, perm32_, tb,
                         out_->pivots, pivdiag_, done_, s_)));
    RID_TRY(tend(nl));
    cur_ ^= 1;
    return 0;
  }

  // kappa_1(L1) from the column sums; an FP64 re-solve of X when it is large (FP32 LU).
  int condition_and_solve(int64_t k) {
    RID_TRY(tbegin(ID_PHASE_OTHER));
    RID_TRY(cuda(cond_colsums<T>(k, (int)p_.b, perm32_, L_, p_.ldl, X_, ldx_, Linv_, csum_, csum_ + p_.ldl, s_)));
    RID_TRY(tend(2));
    std::vector<double> h((size_t)2 * k);
    RID_TRY(cuda(cudaMemcpyAsync(h.data(), csum_, k * sizeof(double), cudaMemcpyDeviceToHost, s_)));
    RID_TRY(cuda(cudaMemcpyAsync(h.data() + k, csum_ + p_.ldl, k * sizeof(double), cudaMemcpyDeviceToHost, s_)));
    RID_TRY(sync_state());
    double n1 = 0.0, ninv = 0.0;
    for (int64_t c = 0; c < k; ++c) {
      n1 = fmax(n1, h[c]);
      ninv = fmax(ninv, h[k + c]);
    }
    cond_ = n1 * ninv;
    const int64_t na = p_.n - k;
    if (p_.f64_solve && na > 0 && (o_.x_solve_f64 == 2 || !(cond_ <= ID_COND_SWITCH))) {
      RID_TRY(tbegin(ID_PHASE_OTHER));
      int nl = 0;
      RID_TRY(cuda(resolve_x_f64<T>(k, (int)p_.b, na, perm32_, act_[cur_], L_, p_.ldl, L1_64_, T64_, Linv64_, iota_,
                                    X_, ldx_, s_, &nl)));
      RID_TRY(tend(nl));
      x_f64_ = 1;
    }
    return 0;
  }

  int finish(int64_t k) {
    if (o_.x_solve_f64 != 0 && k > 0) RID_TRY(condition_and_solve(k));
    RID_TRY(tbegin(ID_PHASE_OTHER));
    RID_TRY(cuda(finalize_x<T>(k, perm32_, X_, ldx_, s_)));
    RID_TRY(tend(1));
    RID_TRY(sync_state());
    int status = ID_OK;
    if (h_.err & kErrTimeout) return ID_ERR_TIMEOUT;
    if (h_.err & kErrNonFinite) return ID_ERR_NONFINITE;
    if (h_.tol_not_met) status |= ID_WARN_TOL_NOT_MET;
    if (h_.zero_pivots) status |= ID_WARN_ZERO_PIVOT;
    out_->status = status;
    out_->k = k;
    out_->est_err = est_zero_ ? 0.0 : h_.est;
    out_->norm_A = sqrt(h_.norm2_A);
    out_->rounds = h_.rounds;
    out_->passes = passes_;
    out_->launches = launches_;
    out_->cond_L1 = cond_;
    out_->x_f64 = x_f64_;
    for (int i = 0; i < kNumPhases; ++i) {
      out_->phase_ms[i] = phase_ms_[i];
      out_->phase_launches[i] = phase_launches_[i];
    }
    if (out_->est_trace != nullptr && out_->trace_cap > 0 && h_.rounds > 0) {
      const int64_t nt = imin(out_->trace_cap, h_.rounds);
      RID_TRY(cuda(cudaMemcpyAsync(out_->est_trace, trace_, nt * sizeof(double), cudaMemcpyDeviceToHost, s_)));
      RID_TRY(cuda(cudaStreamSynchronize(s_)));
    }
    return status;
  }

  Plan p_;
  id_opts o_;
  id_result* out_;
  cudaStream_t s_;
  const T* A_;
  const void* Araw_;
  const float* scale_;  // FP8 block scales
  int64_t lda_;
  DevState* st_;
  DevState h_{};
  T *omega_, *G_, *Gpart_, *S_, *Spart_, *N_, *Linv_, *cand_rows_, *X_;
  int32_t *act_[2], *pivmark_, *perm32_, *piv_, *pivorig_, *cand_i_;
  double *pivdiag_, *cand_v_, *e2_, *normp_, *trace_;
  void* digits_;       // path 65: digit slices of A
  int32_t* colexp_;    // path 65: column exponents of A
  T* L_;               // x_solve_f64: LUPP multipliers by original row (null otherwise)
  double *csum_, *L1_64_, *T64_, *Linv64_;
  int32_t* iota_;
  void *ndig_, *pdig_;   // path 65: digit slices for the tensor-core block update
  int32_t *nexp_, *pexp_;
  void *adig_, *bdig_;   // path 65: digit slices for the tensor-core Schur GEMM
  int32_t *aexp_, *bexp_;
  unsigned long long* colmax_;
  void *f32a_, *f32w_;  // path 33: digits of A and of the pass's Omega rows
  int32_t *f32ae_, *f32we_;
  unsigned long long* f32rmax_;
  long long* sfix_;      // sparse sign with FP64 A: the fixed-point copy of A and its column exponents
  int32_t* sfix_col_;
  const int32_t* done_;
  int64_t ldx_;
  int cur_ = 0;
  int cur_phase_ = 0;
  bool est_zero_ = false;
  int64_t pred_blocks_ = 0;  // blocks certifying the predicted rank (0: no predictor)
  double cond_ = 0.0;        // kappa_1(L1) when requested
  int32_t x_f64_ = 0;
  int64_t predicted_ = 0;
  int32_t passes_ = 0;
  int panel_par_ = 0;  // barrier counter of the next panel launch (alternates)
  int64_t launches_ = 0;
  double phase_ms_[kNumPhases];
  int64_t phase_launches_[kNumPhases];
  std::vector<cudaEvent_t> events_;
  std::vector<int> pending_;
};

int check_ws(const Plan& p, void* ws, size_t ws_bytes) {
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 || ws_bytes < p.total)
    return ID_ERR_WORKSPACE;
  return ID_OK;
}

int check_out(const Plan& p, const id_result* out) {
  if (out == nullptr || out->J == nullptr || out->X == nullptr || out->ldx < p.cap) return -1;
  return ID_OK;
}

void clear_out(id_result* out) {
  out->status = ID_OK;
  out->k = 0;
  out->est_err = 0.0;
  out->norm_A = 0.0;
  out->rounds = 0;
  out->passes = 0;
  out->launches = 0;
  out->cond_L1 = 0.0;
  out->x_f64 = 0;
  for (int i = 0; i < ID_NUM_PHASES; ++i) {
    out->phase_ms[i] = 0.0;
    out->phase_launches[i] = 0;
  }
}

}  // namespace

extern "C" {

int id_workspace_size(const id_matrix* A, const id_opts* opts, int64_t l, size_t* bytes) {
  if (bytes == nullptr) return -4;
  if (l < 0) return -3;
  Plan p;
  const int rc = make_plan(A, opts, l > 0 ? 1 : 0, l, &p);
  if (rc != ID_OK) return rc == kBadA ? -1 : (rc == kBadOpts ? -2 : (rc < -100 ? rc : -3));
  *bytes = p.total;
  return ID_OK;
}

int id_fixed_rank(const id_matrix* A, int64_t k, int64_t l, const id_opts* opts, void* ws, size_t ws_bytes,
                  id_result* out, void* stream) {
  Plan p;
  int rc = make_plan(A, opts, k, l, &p);
  if (rc != ID_OK) return rc == kBadA ? -1 : (rc == kBadOpts ? -4 : (rc == kBadK ? -2 : (rc == kBadL ? -3 : rc)));
  if (check_out(p, out) != ID_OK) return -7;
  if (check_ws(p, ws, ws_bytes) != ID_OK) return ID_ERR_WORKSPACE;
  clear_out(out);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision_path(A, opts) >= 64) {
    Engine<double> e(p, A, opts, ws, out, s);
    return e.run_fixed();
  }
  Engine<float> e(p, A, opts, ws, out, s);
  return e.run_fixed();
}

int id_adaptive(const id_matrix* A, const id_opts* opts, void* ws, size_t ws_bytes, id_result* out, void* stream) {
  Plan p;
  int rc = make_plan(A, opts, 0, 0, &p);
  if (rc != ID_OK) return rc == kBadA ? -1 : (rc == kBadOpts ? -2 : rc);
  if (check_out(p, out) != ID_OK) return -5;
  if (check_ws(p, ws, ws_bytes) != ID_OK) return ID_ERR_WORKSPACE;
  clear_out(out);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision_path(A, opts) >= 64) {
    Engine<double> e(p, A, opts, ws, out, s);
    return e.run_adaptive();
  }
  Engine<float> e(p, A, opts, ws, out, s);
  return e.run_adaptive();
}

namespace {
// Plan of cur_from_id: the panel C = A(:,J) has m rows (the items pivoted) and k
// columns; the interpolation buffer (k x m) follows the engine's workspace.
int cur_plan(const id_matrix* A, int64_t k, Plan* p, size_t* xoff, size_t* total) {
  if (A == nullptr || A->data == nullptr || A->m < 1 || A->n < 1 || A->ld < A->m || A->m >= ((int64_t)1 << 30))
    return -1;
  if (A->dtype != ID_F64 && A->dtype != ID_F32) return ID_ERR_UNSUPPORTED;
  if (k < 1 || k > A->m || k > A->n) return -3;
  id_matrix P = *A;
  P.m = k;  // the panel is gathered, not sketched: only its k columns matter
  P.n = A->m;
  P.ld = k;
  id_opts o;
  memset(&o, 0, sizeof(o));
  o.sketch_prec = o.lu_prec = A->dtype;
  o.block = 64;
  const int rc = make_plan(&P, &o, k, k, p);
  if (rc != ID_OK) return rc;
  *xoff = p->total;
  *total = p->total + align_up((size_t)k * A->m * p->esz);
  return ID_OK;
}
}  // namespace

int id_cur_workspace_size(const id_matrix* A, int64_t k, size_t* bytes) {
  if (bytes == nullptr) return -3;
  Plan p;
  size_t xoff = 0;
  const int rc = cur_plan(A, k, &p, &xoff, bytes);
  return rc == -3 ? -2 : rc;
}

int cur_from_id(const id_matrix* A, const int64_t* J, int64_t k, int64_t* I, void* W, int64_t ldw, void* ws,
                size_t ws_bytes, void* stream) {
  Plan p;
  size_t xoff = 0, total = 0;
  const int rc = cur_plan(A, k, &p, &xoff, &total);
  if (rc != ID_OK) return rc;
  if (J == nullptr) return -2;
  if (I == nullptr) return -4;
  if (W == nullptr || ldw < A->m) return -5;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 || ws_bytes < total)
    return ID_ERR_WORKSPACE;
  id_matrix P = *A;
  P.m = k;
  P.n = A->m;
  P.ld = k;
  id_opts o;
  memset(&o, 0, sizeof(o));
  o.sketch_prec = o.lu_prec = A->dtype;
  o.block = 64;
  id_result out;
  memset(&out, 0, sizeof(out));
  out.J = I;
  out.X = static_cast<unsigned char*>(ws) + xoff;
  out.ldx = k;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st;
  if (A->dtype == ID_F64) {
    Engine<double> e(p, &P, &o, ws, &out, s);
    st = e.run_panel(static_cast<const double*>(A->data), A->m, A->n, A->ld, J);
    if (st >= 0 && transpose_w<double>(static_cast<const double*>(out.X), k, A->m, k, static_cast<double*>(W), ldw,
                                       s) != cudaSuccess)
      return ID_ERR_CUDA;
  } else {
    Engine<float> e(p, &P, &o, ws, &out, s);
    st = e.run_panel(static_cast<const float*>(A->data), A->m, A->n, A->ld, J);
    if (st >= 0 && transpose_w<float>(static_cast<const float*>(out.X), k, A->m, k, static_cast<float*>(W), ldw,
                                      s) != cudaSuccess)
      return ID_ERR_CUDA;
  }
  if (st < 0) return st;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ID_ERR_CUDA;
  return st;
}

int id_gaussian_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t m, id_dtype dtype, void* out, int64_t ld,
                     void* stream) {
  if (row0 < 0) return -2;
  if (rows < 0) return -3;
  if (m < 1) return -4;
  if (dtype != ID_F64 && dtype != ID_F32 && dtype != ID_BF16 && dtype != ID_FP8_E4M3 && dtype != ID_F64_EMU)
    return -5;
  if (out == nullptr) return -6;
  if (ld < m) return -7;
  if (rows == 0) return ID_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype == ID_F64)
    e = gaussian_rows<double>(seed, row0, rows, m, static_cast<double*>(out), ld, nullptr, s);
  else if (dtype == ID_F64_EMU)
    e = f64emu_omega_grid(seed, row0, rows, m, static_cast<double*>(out), ld, s);
  else if (dtype == ID_F32)
    e = gaussian_rows<float>(seed, row0, rows, m, static_cast<float*>(out), ld, nullptr, s);
  else if (dtype == ID_BF16)
    e = gaussian_rows<__nv_bfloat16>(seed, row0, rows, m, static_cast<__nv_bfloat16*>(out), ld, nullptr, s);
  else
    e = gaussian_rows<__nv_fp8_e4m3>(seed, row0, rows, m, static_cast<__nv_fp8_e4m3*>(out), ld, nullptr, s);
  if (e != cudaSuccess) return ID_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ID_ERR_CUDA;
  return ID_OK;
}

int id_sparse_sign_rows(uint64_t seed, int64_t t0, int64_t blocks, int64_t b, int64_t m, int64_t zeta,
                        id_dtype dtype, void* out, int64_t ld, void* stream) {
  if (t0 < 0) return -2;
  if (blocks < 0 || blocks > ((int64_t)1 << 24)) return -3;
  if (b < 1 || b > kSparseMaxB) return -4;
  if (m < 1) return -5;
  if (zeta < 1 || zeta > b) return -6;
  if (dtype != ID_F64 && dtype != ID_F32) return -7;
  if (out == nullptr) return -8;
  if (ld < m) return -9;
  if (blocks == 0) return ID_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = dtype == ID_F64
                      ? sparse_dense<double>(seed, t0, (int)blocks, (int)b, m, (int)zeta, static_cast<double*>(out), ld, s)
                      : sparse_dense<float>(seed, t0, (int)blocks, (int)b, m, (int)zeta, static_cast<float*>(out), ld, s);
  if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return ID_ERR_CUDA;
  return ID_OK;
}

int id_quantize_fp8(const id_matrix* A, void* Q, int64_t ldq, float* block_scale, int pow2, void* stream) {
  if (A == nullptr || A->data == nullptr || A->m < 1 || A->n < 1 || A->ld < A->m ||
      (A->dtype != ID_F64 && A->dtype != ID_F32 && A->dtype != ID_BF16))
    return -1;
  if (Q == nullptr || ldq < A->m) return -2;
  if (block_scale == nullptr) return -4;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (quantize_fp8(A->dtype, A->m, A->n, A->data, A->ld, Q, ldq, block_scale, pow2, s) != cudaSuccess)
    return ID_ERR_CUDA;
  return ID_OK;
}

namespace {
// Split count and workspace of a stand-alone sketch: DevState + split-K partials.
int sketch_plan(const id_matrix* A, int64_t rows, id_dtype prec, int* path, int* splits, size_t* bytes) {
  if (A == nullptr || A->data == nullptr || A->m < 1 || A->n < 1 || A->ld < A->m || A->m >= ((int64_t)1 << 31) ||
      A->n >= ((int64_t)1 << 30))
    return -1;
  if (rows < 1 || rows > ((int64_t)1 << 20)) return -2;
  *path = (A->dtype == ID_F64 && prec == ID_F64)       ? 64
          : (A->dtype == ID_F64 && prec == ID_F64_EMU) ? 65
          : (A->dtype == ID_F32 && prec == ID_F32)     ? 32
          : (A->dtype == ID_F32 && prec == ID_F32_EMU) ? 33
          : (A->dtype == ID_BF16 && prec == ID_BF16)   ? 16
          : (A->dtype == ID_FP8_E4M3 && prec == ID_FP8_E4M3) ? 8
                                                       : 0;
  if (*path == 0) return ID_ERR_UNSUPPORTED;
  const int sms = num_sms();
  if (*path == 8 && A->block_scale == nullptr) return -1;
  const size_t esz = *path >= 64 ? 8 : 4;
  *splits = *path == 16   ? tc_sketch_effective_splits(A->m, tc_sketch_splits(A->m, A->n, rows, sms))
            : *path == 8  ? tc_fp8_effective_splits(A->m, tc_fp8_splits(A->m, A->n, rows, sms))
            : *path == 65 ? f64emu_splits(A->m, A->n, sms)
            : *path == 33 ? sketch_f32emu_splits(A->m, A->n, rows, sms)
            : *path == 32 ? gemm_splits((int)A->m, choose_splits_sgemm(A->n, rows, A->m, sms, 16, 2))
                          : gemm_splits((int)A->m, choose_splits_sgemm(A->n, rows, A->m, sms, 16, 1));
  *bytes = 256 + (*splits > 1 ? align_up((size_t)*splits * A->n * rows * esz) : 0);
  if (*path == 33)  // digits and exponents of A and of Omega
    *bytes += align_up(sketch_f32emu_digit_bytes(A->n, A->m)) + align_up((size_t)A->n * 4) +
              align_up(sketch_f32emu_digit_bytes(rows, A->m)) + align_up((size_t)rows * 4);
  if (*path == 65) {  // digit slices of A, column exponents, two digit planes of Omega
    const size_t mp = (size_t)f64emu_pad(A->m);
    *bytes += align_up(f64emu_digit_bytes(A->m, A->n)) + align_up((size_t)A->n * 4) + align_up(2 * mp * rows * 2);
  }
  return ID_OK;
}
}  // namespace

int id_sketch_workspace_size(const id_matrix* A, int64_t rows, id_dtype sketch_prec, size_t* bytes) {
  if (bytes == nullptr) return -4;
  int path = 0, splits = 1;
  const int rc = sketch_plan(A, rows, sketch_prec, &path, &splits, bytes);
  return rc == -2 ? -2 : rc;
}

namespace {
// The sketch G = (omega A)^T (n x rows, row stride ldg) on path `path` with the
// split-K count sketch_plan chose.  ws: the DevState (256 bytes), then the
// partials and digit planes sketch_plan sized.  Returns the first launch error.
cudaError_t run_sketch(const id_matrix* A, const void* omega, int64_t ld_omega, int64_t rows, int path, int splits,
                       void* G, int64_t ldg, void* ws, cudaStream_t s) {
  DevState* st = static_cast<DevState*>(ws);
  void* part = static_cast<unsigned char*>(ws) + 256;
  cudaError_t e0 = init_state(st, nullptr, nullptr, 0, s);
  if (e0 != cudaSuccess) return e0;
  cudaError_t e = cudaSuccess;
  // split-K partials: row stride rows (what the workspace holds), reduced into G (row stride ldg)
  const int64_t zs = A->n * rows;
  if (path == 16) {
    float* out = splits > 1 ? static_cast<float*>(part) : static_cast<float*>(G);
    e = tc_sketch_bf16(A->data, A->ld, A->m, A->n, omega, ld_omega, rows, out, splits > 1 ? rows : ldg, zs, splits,
                       st, nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<float>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<float*>(part),
                                  static_cast<float*>(G), nullptr, s);
  } else if (path == 8) {
    float* out = splits > 1 ? static_cast<float*>(part) : static_cast<float*>(G);
    e = tc_sketch_fp8(A->data, A->ld, A->m, A->n, A->block_scale, omega, ld_omega, rows, out, splits > 1 ? rows : ldg,
                      zs, splits, st, nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<float>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<float*>(part),
                                  static_cast<float*>(G), nullptr, s);
  } else if (path == 33) {
    unsigned char* w = static_cast<unsigned char*>(part) + (splits > 1 ? align_up((size_t)splits * A->n * rows * 4) : 0);
    void* ad = w;
    int32_t* ae = reinterpret_cast<int32_t*>(w + align_up(sketch_f32emu_digit_bytes(A->n, A->m)));
    void* wd = w + align_up(sketch_f32emu_digit_bytes(A->n, A->m)) + align_up((size_t)A->n * 4);
    int32_t* we = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(wd) +
                                             align_up(sketch_f32emu_digit_bytes(rows, A->m)));
    float* out = splits > 1 ? static_cast<float*>(part) : static_cast<float*>(G);
    e = sketch_f32emu_slice((int)A->n, (int)A->m, static_cast<const float*>(A->data), A->ld, ad, A->n, ae, nullptr,
                            nullptr, s);
    if (e == cudaSuccess)
      e = sketch_f32emu_slice((int)rows, (int)A->m, static_cast<const float*>(omega), ld_omega, wd, rows, we, nullptr,
                              nullptr, s);
    if (e == cudaSuccess)
      e = sketch_f32emu(A->m, A->n, rows, ad, ae, wd, rows, we, out, splits > 1 ? rows : ldg, zs, splits, st, nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<float>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<float*>(part),
                                  static_cast<float*>(G), nullptr, s);
  } else if (path == 65) {
    unsigned char* w = static_cast<unsigned char*>(part) + (splits > 1 ? align_up((size_t)splits * A->n * rows * 8) : 0);
    const size_t mp = (size_t)f64emu_pad(A->m);
    void* digits = w;
    int32_t* colexp = reinterpret_cast<int32_t*>(w + align_up(f64emu_digit_bytes(A->m, A->n)));
    void* wdig = w + align_up(f64emu_digit_bytes(A->m, A->n)) + align_up((size_t)A->n * 4);
    double* out = splits > 1 ? static_cast<double*>(part) : static_cast<double*>(G);
    e = f64emu_prepare(static_cast<const double*>(A->data), A->ld, A->m, A->n, colexp, digits, s);
    if (e == cudaSuccess)
      e = f64emu_omega(0, 0, rows, A->m, rows, static_cast<const double*>(omega), ld_omega, wdig, nullptr, s);
    if (e == cudaSuccess)
      e = f64emu_sketch(digits, colexp, A->m, A->n, wdig, rows, rows, out, splits > 1 ? rows : ldg, zs, splits, st,
                        nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<double>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<double*>(part),
                                   static_cast<double*>(G), nullptr, s);
  } else if (path == 64) {
    Operand<double> a{static_cast<const double*>(A->data), A->ld, nullptr, 0};
    Operand<double> w{static_cast<const double*>(omega), ld_omega, nullptr, 0};
    double* out = splits > 1 ? static_cast<double*>(part) : static_cast<double*>(G);
    EpiArgs<double> ep{out, splits > 1 ? rows : ldg, zs, nullptr, nullptr};
    e = gemm_gather<double>((int)A->n, (int)rows, (int)A->m, splits, true, a, w, kEpiStore, ep, nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<double>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<double*>(part),
                                   static_cast<double*>(G), nullptr, s);
  } else {
    Operand<float> a{static_cast<const float*>(A->data), A->ld, nullptr, 0};
    Operand<float> w{static_cast<const float*>(omega), ld_omega, nullptr, 0};
    float* out = splits > 1 ? static_cast<float*>(part) : static_cast<float*>(G);
    EpiArgs<float> ep{out, splits > 1 ? rows : ldg, zs, nullptr, nullptr};
    e = gemm_gather<float>((int)A->n, (int)rows, (int)A->m, splits, true, a, w, kEpiStore, ep, nullptr, s);
    if (e == cudaSuccess && splits > 1)
      e = splitk_reduce_ld<float>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<float*>(part),
                                  static_cast<float*>(G), nullptr, s);
  }
  return e;
}
}  // namespace

int id_sketch(const id_matrix* A, const void* omega, int64_t ld_omega, int64_t rows, id_dtype sketch_prec, void* G,
              int64_t ldg, void* ws, size_t ws_bytes, void* stream) {
  int path = 0, splits = 1;
  size_t need = 0;
  int rc = sketch_plan(A, rows, sketch_prec, &path, &splits, &need);
  if (rc != ID_OK) return rc == -2 ? -4 : rc;
  if (omega == nullptr || ld_omega < A->m) return -2;
  if (G == nullptr || ldg < rows) return -6;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 || ws_bytes < need)
    return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (path == 16 && !tc_sketch_supported(A->data, A->ld, omega, ld_omega)) return ID_ERR_UNSUPPORTED;
  if (path == 8 && !tc_fp8_supported(A->data, A->ld, omega, ld_omega)) return ID_ERR_UNSUPPORTED;
  DevState* st = static_cast<DevState*>(ws);
  cudaError_t e = run_sketch(A, omega, ld_omega, rows, path, splits, G, ldg, ws, s);
  if (e != cudaSuccess) return ID_ERR_CUDA;
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ID_ERR_CUDA;
  return (h.err & kErrTimeout) ? ID_ERR_TIMEOUT : ID_OK;
}

namespace {
// Workspace of id_sparse_sketch: a DevState, the per-tile lists of the blocks, the
// split-K partials (16-byte exact integers for FP64 A), then for FP64 A its
// fixed-point copy and column exponents.
int sparse_sketch_plan(const id_matrix* A, int64_t rows, int64_t b, int64_t zeta, int* splits, size_t* off_parts,
                       size_t* bytes) {
  if (A == nullptr || A->data == nullptr || A->m < 1 || A->n < 1 || A->ld < A->m || A->m >= ((int64_t)1 << 31) ||
      A->n >= ((int64_t)1 << 30))
    return -1;
  if (A->dtype != ID_F64 && A->dtype != ID_F32 && A->dtype != ID_BF16) return ID_ERR_UNSUPPORTED;
  if (rows < 1 || rows > ((int64_t)1 << 20)) return -2;
  if (b < 1 || b > kSparseMaxB) return -3;
  if (zeta < 1 || zeta > b) return -4;
  if (cdiv(rows, b) > 65535) return -2;
  const int kind = A->dtype == ID_F64 ? 2 : (A->dtype == ID_BF16 ? 1 : 0);
  *splits = sparse_splits(A->m, A->n, num_sms(), kind);
  const size_t psz = A->dtype == ID_F64 ? 16 : 4;
  *off_parts = 256 + align_up(sparse_csr_bytes(A->m, (int)cdiv(rows, b), (int)b, (int)zeta));
  *bytes = *off_parts + (*splits > 1 ? align_up((size_t)*splits * A->n * rows * psz) : 0);
  if (A->dtype == ID_F64)  // the fixed-point copy of A and its column exponents follow
    *bytes += align_up((size_t)A->m * A->n * 8) + align_up((size_t)A->n * 4);
  return ID_OK;
}
}  // namespace

int id_sparse_sketch_workspace_size(const id_matrix* A, int64_t rows, int64_t b, int64_t zeta, size_t* bytes) {
  if (bytes == nullptr) return -5;
  int splits = 1;
  size_t off = 0;
  return sparse_sketch_plan(A, rows, b, zeta, &splits, &off, bytes);
}

int id_sparse_sketch(const id_matrix* A, uint64_t seed, int64_t t0, int64_t rows, int64_t b, int64_t zeta, void* G,
                     int64_t ldg, void* ws, size_t ws_bytes, void* stream) {
  int splits = 1;
  size_t off = 0, need = 0;
  const int rc = sparse_sketch_plan(A, rows, b, zeta, &splits, &off, &need);
  if (rc != ID_OK) return rc == -2 ? -4 : (rc == -3 ? -5 : (rc == -4 ? -6 : rc));
  if (t0 < 0) return -3;
  if (G == nullptr || ldg < rows) return -7;
  // BF16 tiles are copied in element pairs: even leading dimension, 4-byte aligned base
  if (A->dtype == ID_BF16 && ((A->ld & 1) != 0 || (reinterpret_cast<uintptr_t>(A->data) & 3) != 0))
    return ID_ERR_UNSUPPORTED;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 || ws_bytes < need)
    return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  uint16_t* R = reinterpret_cast<uint16_t*>(w + 256);
  void* part = w + off;
  const int64_t zs = A->n * rows;
  const int esz = A->dtype == ID_F64 ? 8 : (A->dtype == ID_BF16 ? 2 : 4);
  cudaError_t e = sparse_csr(seed, t0, (int)cdiv(rows, b), (int)b, A->m, (int)zeta, esz, R, nullptr, s);
  if (e == cudaSuccess) {
    if (A->dtype == ID_F64) {
      unsigned char* fx = w + off + (splits > 1 ? align_up((size_t)splits * A->n * rows * 16) : 0);
      long long* F = reinterpret_cast<long long*>(fx);
      int32_t* col = reinterpret_cast<int32_t*>(fx + align_up((size_t)A->m * A->n * 8));
      e = sparse_fixed_prepare(static_cast<const double*>(A->data), A->ld, A->m, A->n, col, F, s);
      if (e == cudaSuccess)
        e = sparse_sketch_fixed(A->m, A->n, F, col, R, (int)zeta, (int)b, rows, splits, static_cast<double*>(G), ldg,
                                part, rows, zs, nullptr, s);
    } else {
      float* out = splits > 1 ? static_cast<float*>(part) : static_cast<float*>(G);
      if (A->dtype == ID_F32)
        e = sparse_sketch<float>(A->m, A->n, static_cast<const float*>(A->data), A->ld, R, (int)zeta, (int)b, rows,
                                 splits, out, splits > 1 ? rows : ldg, zs, nullptr, s);
      else
        e = sparse_sketch<__nv_bfloat16>(A->m, A->n, static_cast<const __nv_bfloat16*>(A->data), A->ld, R, (int)zeta,
                                         (int)b, rows, splits, out, splits > 1 ? rows : ldg, zs, nullptr, s);
      if (e == cudaSuccess && splits > 1)
        e = splitk_reduce_ld<float>(A->n, (int)rows, rows, ldg, splits, zs, static_cast<float*>(part),
                                    static_cast<float*>(G), nullptr, s);
    }
  }
  if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return ID_ERR_CUDA;
  return ID_OK;
}

}  // extern "C"

namespace {
// Workspace of id_certificate: a DevState, the rows of Omega', the sketch's own
// workspace (sketch_plan), G = (Omega' A)^T (n x q), the index lists, the split-K
// partials of X^T G(J,:), the residual R = G - X^T G(J,:) and its sums of squares.
struct CertPlan {
  int path = 0, sk_splits = 1, nz = 1, nparts = 0;
  size_t esz = 8, wsz = 8;  // bytes per element of G and X, of Omega'
  int64_t ldo = 0;
  size_t off_st = 0, off_omega = 0, off_sk = 0, off_G = 0, off_iota = 0, off_j32 = 0, off_P = 0, off_R = 0,
         off_e2 = 0, total = 0;
};

int cert_plan(const id_matrix* A, int64_t k, int64_t q, id_dtype prec, CertPlan* c) {
  size_t skb = 0;
  const int rc = sketch_plan(A, q, prec, &c->path, &c->sk_splits, &skb);
  if (rc == -2) return -6;
  if (rc != ID_OK) return rc;
  if (k < 1 || k > imin(A->m, A->n)) return -5;
  const int sms = num_sms();
  const bool f64 = c->path >= 64;
  c->esz = f64 ? 8 : 4;
  c->wsz = f64 ? 8 : (c->path == 16 ? 2 : (c->path == 8 ? 1 : 4));
  c->ldo = c->path == 16 ? cdiv(A->m, 8) * 8 : (c->path == 8 ? cdiv(A->m, 16) * 16 : A->m);
  const int want = f64 ? choose_splits_gather(A->n, q, k, sms, 8) : choose_splits_sgemm(A->n, q, k, sms, 32, 2);
  c->nz = gemm_splits((int)k, want);
  c->nparts = 2 * sms;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + (bytes == 0 ? 1 : bytes));
    return at;
  };
  c->off_st = take(256);
  c->off_omega = take((size_t)q * c->ldo * c->wsz);
  c->off_sk = take(skb);
  c->off_G = take((size_t)A->n * q * c->esz);
  c->off_iota = take((size_t)A->n * 4);
  c->off_j32 = take((size_t)k * 4);
  c->off_P = take((size_t)c->nz * A->n * q * c->esz);
  c->off_R = take((size_t)A->n * q * c->esz);
  c->off_e2 = take((size_t)c->nparts * 8);
  c->total = off;
  return ID_OK;
}

// R = G - X^T G(J,:) (the residual of the ID on the fresh sample) and its squared
// norm per block, then E = sqrt(sum / q).
template <typename T>
cudaError_t cert_residual(const CertPlan& c, int64_t n, int64_t k, int64_t q, const void* X, int64_t ldx,
                          unsigned char* w, cudaStream_t s) {
  const T* G = reinterpret_cast<const T*>(w + c.off_G);
  const int32_t* iota = reinterpret_cast<const int32_t*>(w + c.off_iota);
  const int32_t* j32 = reinterpret_cast<const int32_t*>(w + c.off_j32);
  T* P = reinterpret_cast<T*>(w + c.off_P);
  T* R = reinterpret_cast<T*>(w + c.off_R);
  double* e2 = reinterpret_cast<double*>(w + c.off_e2);
  DevState* st = reinterpret_cast<DevState*>(w + c.off_st);
  Operand<T> a{static_cast<const T*>(X), ldx, nullptr, 0};
  Operand<T> b{G, q, j32, 0};
  EpiArgs<T> ep{P, q, n * q, nullptr, nullptr};
  cudaError_t e = gemm_gather<T>((int)n, (int)q, (int)k, c.nz, false, a, b, kEpiStore, ep, nullptr, s);
  if (e == cudaSuccess)
    e = schur_finish<T>((int)n, (int)q, iota, G, q, 0, c.nz, n * q, P, R, q, e2, c.nparts, nullptr, s);
  if (e == cudaSuccess) e = rid::decide(e2, c.nparts, (int)q, INFINITY, 0, 0, 0, nullptr, 0, st, s);
  return e;
}
}  // namespace

extern "C" {

int id_certificate_workspace_size(const id_matrix* A, int64_t k, int64_t q, id_dtype sketch_prec, size_t* bytes) {
  if (bytes == nullptr) return -5;
  CertPlan c;
  const int rc = cert_plan(A, k, q, sketch_prec, &c);
  if (rc != ID_OK) return rc == -5 ? -2 : (rc == -6 ? -3 : (rc == -1 ? -1 : (rc == ID_ERR_UNSUPPORTED ? rc : -4)));
  *bytes = c.total;
  return ID_OK;
}

int id_certificate(const id_matrix* A, const int64_t* J, const void* X, int64_t ldx, int64_t k, int64_t q,
                   id_dtype sketch_prec, uint64_t seed, int64_t row0, const void* omega, int64_t ld_omega,
                   double* est, void* ws, size_t ws_bytes, void* stream) {
  CertPlan c;
  int rc = cert_plan(A, k, q, sketch_prec, &c);
  if (rc == -6) return -6;
  if (rc == -5) return -5;
  if (rc != ID_OK) return rc == ID_ERR_UNSUPPORTED ? rc : (rc == -1 ? -1 : -7);
  if (J == nullptr) return -2;
  if (X == nullptr) return -3;
  if (ldx < k) return -4;
  if (omega == nullptr && row0 < 0) return -9;
  if (omega != nullptr && ld_omega < A->m) return -11;
  if (est == nullptr) return -12;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0 || ws_bytes < c.total)
    return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (omega != nullptr && c.path == 16 && !tc_sketch_supported(A->data, A->ld, omega, ld_omega))
    return ID_ERR_UNSUPPORTED;
  if (omega != nullptr && c.path == 8 && !tc_fp8_supported(A->data, A->ld, omega, ld_omega))
    return ID_ERR_UNSUPPORTED;
  unsigned char* w = static_cast<unsigned char*>(ws);
  DevState* st = reinterpret_cast<DevState*>(w + c.off_st);
  const int64_t m = A->m, n = A->n;
  cudaError_t e = init_state(st, nullptr, nullptr, 0, s);
  const void* Om = omega;
  int64_t ldo = ld_omega;
  if (e == cudaSuccess && omega == nullptr) {  // Omega' rows [row0, row0 + q) of the generator `seed`
    void* buf = w + c.off_omega;
    if (c.path >= 64)
      e = gaussian_rows<double>(seed, row0, q, m, static_cast<double*>(buf), c.ldo, nullptr, s);
    else if (c.path == 16)
      e = gaussian_rows<__nv_bfloat16>(seed, row0, q, m, static_cast<__nv_bfloat16*>(buf), c.ldo, nullptr, s);
    else if (c.path == 8)
      e = gaussian_rows<__nv_fp8_e4m3>(seed, row0, q, m, static_cast<__nv_fp8_e4m3*>(buf), c.ldo, nullptr, s);
    else
      e = gaussian_rows<float>(seed, row0, q, m, static_cast<float*>(buf), c.ldo, nullptr, s);
    Om = buf;
    ldo = c.ldo;
  }
  if (e == cudaSuccess) e = run_sketch(A, Om, ldo, q, c.path, c.sk_splits, w + c.off_G, q, w + c.off_sk, s);
  if (e == cudaSuccess) e = index32(J, k, n, reinterpret_cast<int32_t*>(w + c.off_j32), st, s);
  if (e == cudaSuccess) e = iota32(reinterpret_cast<int32_t*>(w + c.off_iota), n, s);
  if (e == cudaSuccess)
    e = c.path >= 64 ? cert_residual<double>(c, n, k, q, X, ldx, w, s) : cert_residual<float>(c, n, k, q, X, ldx, w, s);
  if (e != cudaSuccess) return ID_ERR_CUDA;
  DevState h, hs;
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hs, w + c.off_sk, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ID_ERR_CUDA;
  if ((h.err | hs.err) & kErrTimeout) return ID_ERR_TIMEOUT;
  if (h.err & kErrBadIndex) return -2;
  *est = h.est;
  return ID_OK;
}

int id_ur_estimates(const id_matrix* A, int64_t k, int64_t p, const id_opts* opts, void* ws, size_t ws_bytes,
                    id_result* out, void* U_r, int64_t ldu, int64_t* J_extra, id_ur_stats* stats, void* stream) {
  if (p < 1 || p > kMaxBlock) return -3;
  if (A != nullptr && (k < 1 || k + p > imin(A->m, A->n))) return k < 1 ? -2 : -3;
  Plan pl;
  int rc = make_plan(A, opts, k, k + p, &pl);
  if (rc != ID_OK) return rc == kBadA ? -1 : (rc == kBadOpts ? -4 : (rc == kBadK ? -2 : (rc == kBadL ? -3 : rc)));
  if (check_ws(pl, ws, ws_bytes) != ID_OK) return ID_ERR_WORKSPACE;
  if (check_out(pl, out) != ID_OK) return -7;
  if (U_r == nullptr || ldu < p) return -8;
  if (stats == nullptr) return -11;
  clear_out(out);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double h[2] = {0.0, 0.0};
  int st;
  if (precision_path(A, opts) >= 64) {
    Engine<double> e(pl, A, opts, ws, out, s);
    st = e.run_ur(p, static_cast<double*>(U_r), ldu, J_extra, h);
  } else {
    Engine<float> e(pl, A, opts, ws, out, s);
    st = e.run_ur(p, static_cast<float*>(U_r), ldu, J_extra, h);
  }
  if (st < 0) return st;
  stats->u_fro = sqrt(h[0]);
  stats->u_max = h[1];
  stats->est = out->est_err;
  stats->bound = sqrt((double)(A->n - k)) * stats->u_fro;
  return st;
}

const char* id_status_string(int status) {
  switch (status) {
    case ID_OK: return "ok";
    case ID_WARN_TOL_NOT_MET: return "warning: rank cap reached before the tolerance was met";
    case ID_WARN_ZERO_PIVOT: return "warning: an exactly zero pivot column was met";
    case ID_WARN_TOL_NOT_MET | ID_WARN_ZERO_PIVOT: return "warning: rank cap reached and a zero pivot was met";
    case ID_ERR_NONFINITE: return "error: the input holds NaN or Inf";
    case ID_ERR_CUDA: return "error: a CUDA runtime call failed";
    case ID_ERR_TIMEOUT: return "error: a bounded device-side wait timed out";
    case ID_ERR_WORKSPACE: return "error: workspace missing, misaligned or too small";
    case ID_ERR_UNSUPPORTED: return "error: this precision combination or entry point is not built";
    default: break;
  }
  if (status < 0 && status > -100) return "error: invalid argument (see -status for its position)";
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------- fixed rank without allocation
// Scratch for id_fixed_rank_noalloc: a static device array, so that callers
// who may not allocate device memory still get a working ID.  In host code
// `g_noalloc_scratch` names a host-side stand-in; kernels only ever receive the
// device address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ID_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch on the current device.  The lookup
// needs that device current and must not run while a stream is being
// captured; its result is kept per device.  Entries are atomic and the first
// lookup on a device runs under a lock, so concurrent first calls from several
// host threads agree on one address.
std::atomic<void*> g_noalloc_addr[64];
std::mutex g_noalloc_mu;

int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ID_ERR_CUDA;
  void* a = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (a == nullptr) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    a = g_noalloc_addr[dev].load(std::memory_order_relaxed);
    if (a == nullptr) {
      if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || a == nullptr) return ID_ERR_CUDA;
      g_noalloc_addr[dev].store(a, std::memory_order_release);
    }
  }
  *out = a;
  return ID_OK;
}

}  // namespace

extern "C" int id_fixed_rank_noalloc(const id_matrix* A, int64_t k, int64_t l, const id_opts* opts,
                                     id_result* out, void* stream) {
  Plan p;
  int rc = make_plan(A, opts, k, l, &p);
  if (rc != ID_OK) return rc == kBadA ? -1 : (rc == kBadOpts ? -4 : (rc == kBadK ? -2 : (rc == kBadL ? -3 : rc)));
  if (check_out(p, out) != ID_OK) return -5;
  if (p.total > ID_NOALLOC_SCRATCH_BYTES) return ID_ERR_WORKSPACE;  // does not fit the static buffer
  void* ws = nullptr;
  rc = noalloc_scratch(&ws);
  if (rc != ID_OK) return rc;
  id_opts o = *opts;
  o.profile = 0;  // no event objects
  clear_out(out);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision_path(A, &o) >= 64) {
    Engine<double> e(p, A, &o, ws, out, s);
    return e.run_fixed();
  }
  Engine<float> e(p, A, &o, ws, out, s);
  return e.run_fixed();
}
