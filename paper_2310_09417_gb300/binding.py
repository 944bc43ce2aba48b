"""Thin Python binding of the C ABI in include/randid.h.

Argument marshalling only: every step of the ID runs in the CUDA library.
PyTorch provides device memory (inputs, outputs, workspace) and the stream.
Matrices are column-major: pass A as a CUDA tensor of shape (m, n) with
stride (1, ld), e.g. ``colmajor(t)``.  If the library has not been built the
first call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librandid.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "randid.h")

# id_dtype
F64, F32, BF16, FP8_E4M3, F64_EMU, F32_EMU = 0, 1, 2, 3, 4, 5
# status
OK, WARN_TOL_NOT_MET, WARN_ZERO_PIVOT = 0, 1, 2
ERR_NONFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_WORKSPACE, ERR_UNSUPPORTED = -101, -102, -103, -104, -105
PHASES = ("omega", "sketch", "schur", "lu", "update", "other")
# id_opts.omega_kind
OMEGA_GAUSSIAN, OMEGA_SPARSE_SIGN = 0, 1
# cur_middle's middle_kind
CUR_PSEUDOINVERSE, CUR_INVERSE = 0, 1

_TORCH_TO_ID = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}
if hasattr(torch, "float8_e4m3fn"):
    _TORCH_TO_ID[torch.float8_e4m3fn] = FP8_E4M3


class IdMatrix(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("m", C.c_int64), ("n", C.c_int64),
                ("ld", C.c_int64), ("block_scale", C.c_void_p)]


class IdOpts(C.Structure):
    _fields_ = [("sketch_prec", C.c_int), ("lu_prec", C.c_int), ("block", C.c_int64),
                ("tol", C.c_double), ("tol_relative", C.c_int), ("k_max", C.c_int64),
                ("k0", C.c_int64), ("blocks_per_pass", C.c_int64), ("seed", C.c_uint64),
                ("omega", C.c_void_p), ("ld_omega", C.c_int64), ("omega_rows", C.c_int64),
                ("profile", C.c_int), ("predictor", C.c_void_p), ("max_pass_rows", C.c_int64),
                ("x_solve_f64", C.c_int), ("omega_kind", C.c_int), ("zeta", C.c_int64)]


class IdResult(C.Structure):
    _fields_ = [("k", C.c_int64), ("J", C.c_void_p), ("X", C.c_void_p), ("ldx", C.c_int64),
                ("pivots", C.c_void_p), ("est_trace", C.c_void_p), ("trace_cap", C.c_int64),
                ("est_err", C.c_double), ("norm_A", C.c_double), ("rounds", C.c_int32),
                ("passes", C.c_int32), ("launches", C.c_int64),
                ("phase_ms", C.c_double * 6), ("phase_launches", C.c_int64 * 6),
                ("status", C.c_int32), ("cond_L1", C.c_double), ("x_f64", C.c_int32)]


_lib = None


def load():
    """Load librandid.so; raise if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librandid.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_2310_09417_gb300.build" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P, i64, u64 = C.c_void_p, C.c_int64, C.c_uint64
    lib.id_workspace_size.argtypes = [P, P, i64, C.POINTER(C.c_size_t)]
    lib.id_fixed_rank.argtypes = [P, i64, i64, P, P, C.c_size_t, P, P]
    lib.id_adaptive.argtypes = [P, P, P, C.c_size_t, P, P]
    lib.id_batched_workspace_size.argtypes = [i64, P, P, C.POINTER(C.c_size_t)]
    lib.id_batched.argtypes = [i64, P, P, P, C.c_size_t, P, P]
    lib.cur_from_id.argtypes = [P, P, i64, P, P, i64, P, C.c_size_t, P]
    lib.id_cur_workspace_size.argtypes = [P, i64, C.POINTER(C.c_size_t)]
    lib.id_cur_workspace_size.restype = C.c_int
    lib.id_gaussian_rows.argtypes = [u64, i64, i64, i64, C.c_int, P, i64, P]
    lib.id_sketch_workspace_size.argtypes = [P, i64, C.c_int, C.POINTER(C.c_size_t)]
    lib.id_sketch.argtypes = [P, P, i64, i64, C.c_int, P, i64, P, C.c_size_t, P]
    lib.id_mlp_param_count.argtypes = []
    lib.id_mlp_param_count.restype = i64
    lib.id_mlp_forward.argtypes = [P, i64, P, P, P]
    lib.id_mlp_loss_grad.argtypes = [P, i64, P, P, P, P, P]
    lib.id_mlp_adam.argtypes = [P, P, P, P, i64, C.c_float, P]
    lib.id_rank_features.argtypes = [P, i64, i64, i64, C.c_double, P, P]
    for f in ("id_mlp_forward", "id_mlp_loss_grad", "id_mlp_adam", "id_rank_features"):
        getattr(lib, f).restype = C.c_int
    lib.id_status_string.argtypes = [C.c_int]
    lib.id_status_string.restype = C.c_char_p
    lib.id_quantize_fp8.argtypes = [P, P, i64, P, C.c_int, P]
    lib.id_fixed_rank_noalloc.argtypes = [P, i64, i64, P, P, P]
    lib.id_certificate_workspace_size.argtypes = [P, i64, i64, C.c_int, C.POINTER(C.c_size_t)]
    lib.id_certificate.argtypes = [P, P, P, i64, i64, i64, C.c_int, u64, i64, P, i64, C.POINTER(C.c_double), P,
                                   C.c_size_t, P]
    lib.id_ur_estimates.argtypes = [P, i64, i64, P, P, C.c_size_t, P, P, i64, P, P, P]
    lib.id_stable_x_workspace_size.argtypes = [P, i64, C.POINTER(C.c_size_t)]
    lib.id_stable_x.argtypes = [P, P, i64, P, i64, P, C.c_size_t, P]
    lib.cur_middle_workspace_size.argtypes = [P, i64, C.c_int, C.POINTER(C.c_size_t)]
    lib.cur_middle.argtypes = [P, P, P, i64, P, i64, C.c_int, P, C.c_size_t, P]
    lib.id_sparse_sign_rows.argtypes = [u64, i64, i64, i64, i64, i64, C.c_int, P, i64, P]
    lib.id_sparse_sketch_workspace_size.argtypes = [P, i64, i64, i64, C.POINTER(C.c_size_t)]
    lib.id_sparse_sketch.argtypes = [P, u64, i64, i64, i64, i64, P, i64, P, C.c_size_t, P]
    lib.id_selftest_timeout.argtypes = [C.c_int, P, C.c_size_t, P]
    for f in ("id_workspace_size", "id_fixed_rank", "id_adaptive", "id_batched_workspace_size",
              "id_batched", "cur_from_id", "id_gaussian_rows", "id_sketch_workspace_size", "id_sketch",
              "id_quantize_fp8", "id_fixed_rank_noalloc", "id_selftest_timeout", "id_certificate_workspace_size",
              "id_certificate", "id_ur_estimates", "id_sparse_sign_rows", "id_sparse_sketch_workspace_size",
              "id_sparse_sketch", "id_stable_x_workspace_size", "id_stable_x", "cur_middle_workspace_size",
              "cur_middle"):
        getattr(lib, f).restype = C.c_int
    # every entry point must have its C signature declared: an undeclared one would
    # pass 64-bit pointers as C ints
    protos = header_prototypes()
    for name, nargs in protos.items():
        f = getattr(lib, name)
        if f.argtypes is None or len(f.argtypes) != nargs:
            raise RuntimeError("binding declares no matching signature for %s (%d arguments)" % (name, nargs))
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions include/randid.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)


def header_prototypes() -> dict:
    """{name: number of parameters} of the functions include/randid.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = {}
    for name, params in re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(([^;{]*)\)\s*;", text, flags=re.M):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def status_string(code: int) -> str:
    return load().id_status_string(code).decode()


class IDError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s (status %d)" % (where, status_string(code), code))
        self.code = code


@dataclasses.dataclass
class IDResult:
    k: int
    J: torch.Tensor          # int64 [k], skeleton columns in pivot order
    X: torch.Tensor          # k x n, column-major view, X[:, J] = I
    est_err: float
    norm_A: float
    rounds: int
    passes: int
    launches: int
    status: int
    trace: list
    pivots: torch.Tensor | None
    phase_ms: dict
    phase_launches: dict
    cond_L1: float = 0.0     # kappa_1(L1) when x_solve_f64 was requested
    x_f64: int = 0           # 1 if X was re-solved in FP64


class IdUrStats(C.Structure):
    _fields_ = [("u_fro", C.c_double), ("u_max", C.c_double), ("est", C.c_double), ("bound", C.c_double)]


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """Return a column-major (Fortran-order) copy/view of a 2-D tensor."""
    if t.dim() != 2:
        raise ValueError("expected a matrix")
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


class FP8Matrix:
    """A stored in FP8 E4M3 with one FP32 scale per 128-row block of each column:
    data (m x n, column-major float8_e4m3fn, ld a multiple of 16), scale
    (ceil(m/128) x n, column-major float32); entry (i, j) = data[i, j] * scale[i // 128, j]."""

    def __init__(self, data: torch.Tensor, scale: torch.Tensor):
        self.data, self.scale = data, scale

    shape = property(lambda self: self.data.shape)
    dtype = property(lambda self: self.data.dtype)
    device = property(lambda self: self.data.device)
    is_cuda = property(lambda self: self.data.is_cuda)

    def stride(self, i):
        return self.data.stride(i)

    def data_ptr(self):
        return self.data.data_ptr()

    def dim(self):
        return 2


def colmajor_padded(t: torch.Tensor, multiple: int) -> torch.Tensor:
    """Column-major copy whose leading dimension is rounded up to `multiple`."""
    m, n = t.shape
    ld = -(-m // multiple) * multiple
    if t.element_size() == 1:  # 8-bit floats: move the bytes
        buf = torch.zeros((n, ld), dtype=torch.uint8, device=t.device)
        buf[:, :m] = t.view(torch.uint8).t()
        return buf.view(t.dtype)[:, :m].t()
    buf = torch.zeros((n, ld), dtype=t.dtype, device=t.device)
    buf[:, :m] = t.t()
    return buf[:, :m].t()


def quantize_fp8(A: torch.Tensor, pow2: bool = True, stream=None) -> FP8Matrix:
    """FP8 storage of A (F64/F32/BF16, column-major): E4M3 values and per-128-row
    block scales (power-of-two scales with pow2, else amax/448)."""
    m, n = A.shape
    ldq = -(-m // 16) * 16
    nbs = -(-m // 128)
    Q = torch.zeros((n, ldq), dtype=torch.uint8, device=A.device)
    S = torch.empty((n, nbs), dtype=torch.float32, device=A.device)
    rc = _call(A.device, "id_quantize_fp8", C.byref(_matrix(A)), Q.data_ptr(), ldq, S.data_ptr(),
               1 if pow2 else 0, _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "id_quantize_fp8")
    return FP8Matrix(Q.view(torch.float8_e4m3fn)[:, :m].t(), S.t())


def _matrix(A) -> IdMatrix:
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dim() != 2 or A.stride(0) != 1 or A.stride(1) < A.shape[0]:
        raise ValueError("A must be column-major (stride (1, ld >= m)); use colmajor(A)")
    if A.dtype not in _TORCH_TO_ID:
        raise ValueError("unsupported dtype %s" % A.dtype)
    scale = None
    if isinstance(A, FP8Matrix):
        sc = A.scale
        if sc.dtype != torch.float32 or sc.stride(0) != 1 or sc.stride(1) != sc.shape[0] \
                or sc.shape != (-(-A.shape[0] // 128), A.shape[1]):
            raise ValueError("FP8 block scales must be a column-major ceil(m/128) x n float32 matrix")
        scale = sc.data_ptr()
    return IdMatrix(A.data_ptr(), _TORCH_TO_ID[A.dtype], A.shape[0], A.shape[1], A.stride(1), scale)


def _opts(A, *, block, tol, relative, k_max, k0, blocks_per_pass, seed, omega, profile,
          sketch_prec=None, lu_prec=None, omega_kind=OMEGA_GAUSSIAN, zeta=0) -> IdOpts:
    dt = _TORCH_TO_ID[A.dtype]
    o = IdOpts()
    o.sketch_prec = dt if sketch_prec is None else sketch_prec
    o.lu_prec = (F64 if dt == F64 else F32) if lu_prec is None else lu_prec
    o.block = block
    o.tol = tol
    o.tol_relative = 1 if relative else 0
    o.k_max = k_max or 0
    o.k0 = k0
    o.blocks_per_pass = blocks_per_pass
    o.seed = seed & 0xFFFFFFFFFFFFFFFF
    if omega is not None:
        if not omega.is_cuda or omega.stride(1) != 1:
            raise ValueError("omega must be a row-major CUDA tensor (rows x m)")
        o.omega = omega.data_ptr()
        o.ld_omega = omega.stride(0)
        o.omega_rows = omega.shape[0]
    o.profile = 1 if profile else 0
    o.omega_kind = omega_kind
    o.zeta = zeta
    return o


def _stream(stream, device) -> int:
    """The stream handle for a call on `device`: its current stream when stream
    is None; a stream of another device is refused."""
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if stream.device != device:
        raise ValueError("the stream is on %s, the data on %s" % (stream.device, device))
    return stream.cuda_stream


def _call(device, name, *args):
    """Library function `name` called with `device` current: the library
    launches on the calling thread's current device."""
    with torch.cuda.device(device):
        return getattr(load(), name)(*args)


def _check_tensor(t, what, device, dtype, min_numel=0):
    """A contiguous tensor of `dtype` on `device` with at least min_numel entries:
    the library reads or writes that many from its first element."""
    if not isinstance(t, torch.Tensor) or t.device != device or t.dtype != dtype:
        raise ValueError("%s must be a %s tensor on %s" % (what, dtype, device))
    if not t.is_contiguous() or t.numel() < min_numel:
        raise ValueError("%s must be contiguous with at least %d entries" % (what, min_numel))


def _check_out(J, Xb, n, kmax, xdt, device, what):
    """Caller-owned outputs of an ID with rank cap kmax: J holds kmax int64 and Xb
    is X^T, an (>= n) x (>= kmax) row-major buffer (Xb[j, c] = X(c, j), row stride
    >= kmax).  The library writes J[0:k] and X(0:k, 0:n) with k <= kmax, so
    anything smaller is refused before any device write."""
    _check_tensor(J, what + ": J", device, torch.int64, kmax)
    if (not isinstance(Xb, torch.Tensor) or Xb.device != device or Xb.dtype != xdt or Xb.dim() != 2
            or Xb.shape[0] < n or Xb.shape[1] < kmax or Xb.stride(1) != 1 or Xb.stride(0) < kmax):
        raise ValueError("%s: X must be a %s tensor on %s of shape (>= %d, >= %d) with stride (>= %d, 1)"
                         % (what, xdt, device, n, kmax, kmax))


def workspace_size(A: torch.Tensor, opts: IdOpts, l: int = 0) -> int:
    n = C.c_size_t(0)
    rc = _call(A.device, "id_workspace_size", C.byref(_matrix(A)), C.byref(opts), l, C.byref(n))
    if rc != 0:
        raise IDError(rc, "id_workspace_size")
    return int(n.value)


def _workspace(nbytes: int, device, ws: torch.Tensor | None) -> torch.Tensor:
    if (ws is not None and ws.dtype == torch.uint8 and ws.is_contiguous() and ws.numel() >= nbytes
            and ws.device == device):
        return ws
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def _result(res: IdResult, J, Xbuf, k, n, status, trace_buf, piv) -> IDResult:
    X = Xbuf.t()[:k]
    trace = list(trace_buf[: min(res.rounds, len(trace_buf))]) if trace_buf is not None else []
    return IDResult(k=k, J=J[:k], X=X, est_err=res.est_err, norm_A=res.norm_A, rounds=res.rounds,
                    passes=res.passes, launches=res.launches, status=status, trace=trace,
                    pivots=None if piv is None else piv[:k],
                    phase_ms={PHASES[i]: res.phase_ms[i] for i in range(6)},
                    phase_launches={PHASES[i]: int(res.phase_launches[i]) for i in range(6)},
                    cond_L1=res.cond_L1, x_f64=int(res.x_f64))


def id_fixed_rank(A: torch.Tensor, k: int, l: int, *, block: int = 64, seed: int = 0,
                  omega: torch.Tensor | None = None, profile: bool = False, pivots: bool = False,
                  stream=None, workspace: torch.Tensor | None = None,
                  sketch_prec: int | None = None, x_solve_f64: int = 0, omega_kind: int = OMEGA_GAUSSIAN,
                  zeta: int = 0) -> IDResult:
    """randLUPP fixed-rank column ID (Sec. 3.1): J (k), X (k x n), estimate from l - k rows.
    sketch_prec=F64_EMU (FP64 A only): the sketch on the tensor cores by digit slicing.
    omega_kind=OMEGA_SPARSE_SIGN: the generated sketching matrix is sparse sign (Sec. 5.1)."""
    m, n = A.shape
    opts = _opts(A, block=block, tol=0.0, relative=False, k_max=k, k0=0, blocks_per_pass=1,
                 seed=seed, omega=omega, profile=profile, sketch_prec=sketch_prec, omega_kind=omega_kind,
                 zeta=zeta)
    opts.x_solve_f64 = x_solve_f64
    ws = _workspace(workspace_size(A, opts, l), A.device, workspace)
    J = torch.empty(k, dtype=torch.int64, device=A.device)
    Xbuf = torch.empty((n, k), dtype=torch.float64 if opts.lu_prec == F64 else torch.float32,
                       device=A.device)
    piv = torch.empty(k, dtype=torch.float64, device=A.device) if pivots else None
    res = IdResult()
    res.J, res.X, res.ldx = J.data_ptr(), Xbuf.data_ptr(), k
    res.pivots = piv.data_ptr() if piv is not None else None
    rc = _call(A.device, "id_fixed_rank", C.byref(_matrix(A)), k, l, C.byref(opts), ws.data_ptr(), ws.numel(),
               C.byref(res), _stream(stream, A.device))
    if rc < 0:
        raise IDError(rc, "id_fixed_rank")
    return _result(res, J, Xbuf, k, n, rc, None, piv)


def id_adaptive(A: torch.Tensor, tol: float, *, block: int = 64, relative: bool = True,
                k_max: int | None = None, k0: int = 0, blocks_per_pass: int = 0, seed: int = 0,
                omega: torch.Tensor | None = None, profile: bool = False, pivots: bool = False,
                trace_cap: int = 4096, stream=None, workspace: torch.Tensor | None = None,
                out: tuple | None = None, predictor: torch.Tensor | None = None,
                max_pass_rows: int = 0, sketch_prec: int | None = None, x_solve_f64: int = 0,
                omega_kind: int = OMEGA_GAUSSIAN, zeta: int = 0) -> IDResult:
    """randLUPPadap column ID (Algorithm 1).  `out` = (J, Xbuf) reuses output buffers
    (J int64 [k_max], Xbuf (n, k_max) row-major == X column-major).  `predictor`:
    FP32 CUDA tensor of id_mlp_param_count() parameters; it sets how many blocks
    the second pass over A sketches (results are those of the plain loop).
    sketch_prec=F64_EMU (FP64 A only): the sketch, Schur GEMM and block update on the
    tensor cores by exact digit slicing, FP64 accurate, with Omega on the grid 2^-11.
    sketch_prec=F32_EMU (FP32 A only): the sketch on the tensor cores in 3 digits per
    operand, FP32 accurate."""
    m, n = A.shape
    kmax = min(m, n) if not k_max else min(k_max, m, n)
    opts = _opts(A, block=block, tol=tol, relative=relative, k_max=kmax, k0=k0,
                 blocks_per_pass=blocks_per_pass, seed=seed, omega=omega, profile=profile,
                 sketch_prec=sketch_prec, omega_kind=omega_kind, zeta=zeta)
    opts.x_solve_f64 = x_solve_f64
    if predictor is not None:
        if not predictor.is_cuda or predictor.dtype != torch.float32 or predictor.numel() != mlp_param_count():
            raise ValueError("predictor must be a CUDA float32 tensor of id_mlp_param_count() values")
        opts.predictor = predictor.data_ptr()
        opts.max_pass_rows = max_pass_rows
    ws = _workspace(workspace_size(A, opts, 0), A.device, workspace)
    xdt = torch.float64 if opts.lu_prec == F64 else torch.float32
    if out is None:
        J = torch.empty(kmax, dtype=torch.int64, device=A.device)
        Xbuf = torch.empty((n, kmax), dtype=xdt, device=A.device)
    else:
        J, Xbuf = out
        _check_out(J, Xbuf, n, kmax, xdt, A.device, "id_adaptive out")
    piv = torch.empty(kmax, dtype=torch.float64, device=A.device) if pivots else None
    trace_buf = (C.c_double * trace_cap)() if trace_cap > 0 else None
    res = IdResult()
    res.J, res.X, res.ldx = J.data_ptr(), Xbuf.data_ptr(), Xbuf.stride(0)
    res.pivots = piv.data_ptr() if piv is not None else None
    res.est_trace = C.cast(trace_buf, C.c_void_p) if trace_buf is not None else None
    res.trace_cap = trace_cap
    rc = _call(A.device, "id_adaptive", C.byref(_matrix(A)), C.byref(opts), ws.data_ptr(), ws.numel(),
               C.byref(res), _stream(stream, A.device))
    if rc < 0:
        raise IDError(rc, "id_adaptive")
    return _result(res, J, Xbuf, int(res.k), n, rc, trace_buf, piv)


def gaussian_rows(seed: int, row0: int, rows: int, m: int, dtype=torch.float64,
                  device="cuda", stream=None, grid: bool = False) -> torch.Tensor:
    """Rows [row0, row0+rows) of the Philox/Box-Muller sketching matrix (rows x m).
    grid=True (dtype float64): the rows the FP64-accurate sketch uses, rounded to
    the grid 2^-11 by that path's own generator."""
    if dtype not in _TORCH_TO_ID:
        raise ValueError("unsupported dtype %s" % dtype)
    if grid and dtype != torch.float64:
        raise ValueError("grid rows are FP64")
    out = torch.empty((rows, m), dtype=dtype, device=device)
    code = F64_EMU if grid else _TORCH_TO_ID[dtype]
    rc = _call(out.device, "id_gaussian_rows", seed & 0xFFFFFFFFFFFFFFFF, row0, rows, m, code,
               out.data_ptr(), m, _stream(stream, out.device))
    if rc != 0:
        raise IDError(rc, "id_gaussian_rows")
    return out


def id_sketch(A: torch.Tensor, omega: torch.Tensor, *, stream=None,
              workspace: torch.Tensor | None = None, sketch_prec: int | None = None) -> torch.Tensor:
    """G = (omega A)^T (n x rows): the sketch step alone.  omega is row-major
    (rows x m) in A's dtype; G is FP64 for FP64 input and FP32 otherwise (BF16
    input runs on the tensor cores).  sketch_prec=F64_EMU (FP64 A): the product
    of omega rounded to the grid 2^-11 and A, FP64 accurate, on the tensor cores."""
    m, n = A.shape
    if (omega.dim() != 2 or omega.shape[1] != m or omega.stride(1) != 1 or omega.dtype != A.dtype
            or omega.device != A.device):
        raise ValueError("omega must be row-major (rows x m) with A's dtype, on A's device")
    rows = omega.shape[0]
    prec = _TORCH_TO_ID[A.dtype] if sketch_prec is None else sketch_prec
    nb = C.c_size_t(0)
    rc = _call(A.device, "id_sketch_workspace_size", C.byref(_matrix(A)), rows, prec, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_sketch_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    G = torch.empty((n, rows), dtype=torch.float64 if A.dtype == torch.float64 else torch.float32,
                    device=A.device)
    rc = _call(A.device, "id_sketch", C.byref(_matrix(A)), omega.data_ptr(), omega.stride(0), rows, prec,
               G.data_ptr(), G.stride(0), ws.data_ptr(), ws.numel(), _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "id_sketch")
    return G


def id_batched(As: list, tol: float, *, block: int = 32, relative: bool = True, k_max: int | None = None,
               seed: int = 0, pivots: bool = False, stream=None,
               workspace: torch.Tensor | None = None, outs: list | None = None) -> list:
    """Adaptive column IDs of many independent matrices in one persistent launch.
    As: column-major CUDA tensors of one dtype (FP64 or FP32), n <= 4096 each.
    Returns one IDResult per matrix (per-problem status in .status)."""
    if not As:
        return []
    dev = As[0].device
    if any(a.device != dev for a in As):
        raise ValueError("id_batched: every matrix must be on one device")
    if outs is not None and len(outs) != len(As):
        raise ValueError("id_batched: outs needs one (J, X) pair per matrix")
    dt = _TORCH_TO_ID[As[0].dtype]
    count = len(As)
    mats = (IdMatrix * count)(*[_matrix(a) for a in As])
    opts = _opts(As[0], block=block, tol=tol, relative=relative, k_max=k_max or 0, k0=0,
                 blocks_per_pass=1, seed=seed, omega=None, profile=False)
    nb = C.c_size_t(0)
    rc = _call(dev, "id_batched_workspace_size", count, mats, C.byref(opts), C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_batched_workspace_size")
    ws = _workspace(int(nb.value), As[0].device, workspace)
    xdt = torch.float64 if dt == F64 else torch.float32
    res = (IdResult * count)()
    keep = []
    for i, a in enumerate(As):
        m, n = a.shape
        kmax = min(m, n) if not k_max else min(k_max, m, n)
        if outs is not None:
            J, Xb = outs[i]
            _check_out(J, Xb, n, kmax, xdt, dev, "id_batched outs[%d]" % i)
        else:
            J = torch.empty(kmax, dtype=torch.int64, device=a.device)
            Xb = torch.empty((n, kmax), dtype=xdt, device=a.device)
        piv = torch.empty(kmax, dtype=torch.float64, device=a.device) if pivots else None
        res[i].J, res[i].X, res[i].ldx = J.data_ptr(), Xb.data_ptr(), Xb.stride(0)
        res[i].pivots = piv.data_ptr() if piv is not None else None
        keep.append((J, Xb, piv))
    rc = _call(dev, "id_batched", count, mats, C.byref(opts), ws.data_ptr(), ws.numel(), res, _stream(stream, dev))
    if rc < 0 and rc != ERR_NONFINITE:
        raise IDError(rc, "id_batched")
    out = []
    for i in range(count):
        J, Xb, piv = keep[i]
        r = res[i]
        k = int(r.k)
        st = int(r.status)
        out.append(IDResult(k=k, J=J[:k], X=Xb.t()[:k], est_err=r.est_err, norm_A=r.norm_A,
                            rounds=r.rounds, passes=r.passes, launches=r.launches, status=st, trace=[],
                            pivots=None if piv is None else piv[:k], phase_ms={}, phase_launches={}))
    return out


def selftest_timeout(which: int, device="cuda", stream=None) -> int:
    """Run one device wait that nothing satisfies (0: the LUPP panel's grid
    barrier, 1: an mbarrier wait of the tensor-core kernels) and return the
    library's status: ERR_TIMEOUT when the bounded wait gave up as designed."""
    ws = torch.empty(256, dtype=torch.uint8, device=device)
    return _call(ws.device, "id_selftest_timeout", which, ws.data_ptr(), ws.numel(), _stream(stream, ws.device))


# ---------------------------------------------------------------- learned rank predictor
MLP_IN, MLP_HIDDEN = 35, 128
MLP_TRAINABLE = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1


def mlp_param_count() -> int:
    return int(load().id_mlp_param_count())


def _check_mlp(params, x):
    """The parameter block (id_mlp_param_count() FP32 values) and a feature
    matrix (batch x 35, FP32) on one device."""
    _check_tensor(params, "params", x.device, torch.float32, mlp_param_count())
    if x.dim() != 2 or x.shape[1] != MLP_IN or x.shape[0] < 1:
        raise ValueError("x must be batch x %d" % MLP_IN)
    _check_tensor(x, "x", x.device, torch.float32)


def mlp_forward(params: torch.Tensor, x: torch.Tensor, stream=None) -> torch.Tensor:
    """Predicted log2 rank for each feature row of x (batch x 35, FP32, CUDA)."""
    x = x.contiguous()
    _check_mlp(params, x)
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    rc = _call(x.device, "id_mlp_forward", params.data_ptr(), x.shape[0], x.data_ptr(), y.data_ptr(),
               _stream(stream, x.device))
    if rc != 0:
        raise IDError(rc, "id_mlp_forward")
    return y


def mlp_loss_grad(params: torch.Tensor, x: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
                  stream=None):
    """(loss, grad): mean squared error on the standardised output and its gradient
    with respect to the trainable parameters."""
    x = x.contiguous()
    target = target.contiguous()
    _check_mlp(params, x)
    _check_tensor(target, "target", x.device, torch.float32, x.shape[0])
    if grad is None:
        grad = torch.empty(MLP_TRAINABLE, dtype=torch.float32, device=x.device)
    _check_tensor(grad, "grad", x.device, torch.float32, MLP_TRAINABLE)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    rc = _call(x.device, "id_mlp_loss_grad", params.data_ptr(), x.shape[0], x.data_ptr(), target.data_ptr(),
               grad.data_ptr(), loss.data_ptr(), _stream(stream, x.device))
    if rc != 0:
        raise IDError(rc, "id_mlp_loss_grad")
    return loss, grad


def mlp_adam(params: torch.Tensor, grad: torch.Tensor, m1: torch.Tensor, m2: torch.Tensor, step: int,
             lr: float, stream=None) -> None:
    dev = params.device
    _check_tensor(params, "params", dev, torch.float32, mlp_param_count())
    for t, what in ((grad, "grad"), (m1, "m1"), (m2, "m2")):
        _check_tensor(t, what, dev, torch.float32, MLP_TRAINABLE)
    rc = _call(dev, "id_mlp_adam", params.data_ptr(), grad.data_ptr(), m1.data_ptr(), m2.data_ptr(), step, lr,
               _stream(stream, dev))
    if rc != 0:
        raise IDError(rc, "id_mlp_adam")


def rank_features(pivots: torch.Tensor, m: int, n: int, rel_tol: float, stream=None) -> torch.Tensor:
    """The 35 predictor features from the first pivots |U(i,i)| (CUDA float64)."""
    _check_tensor(pivots, "pivots", pivots.device, torch.float64)
    x = torch.empty(MLP_IN, dtype=torch.float32, device=pivots.device)
    rc = _call(pivots.device, "id_rank_features", pivots.data_ptr(), pivots.numel(), m, n, rel_tol, x.data_ptr(),
               _stream(stream, pivots.device))
    if rc != 0:
        raise IDError(rc, "id_rank_features")
    return x


def cur_from_id(A: torch.Tensor, J: torch.Tensor, *, stream=None,
                workspace: torch.Tensor | None = None):
    """Row skeletons I and the row interpolation matrix W (m x k) of C = A(:, J):
    A ~ W A(I, J) X (two-sided ID).  Returns (I, W)."""
    m, n = A.shape
    k = J.numel()
    nb = C.c_size_t(0)
    rc = _call(A.device, "id_cur_workspace_size", C.byref(_matrix(A)), k, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_cur_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    I = torch.empty(k, dtype=torch.int64, device=A.device)
    W = torch.empty((k, m), dtype=A.dtype, device=A.device).t()  # column-major m x k
    J = J.to(device=A.device, dtype=torch.int64).contiguous()
    rc = _call(A.device, "cur_from_id", C.byref(_matrix(A)), J.data_ptr(), k, I.data_ptr(), W.data_ptr(),
               W.stride(1), ws.data_ptr(), ws.numel(), _stream(stream, A.device))
    if rc < 0:
        raise IDError(rc, "cur_from_id")
    return I, W


# ---------------------------------------------------------------- after the ID
def certificate(A, J: torch.Tensor, X: torch.Tensor, q: int, *, seed: int = 0, row0: int = 0,
                omega: torch.Tensor | None = None, sketch_prec: int | None = None, stream=None,
                workspace: torch.Tensor | None = None) -> float:
    """A-posteriori estimate ||Omega' A - (Omega' A)(:,J) X||_F / sqrt(q) of a column
    ID's error from q fresh Gaussian rows (rows [row0, row0+q) of the generator
    `seed`, or the caller's omega, q x m row-major in the sketch's input type).
    X: k x n (column-major, e.g. an IDResult's X), FP64 for FP64 A, else FP32."""
    m, n = A.shape
    k = J.numel()
    prec = _TORCH_TO_ID[A.dtype] if sketch_prec is None else sketch_prec
    xdt = torch.float64 if A.dtype == torch.float64 else torch.float32
    if (X.dim() != 2 or X.shape[0] != k or X.shape[1] != n or X.dtype != xdt or X.device != A.device
            or X.stride(0) != 1 or X.stride(1) < k):
        raise ValueError("X must be a column-major %s (%d x %d) on %s" % (xdt, k, n, A.device))
    _check_tensor(J, "J", A.device, torch.int64, k)
    ld_om = 0
    om_ptr = None
    if omega is not None:
        if omega.device != A.device or omega.dim() != 2 or omega.shape != (q, m) or omega.stride(1) != 1:
            raise ValueError("omega must be a row-major q x m tensor on A's device")
        om_ptr, ld_om = omega.data_ptr(), omega.stride(0)
    nb = C.c_size_t(0)
    rc = _call(A.device, "id_certificate_workspace_size", C.byref(_matrix(A)), k, q, prec, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_certificate_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    est = C.c_double(0.0)
    rc = _call(A.device, "id_certificate", C.byref(_matrix(A)), J.data_ptr(), X.data_ptr(), X.stride(1), k, q, prec,
               seed & 0xFFFFFFFFFFFFFFFF, row0, om_ptr, ld_om, C.byref(est), ws.data_ptr(), ws.numel(),
               _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "id_certificate")
    return float(est.value)


@dataclasses.dataclass
class URResult:
    id: IDResult             # the rank-k fixed-rank ID
    U_r: torch.Tensor        # p x p (upper triangular), lu precision
    J_extra: torch.Tensor    # int64 [p], the columns the p extra pivots pick
    u_fro: float             # ||U_r||_F
    u_max: float             # max |U_r(i,j)|
    est: float               # ||L_r U_r||_F / sqrt(p)
    bound: float             # sqrt(n - k) ||U_r||_F


def ur_estimates(A, k: int, p: int, *, block: int = 64, seed: int = 0, omega: torch.Tensor | None = None,
                 sketch_prec: int | None = None, stream=None, workspace: torch.Tensor | None = None) -> URResult:
    """Remark 1: the rank-k ID from k + p sketch rows and the trailing p x p block U_r
    of the LUPP continued for p more steps."""
    m, n = A.shape
    opts = _opts(A, block=block, tol=0.0, relative=False, k_max=k, k0=0, blocks_per_pass=1, seed=seed,
                 omega=omega, profile=False, sketch_prec=sketch_prec)
    ws = _workspace(workspace_size(A, opts, k + p), A.device, workspace)
    xdt = torch.float64 if opts.lu_prec == F64 else torch.float32
    J = torch.empty(k, dtype=torch.int64, device=A.device)
    Xbuf = torch.empty((n, k), dtype=xdt, device=A.device)
    U = torch.zeros((p, p), dtype=xdt, device=A.device)  # column-major: U[j, c] = U_r(c, j)
    Jx = torch.empty(p, dtype=torch.int64, device=A.device)
    res = IdResult()
    res.J, res.X, res.ldx = J.data_ptr(), Xbuf.data_ptr(), k
    stats = IdUrStats()
    rc = _call(A.device, "id_ur_estimates", C.byref(_matrix(A)), k, p, C.byref(opts), ws.data_ptr(), ws.numel(),
               C.byref(res), U.data_ptr(), p, Jx.data_ptr(), C.byref(stats), _stream(stream, A.device))
    if rc < 0:
        raise IDError(rc, "id_ur_estimates")
    return URResult(id=_result(res, J, Xbuf, k, n, rc, None, None), U_r=U.t(), J_extra=Jx, u_fro=stats.u_fro,
                    u_max=stats.u_max, est=stats.est, bound=stats.bound)


# ---------------------------------------------------------------- sparse sign
def sparse_sign_rows(seed: int, t0: int, blocks: int, b: int, m: int, zeta: int = 8, dtype=torch.float64,
                     device="cuda", stream=None) -> torch.Tensor:
    """Blocks t0 .. t0+blocks-1 of the sparse-sign sketching matrix as dense rows
    ((blocks*b) x m): zeta entries +-sqrt(b/zeta) per column of each block."""
    if dtype not in (torch.float64, torch.float32):
        raise ValueError("sparse_sign_rows: dtype float64 or float32")
    out = torch.empty((blocks * b, m), dtype=dtype, device=device)
    rc = _call(out.device, "id_sparse_sign_rows", seed & 0xFFFFFFFFFFFFFFFF, t0, blocks, b, m, zeta,
               _TORCH_TO_ID[dtype], out.data_ptr(), m, _stream(stream, out.device))
    if rc != 0:
        raise IDError(rc, "id_sparse_sign_rows")
    return out


def sparse_sketch(A, rows: int, b: int, *, seed: int = 0, t0: int = 0, zeta: int = 8, stream=None,
                  workspace: torch.Tensor | None = None) -> torch.Tensor:
    """G = (Omega A)^T (n x rows) for rows [t0*b, t0*b + rows) of the sparse-sign matrix:
    the gather-add sketch alone (FP64 for FP64 A, FP32 for FP32 and BF16 A)."""
    m, n = A.shape
    nb = C.c_size_t(0)
    rc = _call(A.device, "id_sparse_sketch_workspace_size", C.byref(_matrix(A)), rows, b, zeta, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_sparse_sketch_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    G = torch.empty((n, rows), dtype=torch.float64 if A.dtype == torch.float64 else torch.float32, device=A.device)
    rc = _call(A.device, "id_sparse_sketch", C.byref(_matrix(A)), seed & 0xFFFFFFFFFFFFFFFF, t0, rows, b, zeta,
               G.data_ptr(), G.stride(0), ws.data_ptr(), ws.numel(), _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "id_sparse_sketch")
    return G


# ---------------------------------------------------------------- stable X and CUR
def stable_x(A, J: torch.Tensor, *, stream=None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """X = A(:,J)^+ A (k x n, column-major view), by a Householder QR of A(:,J) on
    the device: the stable interpolation matrix (Eq. sID in column form)."""
    m, n = A.shape
    k = J.numel()
    _check_tensor(J, "J", A.device, torch.int64, k)
    nb = C.c_size_t(0)
    rc = _call(A.device, "id_stable_x_workspace_size", C.byref(_matrix(A)), k, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "id_stable_x_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    Xb = torch.empty((n, k), dtype=A.dtype, device=A.device)  # X column-major, ld k
    rc = _call(A.device, "id_stable_x", C.byref(_matrix(A)), J.data_ptr(), k, Xb.data_ptr(), k, ws.data_ptr(),
               ws.numel(), _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "id_stable_x")
    return Xb.t()


def cur_middle(A, I: torch.Tensor, J: torch.Tensor, kind: int = CUR_PSEUDOINVERSE, *, stream=None,
               workspace: torch.Tensor | None = None) -> torch.Tensor:
    """The k x k middle factor: C^+ A R^+ (CUR_PSEUDOINVERSE, C = A(:,J), R = A(I,:))
    or A(I,J)^{-1} (CUR_INVERSE).  Returns U (column-major view)."""
    k = J.numel()
    if I.numel() != k:
        raise ValueError("I and J need the same length")
    _check_tensor(I, "I", A.device, torch.int64, k)
    _check_tensor(J, "J", A.device, torch.int64, k)
    nb = C.c_size_t(0)
    rc = _call(A.device, "cur_middle_workspace_size", C.byref(_matrix(A)), k, kind, C.byref(nb))
    if rc != 0:
        raise IDError(rc, "cur_middle_workspace_size")
    ws = _workspace(int(nb.value), A.device, workspace)
    Ub = torch.empty((k, k), dtype=A.dtype, device=A.device)  # U column-major, ld k
    rc = _call(A.device, "cur_middle", C.byref(_matrix(A)), I.data_ptr(), J.data_ptr(), k, Ub.data_ptr(), k, kind,
               ws.data_ptr(), ws.numel(), _stream(stream, A.device))
    if rc != 0:
        raise IDError(rc, "cur_middle")
    return Ub.t()
