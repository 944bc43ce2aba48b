"""FP64 CPU oracle for the randomized column ID of arXiv:2310.09417.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It wraps ``oracle.c`` (plain C, FP64, OpenMP over independent
columns) with ctypes and numpy; it shares no code with the GPU library.

Every function follows the paper step by step; see ``oracle.h`` for the
conventions (column ID orientation, tie rule, Gaussian generator, the
variance reading of the estimator's scale).

Every function is pinned by ``tests/test_oracle_pins.py`` or
``tests/test_oracle_mlp.py``.  The factor (4 log k / k) sqrt(n-k) that Eq.
normUest and Eq. maxUest put in front of ||U_r||_F and max|U_r| is not
computed here: the paper supports it only with a figure, so nothing pins it
(see ``ur_estimates``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

OK, TOL_NOT_MET, BAD_ARG, NONFINITE = 0, 1, -1, -2


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    i64, f64p, i64p = C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    u64p = C.POINTER(C.c_uint64)
    lib.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
    lib.orc_philox4x64_10.restype = None
    lib.orc_gaussian_rows.argtypes = [C.c_uint64, i64, i64, i64, f64p]
    lib.orc_gaussian_rows.restype = None
    lib.orc_sketch_t.argtypes = [i64, i64, f64p, i64, i64, f64p, f64p]
    lib.orc_sketch_t.restype = None
    lib.orc_lupp.argtypes = [i64, i64, i64, f64p, i64, i64p]
    lib.orc_lupp.restype = i64
    lib.orc_id_fixed_rank.argtypes = [i64, i64, f64p, i64, i64, f64p, i64, i64p, f64p, i64,
                                      f64p, f64p]
    lib.orc_id_fixed_rank.restype = C.c_int
    lib.orc_id_adaptive.argtypes = [i64, i64, f64p, i64, i64, C.c_double, i64, f64p, i64,
                                    i64p, i64p, f64p, i64, f64p, i64, i64p, f64p]
    lib.orc_id_adaptive.restype = C.c_int
    lib.orc_sparse_sign_block.argtypes = [C.c_uint64, i64, i64, i64, i64, f64p]
    lib.orc_sparse_sign_block.restype = None
    lib.orc_fro_norm.argtypes = [i64, i64, f64p, i64]
    lib.orc_fro_norm.restype = C.c_double
    lib.orc_id_residual.argtypes = [i64, i64, f64p, i64, i64, i64p, f64p, i64]
    lib.orc_id_residual.restype = C.c_double
    lib.orc_stable_residual.argtypes = [i64, i64, f64p, i64, i64, i64p]
    lib.orc_stable_residual.restype = C.c_double
    _lib = lib
    return lib


def _f64(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _colmajor(A):
    """Return A as a Fortran-ordered float64 array (the oracle's layout)."""
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def philox4x64_10(ctr, key):
    """Philox4x64-10 block function on one 256-bit counter (Salmon et al. 2011)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    P = C.POINTER(C.c_uint64)
    lib.orc_philox4x64_10(c.ctypes.data_as(P), k.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def gaussian_rows(seed: int, row0: int, rows: int, m: int) -> np.ndarray:
    """Rows [row0, row0+rows) of the N(0,1) sketching matrix, shape (rows, m)."""
    out = np.zeros((rows, m), dtype=np.float64)
    _load().orc_gaussian_rows(C.c_uint64(seed), row0, rows, m, _f64(out))
    return out


def sparse_sign_rows(seed: int, t0: int, blocks: int, b: int, m: int, zeta: int = 8) -> np.ndarray:
    """Blocks t0 .. t0+blocks-1 of the sparse-sign sketching matrix (Sec. 5.1,
    "Sparse Sign"; zeta = 8 as the paper chooses), stacked: (blocks*b) x m.
    Each column of each block holds zeta entries +-sqrt(b/zeta) at distinct
    rows (the counter-based definition is in oracle.h)."""
    if not (1 <= zeta <= b):
        raise ValueError("sparse sign needs 1 <= zeta <= b")
    out = np.zeros((blocks * b, m), dtype=np.float64)
    for q in range(blocks):
        blk = np.zeros((b, m), dtype=np.float64)
        _load().orc_sparse_sign_block(C.c_uint64(seed), t0 + q, b, m, zeta, _f64(blk))
        out[q * b:(q + 1) * b] = blk
    return out


def sketch_t(A, Omega) -> np.ndarray:
    """Y^T = (Omega A)^T, shape (n, rows)."""
    A = _colmajor(A)
    m, n = A.shape
    Om = np.ascontiguousarray(Omega, dtype=np.float64)
    assert Om.shape[1] == m
    YT = np.zeros((n, Om.shape[0]), dtype=np.float64, order="F")
    _load().orc_sketch_t(m, n, _f64(A), m, Om.shape[0], _f64(Om), _f64(YT))
    return YT


def lupp(M, steps=None, labels=None):
    """LU with partial pivoting of M (nr x nc) for `steps` steps.

    Returns (LU, perm, zero_pivots): LU holds L strictly below the diagonal of
    the first `steps` columns and U / the Schur complement elsewhere; perm[i] is
    the label of the row now at position i (labels default to 0..nr-1).
    """
    M = np.array(M, dtype=np.float64, order="F", copy=True)
    nr, nc = M.shape
    if steps is None:
        steps = min(nr, nc)
    orig = np.arange(nr, dtype=np.int64) if labels is None else np.array(labels, dtype=np.int64)
    z = _load().orc_lupp(nr, nc, steps, _f64(M), nr, _i64(orig))
    return M, orig, int(z)


def id_fixed_rank(A, Omega, k: int):
    """randLUPP column ID.  Returns dict(J, X (k x n), est, pivots, status)."""
    A = _colmajor(A)
    m, n = A.shape
    Om = np.ascontiguousarray(Omega, dtype=np.float64)
    l = Om.shape[0]
    J = np.zeros(k, dtype=np.int64)
    X = np.zeros((k, n), dtype=np.float64, order="F")
    est = np.zeros(1)
    piv = np.zeros(k)
    st = _load().orc_id_fixed_rank(m, n, _f64(A), m, l, _f64(Om), k, _i64(J), _f64(X), k,
                                   _f64(est), _f64(piv))
    if st < 0:
        raise ValueError("oracle id_fixed_rank failed with status %d" % st)
    return dict(J=J, X=X, est=float(est[0]), pivots=piv, status=st)


def id_adaptive(A, Omega, b: int, tol: float, kmax: int | None = None):
    """randLUPPadap column ID (Algorithm 1) with absolute tolerance `tol`.

    Omega must hold every row the run can draw: at least (ceil(kmax/b)+1)*b rows.
    Returns dict(k, J, X (k x n), trace, rounds, pivots, status).
    """
    A = _colmajor(A)
    m, n = A.shape
    if kmax is None:
        kmax = min(m, n)
    Om = np.ascontiguousarray(Omega, dtype=np.float64)
    assert Om.shape[1] == m
    J = np.zeros(kmax, dtype=np.int64)
    X = np.zeros((kmax, n), dtype=np.float64, order="F")
    tcap = kmax // max(b, 1) + 2
    trace = np.zeros(tcap)
    piv = np.zeros(kmax)
    k = np.zeros(1, dtype=np.int64)
    rounds = np.zeros(1, dtype=np.int64)
    st = _load().orc_id_adaptive(m, n, _f64(A), m, b, float(tol), kmax, _f64(Om), Om.shape[0],
                                 _i64(k), _i64(J), _f64(X), kmax, _f64(trace), tcap,
                                 _i64(rounds), _f64(piv))
    if st < 0:
        raise ValueError("oracle id_adaptive failed with status %d" % st)
    kk = int(k[0])
    r = int(rounds[0])
    return dict(k=kk, J=J[:kk].copy(), X=np.asfortranarray(X[:kk]), trace=trace[:r].copy(),
                rounds=r, pivots=piv[:kk].copy(), status=st)


def fro_norm(A) -> float:
    A = _colmajor(A)
    return float(_load().orc_fro_norm(A.shape[0], A.shape[1], _f64(A), A.shape[0]))


def id_residual(A, J, X) -> float:
    """||A - A(:,J) X||_F."""
    A = _colmajor(A)
    J = np.ascontiguousarray(J, dtype=np.int64)
    X = np.asfortranarray(np.asarray(X, dtype=np.float64))
    k = len(J)
    return float(_load().orc_id_residual(A.shape[0], A.shape[1], _f64(A), A.shape[0], k,
                                         _i64(J), _f64(X), X.shape[0]))


def stable_residual(A, J) -> float:
    """||A - Q Q^T A||_F with Q from Householder QR of A(:,J)."""
    A = _colmajor(A)
    J = np.ascontiguousarray(J, dtype=np.int64)
    return float(_load().orc_stable_residual(A.shape[0], A.shape[1], _f64(A), A.shape[0],
                                             len(J), _i64(J)))


def stable_x(A, J) -> np.ndarray:
    """The stable interpolation matrix of the column ID: X = A(:,J)^+ A, the
    orthogonal projection onto the skeleton columns (column form of Eq. sID,
    Sec. 2.2), through a Householder QR of A(:,J): X = R^{-1} Q^T A.  Returns
    X (k x n); X(:,J) = I up to rounding, and ||A - A(:,J) X||_F is the stable
    ID error."""
    import scipy.linalg as sla

    A = _colmajor(A)
    J = np.asarray(J, dtype=np.int64)
    Q, R = np.linalg.qr(A[:, J], mode="reduced")  # library QR: a step, as the paper's qr
    return sla.solve_triangular(R, Q.T @ A, lower=False)


def ur_estimates(A, Omega, k: int) -> dict:
    """The residual block U_r of Remark 1 (Sec. 3.2), in column form.

    Omega has k + p rows: the first k give the rank-k skeleton, the last p are
    the independent sample set aside for the estimate.  LUPP of the transposed
    sketch Y^T = (Omega A)^T (n x (k+p)) continued for all k + p steps gives
    P Y^T = [L1; L2 L_r] [U1 U2; 0 U_r] with U_r the trailing p x p block.
    Returns U_r, L_r ((n-k) x p, unit lower trapezoidal), the Schur estimate
    E = ||L_r U_r||_F / sqrt(p) (Eq. errSch), the bound sqrt(n-k) ||U_r||_F,
    and the two norms Eq. normUest and Eq. maxUest are built from:
    u_fro = ||U_r||_F and u_max = max |U_r(i,j)|.  The paper multiplies them by
    (4 log k / k) sqrt(n-k) (the reciprocal of the growth-factor bound
    k / (4 log k) it borrows); that factor has no support but a figure the text
    does not carry, so it is left to the caller and nothing here depends on it."""
    A = _colmajor(A)
    n = A.shape[1]
    l = Omega.shape[0]
    p = l - k
    if not (1 <= k and 1 <= p and l <= n):
        raise ValueError("ur_estimates needs k >= 1, at least one extra row and k + p <= n")
    LU, perm, _ = lupp(sketch_t(A, Omega), steps=l)
    U_r = np.triu(LU[k:l, k:l])
    L_r = np.tril(LU[k:, k:l], -1) + np.eye(n - k, p)
    nrm, mx = float(np.linalg.norm(U_r)), float(np.abs(U_r).max())
    return dict(U_r=U_r, L_r=L_r, perm=perm, est=float(np.linalg.norm(L_r @ U_r)) / np.sqrt(p),
                bound=np.sqrt(n - k) * nrm, u_fro=nrm, u_max=mx)


def certificate(A, J, X, Omega_post) -> float:
    """An a-posteriori estimate of ||A - A(:,J) X||_F from a fresh Gaussian
    sample Omega_post (q x m) drawn after the skeletons are chosen (the
    certificate Remark 1 points to): ||Omega' A - (Omega' A)(:,J) X||_F / sqrt(q),
    whose square is unbiased for the squared error (Sec. 4.2)."""
    G = sketch_t(A, Omega_post)  # n x q: row j is the sample of column j
    J = np.asarray(J, dtype=np.int64)
    R = G.T - G[J].T @ np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(R)) / np.sqrt(G.shape[1])


def row_id_of_columns(A, J) -> tuple:
    """Row skeletons I and row interpolation matrix W of C = A(:,J) (m x k), from
    LUPP of C (Sec. 3.1: the CUR row step; Eq. inty in row form):
    W = P^T [I; L2 L1^{-1}], so that C = W C(I,:) and W(I,:) = I.  It is the
    oracle's column ID of C^T with Omega = I_k.  Returns (I, W)."""
    A = _colmajor(A)
    J = np.asarray(J, dtype=np.int64)
    Cm = A[:, J]
    k = len(J)
    r = id_fixed_rank(np.ascontiguousarray(Cm.T), np.eye(k), k)
    return r["J"], np.asarray(r["X"]).T.copy()


def cur_middle(A, I, J) -> np.ndarray:
    """The CUR middle factor U = C^+ A R^+ with C = A(:,J), R = A(I,:)
    (Sec. 2.2.1, CUR): the Frobenius-optimal k x k matrix between C and R."""
    A = _colmajor(A)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    return np.linalg.pinv(A[:, J]) @ A @ np.linalg.pinv(A[I, :])  # library pseudo-inverses as steps


def cur_inverse_middle(A, I, J) -> np.ndarray:
    """The middle factor U = A(I,J)^{-1} (Sec. 2.2.1: the two-sided ID's A(I,J),
    inverted), for which C U R with C = A(:,J), R = A(I,:) reproduces A on the
    rows I and on the columns J."""
    A = _colmajor(A)
    return np.linalg.inv(A[np.ix_(np.asarray(I, dtype=np.int64), np.asarray(J, dtype=np.int64))])


def two_sided_residual(A, I, J, W, X) -> float:
    """||A - W A(I,J) X||_F, the two-sided ID error (Sec. 2.2.1)."""
    A = _colmajor(A)
    S = A[np.ix_(np.asarray(I, dtype=np.int64), np.asarray(J, dtype=np.int64))]
    return float(np.linalg.norm(A - np.asarray(W) @ S @ np.asarray(X)))


def cur_residual(A, I, J, U) -> float:
    """||A - C U R||_F with C = A(:,J), R = A(I,:) (Sec. 2.2.1, CUR)."""
    A = _colmajor(A)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    return float(np.linalg.norm(A - A[:, J] @ np.asarray(U) @ A[I, :]))


def rows_needed(n: int, b: int, kmax: int | None = None, m: int | None = None) -> int:
    """Sketch rows an adaptive run may draw: one block per round plus the first."""
    cap = n if kmax is None else min(n, kmax)
    if m is not None:
        cap = min(cap, m)
    return (-(-cap // b) + 1) * b
