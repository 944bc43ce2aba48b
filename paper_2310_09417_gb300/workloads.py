"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds test matrices; it holds none of the ID method's
arithmetic and imports neither the CUDA binding nor the CPU oracle, so both
sides can share it.

Families (Sec. 5.1 of arXiv:2310.09417 and the benchmark configurations):
  * ``fast_decay``   A = U diag(d) V^T, d_i = beta^((i-1)/(n-1))        (Sec. 5.1)
  * ``geometric``    s_j = 10^(-j/20)                        (2000 x 2000 fixed-rank case)
  * ``poly``         s_j = (1 + j)^-2                        (40000 x 10000 adaptive case)
  * ``step``         s_j = 1 for j < 600, 1e-9 after          (40000 x 10000 adaptive case)
  * ``kahan``        D_n K_n with zeta = 0.99                (Sec. 5.1)
  * ``chan``         unit lower triangular, -1 below the diagonal (Appendix)
  * Gaussian kernel blocks exp(-|x-y|^2/h^2) between k-d tree leaves (batched case)

U and V have orthonormal columns from the QR factorisation of a Gaussian
matrix with the sign of diag(R) made positive (Haar measure).  For sizes too
large for a host QR, ``spectral_matrix_torch`` runs the same construction on
the GPU in FP32; the columns are then orthonormal to about 1e-6, which moves
each singular value by a relative 1e-6 and keeps the spectrum's shape.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- spectra
def spectrum(kind: str, n: int, **kw) -> np.ndarray:
    j = np.arange(n, dtype=np.float64)
    if kind == "geometric":          # 10^(-j/20)
        return 10.0 ** (-j / kw.get("per_decade", 20.0))
    if kind == "fast_decay":         # beta^((i-1)/(n-1)), beta = 1e-16
        beta = kw.get("beta", 1e-16)
        return beta ** (j / max(n - 1, 1))
    if kind == "poly":               # (1+j)^-2
        return (1.0 + j) ** (-kw.get("power", 2.0))
    if kind == "step":               # rank r at 1, then `floor`
        r = kw.get("rank", 600)
        s = np.full(n, kw.get("floor", 1e-9))
        s[: min(r, n)] = 1.0
        return s
    if kind == "exponential":        # exp(-j / scale)
        return np.exp(-j / kw.get("scale", n / 20.0))
    raise ValueError("unknown spectrum kind %r" % kind)


def haar_columns(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with Haar-distributed orthonormal columns (m >= n)."""
    G = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def spectral_matrix(m: int, n: int, s: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(s) V^T (float64, Fortran order), U m x r, V n x r, r = len(s)."""
    rng = np.random.default_rng(seed)
    r = len(s)
    U = haar_columns(rng, m, r)
    V = haar_columns(rng, n, r)
    return np.asfortranarray((U * s) @ V.T)


def spectral_matrix_torch(m: int, n: int, s: np.ndarray, seed: int, dtype, device):
    """GPU version of :func:`spectral_matrix` for large sizes (column-major).

    Returns a torch tensor of shape (n, m) whose row-major storage is A in
    column-major order (so ``t.data_ptr()`` is A with leading dimension m).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    r = len(s)

    def haar(rows, cols):
        G = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
        Q, R = torch.linalg.qr(G)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1
        return Q * d

    U = haar(m, r).to(torch.float64)
    V = haar(n, r).to(torch.float64)
    sv = torch.as_tensor(s, dtype=torch.float64, device=device)
    # A^T = V diag(s) U^T  (n x m, row-major == A column-major)
    At = (V * sv) @ U.T
    del U, V
    return At.to(dtype).contiguous()


def kahan(n: int, zeta: float = 0.99) -> np.ndarray:
    """Kahan matrix D_n K_n (Sec. 5.1): zeta^2 + phi^2 = 1."""
    phi = math.sqrt(1.0 - zeta * zeta)
    K = np.triu(-phi * np.ones((n, n)), 1) + np.eye(n)
    D = zeta ** np.arange(n)
    return np.asfortranarray(D[:, None] * K)


def chan(n: int) -> np.ndarray:
    """Unit lower triangular matrix with -1 below the diagonal (Appendix)."""
    return np.asfortranarray(np.tril(-np.ones((n, n)), -1) + np.eye(n))


def low_rank(m: int, n: int, r: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Exactly rank-r A = B C with Gaussian factors; returns (A, B, C)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, r))
    Cf = rng.standard_normal((r, n))
    return np.asfortranarray(B @ Cf), B, Cf


def gaussian_omega(seed: int, rows: int, m: int) -> np.ndarray:
    """A caller-supplied N(0,1) sketching matrix (rows x m), from numpy's PCG64."""
    return np.random.default_rng(seed).standard_normal((rows, m))


# ---------------------------------------------------------------- kernel blocks
def kd_tree_leaves(points: np.ndarray, leaf_max: int, rng: np.random.Generator) -> list:
    """Split the widest box side at a random fraction in [0.3, 0.7] until each
    leaf holds at most ``leaf_max`` points.  Returns a list of index arrays."""
    leaves = []
    stack = [np.arange(len(points))]
    while stack:
        idx = stack.pop()
        if len(idx) <= leaf_max:
            leaves.append(idx)
            continue
        P = points[idx]
        lo, hi = P.min(axis=0), P.max(axis=0)
        d = int(np.argmax(hi - lo))
        cut = lo[d] + rng.uniform(0.3, 0.7) * (hi[d] - lo[d])
        left = idx[P[:, d] < cut]
        right = idx[P[:, d] >= cut]
        if len(left) == 0 or len(right) == 0:  # degenerate split: halve by rank
            order = idx[np.argsort(P[:, d], kind="stable")]
            left, right = order[: len(order) // 2], order[len(order) // 2:]
        stack.append(right)
        stack.append(left)
    return leaves


def kernel_block_pairs(n_points: int, count: int, seed: int, leaf_max: int = 1024,
                       size_min: int = 64):
    """Points ~ U[0,1]^3, k-d tree leaves, and `count` (row-leaf, col-leaf) pairs
    whose sizes lie in [size_min, leaf_max]: near pairs (nearest leaf centres)
    and seeded random far pairs.  Returns (points, leaves, pairs)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n_points, 3))
    leaves = [l for l in kd_tree_leaves(pts, leaf_max, rng) if len(l) >= size_min]
    cent = np.array([pts[l].mean(axis=0) for l in leaves])
    pairs = []
    nl = len(leaves)
    # near pairs: each leaf with its nearest other leaf
    for a in range(nl):
        d = np.sum((cent - cent[a]) ** 2, axis=1)
        d[a] = np.inf
        pairs.append((a, int(np.argmin(d))))
        if len(pairs) >= count // 2:
            break
    while len(pairs) < count:
        a, b = rng.integers(0, nl, 2)
        if a != b:
            pairs.append((int(a), int(b)))
    return pts, leaves, pairs[:count]


def gaussian_kernel_block(pts: np.ndarray, rows: np.ndarray, cols: np.ndarray,
                          h: float = 0.3) -> np.ndarray:
    """K_ij = exp(-|x_i - y_j|^2 / h^2), column-major float64."""
    X = pts[rows]
    Y = pts[cols]
    d2 = np.sum(X * X, 1)[:, None] + np.sum(Y * Y, 1)[None, :] - 2.0 * X @ Y.T
    return np.asfortranarray(np.exp(-np.maximum(d2, 0.0) / (h * h)))
