"""Shared check for adaptive runs in reduced precision.

Algorithm 1 stops at the first block whose estimate E is at most tol.  Where the
GPU's estimate and the oracle's lie on either side of tol at a block boundary,
the two runs stop one block apart, and their errors are not comparable.  The
adaptive run is the fixed-rank run on the same leading sample rows (Sec. 5.2;
pinned by test_adaptive_equals_fixed_rank_with_same_rows).  So the oracle's
error at a rank k is that of the fixed-rank ID with Omega's first k + b rows.
The tests compare at the smaller of the two ranks: where the GPU stopped a
block later, its error is held to the oracle's at the oracle's own rank.
"""


def oracle_error_at_rank(orc, A, Om, r, k, b):
    """||A - A(:,J)X||_F of the oracle's ID at rank k: the adaptive result r
    itself when it stopped at k, else the fixed-rank ID with Om[:k + b]."""
    if k == r["k"]:
        return orc.id_residual(A, r["J"], r["X"])
    rk = orc.id_fixed_rank(A, Om[: k + b], k)
    return orc.id_residual(A, rk["J"], rk["X"])
