"""CPU check of the same-rank comparison used by the reduced-precision GPU tests:
the oracle's error at another run's rank, taken from the fixed-rank ID on the
same leading sample rows, is the error of the adaptive run that stops there."""
import numpy as np
import pytest

from idcheck import oracle_error_at_rank
from paper_2310_09417_gb300 import workloads as W


def test_error_at_rank_is_the_adaptive_error_there(orc):
    m, n, b = 400, 240, 16
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=21)
    Om = W.gaussian_omega(22, orc.rows_needed(n, b), m)
    nA = np.linalg.norm(A)
    tight = orc.id_adaptive(A, Om, b, 1e-8 * nA)
    loose = orc.id_adaptive(A, Om, b, 1e-3 * nA)
    assert loose["k"] < tight["k"]
    e_loose = orc.id_residual(A, loose["J"], loose["X"])
    assert oracle_error_at_rank(orc, A, Om, tight, loose["k"], b) == pytest.approx(e_loose, rel=1e-10)
    e_tight = orc.id_residual(A, tight["J"], tight["X"])
    assert oracle_error_at_rank(orc, A, Om, tight, tight["k"], b) == e_tight
    # and the other way round: a rank above the run's own
    assert oracle_error_at_rank(orc, A, Om, loose, tight["k"], b) == pytest.approx(e_tight, rel=1e-10)
