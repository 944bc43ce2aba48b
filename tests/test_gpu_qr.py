"""GPU parity of the Householder-QR products: the stable interpolation matrix
X_s = A(:,J)^+ A (column form of Eq. sID, Sec. 2.2) and the CUR / two-sided ID
middle factors (Sec. 2.2.1), against the oracle (LAPACK QR / least squares and
library inverses as its steps, pinned in test_oracle_pins).

* X_s: the projection A(:,J) X_s within 1e-12 ||A||_F of the oracle's (it is
  well conditioned), X_s itself within max(1e-10, 100 u cond(A(:,J))), the
  stable error within 1e-8 of the oracle's; panels of 32 columns with a ragged
  last panel; on an exactly rank-k matrix X_s equals the ID's X.
* U = C^+ A R^+: the product C U R within 1e-11 ||A||_F of the oracle's, U
  within a conditioning-scaled bar; U = A(I,J)^{-1}: against the oracle's
  inverse, and C U R reproduces A on the rows I and the columns J.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import dev_cm  # noqa: E402

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


def _skeleton(orc, A, k, seed):
    return orc.id_fixed_rank(A, W.gaussian_omega(seed, k + 8, A.shape[0]), k)["J"]


@pytest.mark.parametrize("m,n,k,kind", [(600, 400, 50, "geometric"), (2000, 1500, 129, "poly"),
                                         (900, 700, 37, "fast_decay"), (300, 300, 300, "geometric"),
                                         (5000, 300, 64, "poly")])
def test_stable_x_matches_oracle(B, orc, m, n, k, kind):
    A = W.spectral_matrix(m, n, W.spectrum(kind, min(m, n)), seed=m + k)
    J = _skeleton(orc, A, k, m + 1) if k < min(m, n) else np.arange(k)
    Jd = torch.from_numpy(J).to("cuda")
    Xg = B.stable_x(dev_cm(A), Jd).cpu().numpy()
    Xo = orc.stable_x(A, J)
    nA = np.linalg.norm(A)
    C = A[:, J]
    assert np.linalg.norm(C @ (Xg - Xo)) <= 1e-12 * nA
    cond = np.linalg.cond(C)
    bar = max(1e-10, 100 * U64 * cond)
    rel = np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)
    assert rel <= bar, (rel, bar, cond)
    eg = np.linalg.norm(A - C @ Xg) / nA
    eo = orc.stable_residual(A, J) / nA
    assert abs(eg - eo) <= 1e-8 * eo + 1e-13, (eg, eo)


def test_stable_x_exact_rank_equals_id_x(B, orc):
    m, n, k = 700, 500, 40
    A, _, _ = W.low_rank(m, n, k, seed=3)
    Om = W.gaussian_omega(4, k + 8, m)
    r = orc.id_fixed_rank(A, Om, k)
    Xg = B.stable_x(dev_cm(A), torch.from_numpy(r["J"]).to("cuda")).cpu().numpy()
    np.testing.assert_allclose(Xg, r["X"], rtol=0, atol=1e-9 * np.abs(r["X"]).max())


def test_stable_x_f32(B, orc):
    m, n, k = 1000, 600, 60
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=80.0), seed=5).astype(np.float32)
    A64 = A.astype(np.float64)
    J = _skeleton(orc, A64, k, 6)
    Xg = B.stable_x(dev_cm(A, torch.float32), torch.from_numpy(J).to("cuda")).cpu().numpy().astype(np.float64)
    eg = np.linalg.norm(A64 - A64[:, J] @ Xg)
    eo = orc.stable_residual(A64, J)
    assert eg <= eo * (1.0 + 1e-3) + 1e-5 * np.linalg.norm(A64)


@pytest.mark.parametrize("m,n,k", [(500, 400, 40), (1200, 900, 100), (300, 700, 33)])
def test_cur_middle_pseudoinverse(B, orc, m, n, k):
    A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n), per_decade=60.0), seed=m + n)
    J = _skeleton(orc, A, k, 9)
    I, _ = orc.row_id_of_columns(A, J)
    Ug = B.cur_middle(dev_cm(A), torch.from_numpy(I).to("cuda"), torch.from_numpy(J).to("cuda"),
                      B.CUR_PSEUDOINVERSE).cpu().numpy()
    Uo = orc.cur_middle(A, I, J)
    C, R = A[:, J], A[I, :]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(C @ (Ug - Uo) @ R) <= 1e-11 * nA
    assert orc.cur_residual(A, I, J, Ug) == pytest.approx(orc.cur_residual(A, I, J, Uo), rel=1e-8, abs=1e-13 * nA)
    bar = max(1e-10, 100 * U64 * np.linalg.cond(C) * np.linalg.cond(R))
    assert np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo) <= bar


def test_cur_middle_inverse(B, orc):
    m, n, k = 800, 600, 70
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=90.0), seed=10)
    J = _skeleton(orc, A, k, 11)
    I, _ = orc.row_id_of_columns(A, J)
    Ug = B.cur_middle(dev_cm(A), torch.from_numpy(I).to("cuda"), torch.from_numpy(J).to("cuda"),
                      B.CUR_INVERSE).cpu().numpy()
    Uo = orc.cur_inverse_middle(A, I, J)
    S = A[np.ix_(I, J)]
    bar = max(1e-10, 100 * U64 * np.linalg.cond(S))
    assert np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo) <= bar
    CUR = A[:, J] @ Ug @ A[I, :]
    np.testing.assert_allclose(CUR[I, :], A[I, :], rtol=0, atol=bar * np.abs(A).max() * 10)


def test_cur_middle_bad_index(B):
    A = B.colmajor(torch.randn(100, 80, dtype=torch.float64, device="cuda"))
    I = torch.arange(10, device="cuda")
    J = torch.arange(10, device="cuda")
    J[2] = 500
    with pytest.raises(B.IDError) as e:
        B.cur_middle(A, I, J, B.CUR_INVERSE)
    assert e.value.code == -2
