"""Two-sided ID from a column skeleton (cur_from_id) against the oracle.

The oracle's fixed-rank column ID of C^T with Omega = I_k is exactly the LUPP
of C = A(:, J): its skeletons are the row skeletons I and its X is W^T."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("m,n,tol,dtype", [(700, 500, 1e-7, torch.float64), (333, 901, 1e-5, torch.float64),
                                           (1200, 600, 1e-4, torch.float32)])
def test_cur_from_id_matches_oracle(B, orc, m, n, tol, dtype):
    A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n), per_decade=25.0), seed=m + n)
    Ad = B.colmajor(torch.from_numpy(A).to("cuda", dtype))
    g = B.id_adaptive(Ad, tol, block=32, seed=2)
    I, Wm = B.cur_from_id(Ad, g.J)
    k = g.k
    A64 = Ad.double().cpu().numpy()
    J = g.J.cpu().numpy()
    C = A64[:, J]
    r = orc.id_fixed_rank(C.T.copy(), np.eye(k), k)
    if dtype == torch.float64:
        assert np.array_equal(I.cpu().numpy(), r["J"])
        Wg = Wm.double().cpu().numpy()
        np.testing.assert_array_equal(Wg[I.cpu().numpy()], np.eye(k))
        # C = W C(I,:) to rounding, like the oracle's
        assert np.linalg.norm(C - Wg @ C[I.cpu().numpy()]) <= 1e-10 * np.linalg.norm(C)
    else:
        # FP32: the leading (well-separated) row skeletons agree with the FP64 LUPP's;
        # late pivots sit at the FP32 rounding floor of C and are not compared
        h = k // 2
        overlap = len(set(I.cpu().numpy()[:h]) & set(r["J"][:h])) / h
        assert overlap >= 0.9
        Wg = Wm.double().cpu().numpy()
        np.testing.assert_array_equal(Wg[I.cpu().numpy()], np.eye(k))
        assert np.linalg.norm(C - Wg @ C[I.cpu().numpy()]) <= 1e-3 * np.linalg.norm(C)
    # two-sided ID: A ~ W A(I,J) X, as accurate as the column ID (up to a modest factor)
    Ii = I.cpu().numpy()
    X = g.X.double().cpu().numpy()
    two = np.linalg.norm(A64 - Wm.double().cpu().numpy() @ A64[np.ix_(Ii, J)] @ X)
    one = np.linalg.norm(A64 - C @ X)
    assert two <= 10 * one + 1e-12 * np.linalg.norm(A64)


def test_cur_from_id_rejects_bad_index(B):
    A = B.colmajor(torch.randn(50, 40, dtype=torch.float64, device="cuda"))
    J = torch.tensor([0, 3, 99], dtype=torch.int64, device="cuda")
    with pytest.raises(B.IDError) as e:
        B.cur_from_id(A, J)
    assert e.value.code == -2
