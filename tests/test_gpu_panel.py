"""GPU tests of the LUPP panel's pivot exchange (Algorithm 1, the partial
pivoting of Y^T): the candidates of one step are spread over many blocks and
either agree in the leading 32 bits of their magnitude (the FP64 panel then
compares the full bit patterns) or tie exactly (the smaller row wins).

With Omega = I (k x k) the sketch is Y = A, so Y^T's first column is A's first
row and the first pivot is the argmax of |A(0, :)| with ties to the smaller
column index, in the oracle and in the CUDA path alike.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from test_gpu_parity import dev, dev_cm  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


def first_row(mode, n, dtype):
    j = np.arange(n)
    sign = np.where(j % 3 == 1, -1.0, 1.0)
    if mode == "near_tie":
        # |A(0, j)| = 1 + (j mod 97) u: all share 1.0's leading bits; the largest
        # magnitude first occurs at j = 96
        u = 2.0 ** -45 if dtype == torch.float64 else 2.0 ** -20
        return sign * (1.0 + (j % 97) * u), 96
    if mode == "late_max":
        # one slightly larger magnitude near the end (the last blocks)
        u = 2.0 ** -40 if dtype == torch.float64 else 2.0 ** -20
        return sign * (1.0 + (j == n - 5) * u), n - 5
    # exact ties everywhere: the smallest column wins
    return sign * 2.0, 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mode", ["near_tie", "late_max", "exact_tie"])
def test_pivot_exchange_across_blocks(B, orc, mode, dtype):
    k, n = 6, 4000  # 4000 rows of Y^T: more than a hundred panel blocks
    rng = np.random.default_rng(11)
    A = rng.standard_normal((k, n))
    A[0], j0 = first_row(mode, n, dtype)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    A = A.astype(npdt).astype(np.float64)
    assert int(np.argmax(np.abs(A[0]))) == j0  # the construction survives the rounding
    Om = np.eye(k)
    g = B.id_fixed_rank(dev_cm(A, dtype), k, k, omega=dev(Om, dtype))
    r = orc.id_fixed_rank(A, Om, k)
    assert g.status == 0
    J = g.J.cpu().numpy()
    assert J[0] == j0 == r["J"][0]
    assert len(set(J.tolist())) == k
    if dtype == torch.float64:
        assert np.array_equal(J, r["J"])
