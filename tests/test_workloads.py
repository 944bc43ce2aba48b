"""CPU checks of the seeded input recipe shared by the oracle and the CUDA tests
(the synthetic stand-ins for the paper's test matrices, Sec. 5.1 and the
benchmark configurations): each generator produces the matrix it claims."""
import numpy as np
import pytest

from paper_2310_09417_gb300 import workloads as W


def test_spectra_definitions():
    n = 12
    j = np.arange(n)
    np.testing.assert_array_equal(W.spectrum("poly", n), (1.0 + j) ** -2.0)
    np.testing.assert_allclose(W.spectrum("geometric", n), 10.0 ** (-j / 20.0), rtol=1e-15)
    fd = W.spectrum("fast_decay", n)
    assert fd[0] == 1.0 and fd[-1] == pytest.approx(1e-16, rel=1e-12)
    np.testing.assert_allclose(np.diff(np.log(fd)), np.log(1e-16) / (n - 1), rtol=1e-12)
    st = W.spectrum("step", 10, rank=4, floor=1e-9)
    np.testing.assert_array_equal(st, [1.0] * 4 + [1e-9] * 6)
    with pytest.raises(ValueError):
        W.spectrum("unknown", 3)


@pytest.mark.parametrize("m,n,kind", [(300, 200, "poly"), (150, 150, "geometric"), (250, 120, "fast_decay")])
def test_spectral_matrix_has_the_spectrum(m, n, kind):
    s = W.spectrum(kind, n)
    A = W.spectral_matrix(m, n, s, seed=4)
    assert A.shape == (m, n) and A.flags.f_contiguous
    sv = np.linalg.svd(A, compute_uv=False)
    # Weyl: forming U diag(s) V^T in FP64 moves each singular value by at most a few
    # u ||A||, so the check is relative plus absolute at that level
    np.testing.assert_allclose(sv, s, rtol=1e-10, atol=1e-14 * s[0])
    # same seed, same matrix; another seed, another one
    np.testing.assert_array_equal(A, W.spectral_matrix(m, n, s, seed=4))
    assert not np.array_equal(A, W.spectral_matrix(m, n, s, seed=5))


def test_haar_columns_are_orthonormal():
    Q = W.haar_columns(np.random.default_rng(1), 80, 30)
    np.testing.assert_allclose(Q.T @ Q, np.eye(30), atol=1e-13)


def test_kahan_structure():
    n, zeta = 7, 0.99
    K = W.kahan(n, zeta)
    phi = np.sqrt(1 - zeta * zeta)
    for i in range(n):
        assert K[i, i] == pytest.approx(zeta ** i, rel=1e-15)
        for j in range(n):
            if j > i:
                assert K[i, j] == pytest.approx(-phi * zeta ** i, rel=1e-15)
            elif j < i:
                assert K[i, j] == 0.0


def test_chan_structure():
    C = W.chan(5)
    np.testing.assert_array_equal(C, np.eye(5) + np.tril(-np.ones((5, 5)), -1))


def test_low_rank_is_exactly_rank_r():
    A, B, Cf = W.low_rank(120, 90, 7, seed=3)
    np.testing.assert_allclose(A, B @ Cf, rtol=0, atol=0)
    sv = np.linalg.svd(A, compute_uv=False)
    assert sv[6] > 1e-3 * sv[0] and sv[7] < 1e-12 * sv[0]


def test_kd_tree_leaves_partition_the_points():
    rng = np.random.default_rng(2)
    pts = rng.random((5000, 3))
    leaves = W.kd_tree_leaves(pts, 200, rng)
    allidx = np.sort(np.concatenate(leaves))
    np.testing.assert_array_equal(allidx, np.arange(5000))
    assert max(len(l) for l in leaves) <= 200


def test_kernel_block_pairs_and_blocks():
    pts, leaves, pairs = W.kernel_block_pairs(20000, 40, seed=6, leaf_max=256, size_min=32)
    assert len(pairs) == 40
    for a, b in pairs:
        assert a != b
        assert 32 <= len(leaves[a]) <= 256 and 32 <= len(leaves[b]) <= 256
        assert len(np.intersect1d(leaves[a], leaves[b])) == 0  # off-diagonal blocks
    again = W.kernel_block_pairs(20000, 40, seed=6, leaf_max=256, size_min=32)[2]
    assert again == pairs
    a, b = pairs[0]
    K = W.gaussian_kernel_block(pts, leaves[a], leaves[b], h=0.3)
    x, y = pts[leaves[a][3]], pts[leaves[b][5]]
    assert K[3, 5] == pytest.approx(np.exp(-np.sum((x - y) ** 2) / 0.09), rel=1e-13)
    assert np.all(K > 0) and np.all(K <= 1)
    S = W.gaussian_kernel_block(pts, leaves[a], leaves[a], h=0.3)
    np.testing.assert_allclose(S, S.T, rtol=1e-14)
    np.testing.assert_allclose(np.diag(S), 1.0, rtol=1e-14)


def test_gaussian_omega_is_seeded_standard_normal():
    Om = W.gaussian_omega(3, 200, 500)
    assert Om.shape == (200, 500)
    np.testing.assert_array_equal(Om, W.gaussian_omega(3, 200, 500))
    assert abs(Om.mean()) < 0.01 and abs(Om.std() - 1.0) < 0.01
