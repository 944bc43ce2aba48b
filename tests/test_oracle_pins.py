"""Pins for the CPU oracle: each test checks it against something other than
itself -- a library routine, a closed form, a hand-worked example, an
invariant of the paper, or brute force -- so that a dropped term, a sign or
index error, or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2310_09417_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ random numbers
@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1], [2**64 - 1, 2**64 - 1]),
    ([123456789, 987654321, 0, 0], [2310_09417, 0]),
])
def test_philox_matches_numpy_library(orc, ctr, key):
    """Philox4x64-10 (Salmon et al. 2011) against numpy's independent
    implementation; numpy's first output block uses counter + 1."""
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    prev = c.copy()
    # numpy increments the 256-bit counter before generating the first block
    borrow = True
    for i in range(4):
        if borrow:
            borrow = prev[i] == 0
            prev[i] = prev[i] - np.uint64(1) if prev[i] != 0 else np.uint64(2**64 - 1)
    ref = np.random.Philox(counter=prev, key=k).random_raw(4)
    assert np.array_equal(orc.philox4x64_10(c, k), ref)


def test_gaussian_rows_moments(orc):
    """Box-Muller output is N(0,1): mean 0, variance 1, kurtosis 3, no
    correlation between rows or between neighbouring entries."""
    Z = orc.gaussian_rows(7, 0, 64, 8192)
    z = Z.ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 5 * np.sqrt(96 / n)
    C = np.corrcoef(Z)
    off = C[~np.eye(64, dtype=bool)]
    assert np.abs(off).max() < 6 / np.sqrt(8192)
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5 / np.sqrt(n)


def test_gaussian_rows_counter_addressing(orc):
    """Row i of the sketching matrix depends only on (seed, i): a window drawn
    at an offset equals the same rows of a larger draw."""
    big = orc.gaussian_rows(11, 0, 40, 130)
    win = orc.gaussian_rows(11, 17, 9, 130)
    assert np.array_equal(big[17:26], win)
    assert not np.array_equal(orc.gaussian_rows(12, 0, 1, 130), big[:1])


# ------------------------------------------------------------ sketch / norms
def test_sketch_matches_matmul(orc):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((37, 23))
    Om = rng.standard_normal((5, 37))
    YT = orc.sketch_t(A, Om)
    np.testing.assert_allclose(YT, (Om @ A).T, rtol=1e-13, atol=1e-13)


def test_norms_and_residual_match_numpy(orc):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((31, 19))
    assert orc.fro_norm(A) == pytest.approx(np.linalg.norm(A), rel=1e-14)
    J = np.array([4, 0, 11])
    X = rng.standard_normal((3, 19))
    ref = np.linalg.norm(A - A[:, J] @ X)
    assert orc.id_residual(A, J, X) == pytest.approx(ref, rel=1e-13)
    Q, _ = np.linalg.qr(A[:, J])
    assert orc.stable_residual(A, J) == pytest.approx(np.linalg.norm(A - Q @ (Q.T @ A)), rel=1e-11)


def test_residual_sums_columns_in_order(orc):
    """The residual's column sums are added in column order, whatever the
    threads: the value is that of the sequential sum, call after call."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 300))
    J = np.array([7, 150, 3, 299])
    X = rng.standard_normal((4, 300))
    D = A - A[:, J] @ X
    seq = 0.0
    for j in range(300):  # the same per-column sums, added in order
        seq += float(np.sum(D[:, j] ** 2))
    vals = {orc.id_residual(A, J, X) for _ in range(20)}
    assert len(vals) == 1
    assert vals.pop() == pytest.approx(np.sqrt(seq), rel=1e-14)


# ------------------------------------------------------------ LUPP
def test_lupp_hand_worked_example(orc):
    g = json.load(open(os.path.join(GOLDEN, "lupp_4x3_hand.json")))
    M = np.array(g["M"], dtype=float)
    LU, perm, z = orc.lupp(M)
    assert z == 0
    assert perm.tolist() == g["perm"]
    L = np.tril(LU, -1)[:, :3] + np.eye(4, 3)
    U = np.triu(LU[:3])
    np.testing.assert_allclose(L, np.array(g["L"]), atol=1e-15)
    np.testing.assert_allclose(U, np.array(g["U"]), atol=1e-14)


def test_fixed_rank_hand_worked_example(orc):
    """Same example as a column ID: Omega = I (3 x 3), A = M^T (3 x 4), k = 2."""
    g = json.load(open(os.path.join(GOLDEN, "lupp_4x3_hand.json")))
    A = np.array(g["M"], dtype=float).T
    r = orc.id_fixed_rank(A, np.eye(3), g["k"])
    assert r["J"].tolist() == g["J"]
    np.testing.assert_allclose(r["X"], np.array(g["X"]), atol=1e-15)
    assert r["est"] == pytest.approx(g["est"], rel=1e-14)


@pytest.mark.parametrize("shape", [(60, 17), (17, 17), (200, 40), (9, 30)])
def test_lupp_matches_lapack_getrf(orc, shape):
    """Partial pivoting on Gaussian data has no ties, so the textbook LUPP is
    LAPACK's getrf (scipy.linalg.lu): same permutation, same L and U."""
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    M = rng.standard_normal(shape)
    LU, perm, _ = orc.lupp(M)
    P, L, U = sla.lu(M)
    kk = min(shape)
    assert np.array_equal(np.argmax(P, axis=0), perm)
    np.testing.assert_allclose(np.tril(LU, -1)[:, :kk] + np.eye(shape[0], kk), L, atol=1e-13)
    np.testing.assert_allclose(np.triu(LU[:kk]), U, atol=1e-12)


def test_column_id_is_the_row_id_of_the_transpose(orc):
    """The paper states randLUPP as a row ID (Sec. 3.1): Y = B Omega_r, LUPP of
    Y, the first k pivot rows I, and B ~ W B(I,:) with W = P^T [I; L2 L1^{-1}]
    (Eq. inty).  Written here in that form with LAPACK's getrf (no ties on
    Gaussian data), applied to B = A^T with Omega_r = Omega^T, it gives the
    oracle's column ID of A: J = I and X = W^T."""
    rng = np.random.default_rng(17)
    m, n, l, k = 50, 40, 12, 8
    A = rng.standard_normal((m, n))
    Om = rng.standard_normal((l, m))
    B, Om_r = A.T, Om.T
    Y = B @ Om_r  # n x l
    P, L, _ = sla.lu(Y)
    perm = np.argmax(P, axis=0)  # Y[perm] = L U
    T = sla.solve_triangular(L[:k, :k], L[k:, :k].T, trans="T", lower=True, unit_diagonal=True).T
    Wt = np.zeros((n, k))
    Wt[perm[:k]] = np.eye(k)
    Wt[perm[k:]] = T
    r = orc.id_fixed_rank(A, Om, k)
    assert np.array_equal(r["J"], perm[:k])
    np.testing.assert_allclose(r["X"], Wt.T, rtol=0, atol=1e-12 * np.abs(Wt).max())
    # W(I,:) = I: the skeleton rows are reproduced exactly by the row ID
    np.testing.assert_array_equal(Wt[perm[:k]], np.eye(k))


def test_lupp_invariants(orc):
    """PA = LU to O(u)||A||, unit diagonal, |L| <= 1 (Eq. lupp)."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((300, 50)) * np.logspace(0, -6, 50)
    LU, perm, _ = orc.lupp(M)
    L = np.tril(LU, -1)[:, :50] + np.eye(300, 50)
    U = np.triu(LU[:50])
    assert np.abs(L).max() <= 1.0
    err = np.linalg.norm(M[perm] - L @ U) / np.linalg.norm(M)
    assert err < 50 * np.finfo(float).eps


def test_lupp_chan_matrix_ties(orc):
    """Chan's matrix (Appendix): every pivot column ties at |1| = |-1|; with ties
    going to the smallest label no row moves and the factors are L = A, U = I."""
    n = 12
    A = W.chan(n)
    LU, perm, _ = orc.lupp(A)
    assert perm.tolist() == list(range(n))
    np.testing.assert_array_equal(np.tril(LU, -1) + np.eye(n), A)
    np.testing.assert_array_equal(np.triu(LU), np.eye(n))


def test_lupp_growth_factor_closed_form(orc):
    """Chan's matrix with a last column of ones (Wilkinson's example) reaches
    the growth bound rho = 2^(n-1) of Sec. 2.3.2 exactly: U(j, n-1) = 2^j."""
    n = 20
    A = W.chan(n)
    A[:, -1] = 1.0
    LU, _, _ = orc.lupp(A)
    np.testing.assert_array_equal(np.diag(LU)[:-1], np.ones(n - 1))
    np.testing.assert_array_equal(LU[np.arange(n), n - 1], 2.0 ** np.arange(n))


def test_lupp_zero_column_is_skipped(orc):
    rng = np.random.default_rng(4)
    M = rng.standard_normal((10, 4))
    M[:, 1] = 0.0
    M[:, 2] = M[:, 0]  # column 2 becomes exactly zero after step 1
    LU, perm, z = orc.lupp(M)
    assert z == 2
    L = np.tril(LU, -1)[:, :4] + np.eye(10, 4)
    U = np.triu(LU[:4])
    np.testing.assert_allclose(M[perm], L @ U, atol=1e-14)


# ------------------------------------------------------------ column ID
def test_exact_recovery_rank_r(orc):
    """A = B C of rank r, k = r: X(:,J^c) = C_J^{-1} C_{J^c} independent of Omega
    (X = (Omega A)_J^{-1} (Omega A) = C_J^{-1} C), and the residual and the
    Schur estimate vanish to rounding."""
    m, n, r = 80, 60, 7
    A, B, Cf = W.low_rank(m, n, r, seed=5)
    Om = W.gaussian_omega(6, r + 4, m)
    res = orc.id_fixed_rank(A, Om, r)
    J = res["J"]
    Xref = np.linalg.solve(Cf[:, J], Cf)
    np.testing.assert_allclose(res["X"], Xref, atol=1e-10)
    np.testing.assert_allclose(res["X"][:, J], np.eye(r), atol=0)
    nA = np.linalg.norm(A)
    assert orc.id_residual(A, J, res["X"]) < 1e-12 * nA
    assert res["est"] < 1e-12 * nA


def test_brute_force_best_skeleton_tiny(orc):
    """On tiny inputs: SVD tail <= best k-subset projection error <= the method's
    stable ID error <= its ID error (Sec. 2.2, Eq. sID_row, Eckart-Young)."""
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        m, n, k = 9, 7, 3
        A = rng.standard_normal((m, n)) @ np.diag(0.3 ** np.arange(n)) @ rng.standard_normal((n, n))
        sv = np.linalg.svd(A, compute_uv=False)
        tail = np.sqrt(np.sum(sv[k:] ** 2))
        best = np.inf
        for S in itertools.combinations(range(n), k):
            Q, _ = np.linalg.qr(A[:, list(S)])
            best = min(best, np.linalg.norm(A - Q @ (Q.T @ A)))
        r = orc.id_fixed_rank(A, W.gaussian_omega(seed, k + 2, m), k)
        st = orc.stable_residual(A, r["J"])
        idr = orc.id_residual(A, r["J"], r["X"])
        eps = 1e-12 * np.linalg.norm(A)
        assert tail <= best + eps
        assert best <= st + eps
        assert st <= idr + eps


def test_schur_estimate_is_unbiased(orc):
    """E_Omega[E^2] = ||A - A(:,J) X||_F^2 (Sec. 4.2) for N(0,1) estimation
    blocks with E = ||S||_F / sqrt(b): the mean ratio over many independent
    draws is 1 within sampling error (the relative sd of one ratio <= sqrt(2/b))."""
    m, n, k, b = 120, 90, 10, 8
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=10.0), seed=7)
    ratios = []
    for seed in range(300):
        Om = W.gaussian_omega(1000 + seed, k + b, m)
        r = orc.id_fixed_rank(A, Om, k)
        true = orc.id_residual(A, r["J"], r["X"])
        ratios.append(r["est"] ** 2 / true ** 2)
    mean = float(np.mean(ratios))
    sd = float(np.std(ratios) / np.sqrt(len(ratios)))
    assert abs(mean - 1.0) < 4 * sd + 0.02, (mean, sd)
    assert sd < 0.05


def test_adaptive_equals_fixed_rank_with_same_rows(orc):
    """randLUPPadap is randLUPP with the same total sketch (Sec. 5.2): same J,
    same X and the same final estimate."""
    m, n, b = 300, 200, 16
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=8)
    Om = W.gaussian_omega(9, orc.rows_needed(n, b), m)
    ad = orc.id_adaptive(A, Om, b, 1e-6 * np.linalg.norm(A))
    k = ad["k"]
    assert k % b == 0 and ad["status"] == 0
    fx = orc.id_fixed_rank(A, Om[: k + b], k)
    assert np.array_equal(ad["J"], fx["J"])
    np.testing.assert_allclose(ad["X"], fx["X"], rtol=0, atol=1e-12)
    assert ad["trace"][-1] == pytest.approx(fx["est"], rel=1e-12)


def test_adaptive_stopping_rule(orc):
    """Algorithm 1 stops at the first round whose estimate is <= tol and the
    rank it returns is the one that estimate certifies; every earlier estimate
    exceeded tol; the estimate tracks the true error of each prefix rank."""
    m, n, b = 400, 250, 10
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=25.0), seed=10)
    Om = W.gaussian_omega(11, orc.rows_needed(n, b), m)
    tol = 1e-5 * np.linalg.norm(A)
    ad = orc.id_adaptive(A, Om, b, tol)
    tr = ad["trace"]
    assert tr[-1] <= tol and np.all(tr[:-1] > tol)
    assert ad["k"] == b * len(tr)
    for t, e in enumerate(tr):
        kk = b * (t + 1)
        fx = orc.id_fixed_rank(A, Om[: kk + b], kk)
        true = orc.id_residual(A, fx["J"], fx["X"])
        assert 0.25 < e / true < 4.0
    # the SVD tail lower-bounds the achieved error (Eckart-Young)
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.sqrt(np.sum(sv[ad["k"]:] ** 2)) <= orc.id_residual(A, ad["J"], ad["X"]) * (1 + 1e-9)


def test_permutation_equivariance(orc):
    """Relabelling the columns of A relabels J and the columns of X (the sketch
    of A(:,pi) is Y(:,pi); ties do not occur on Gaussian data)."""
    m, n, k = 70, 50, 9
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=12)
    Om = W.gaussian_omega(13, k + 3, m)
    pi = np.random.default_rng(14).permutation(n)
    r1 = orc.id_fixed_rank(A, Om, k)
    r2 = orc.id_fixed_rank(A[:, pi], Om, k)
    assert np.array_equal(pi[r2["J"]], r1["J"])
    np.testing.assert_allclose(r2["X"], r1["X"][:, pi], atol=1e-12)


def test_scale_invariance(orc):
    m, n, k = 60, 40, 6
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=15)
    Om = W.gaussian_omega(16, k + 4, m)
    r1 = orc.id_fixed_rank(A, Om, k)
    r2 = orc.id_fixed_rank(A * 2.0 ** -20, Om, k)
    assert np.array_equal(r1["J"], r2["J"])
    np.testing.assert_array_equal(r1["X"], r2["X"])
    assert r2["est"] == pytest.approx(r1["est"] * 2.0 ** -20, rel=1e-15)


def test_rank_cap_and_full_rank(orc):
    """When the tolerance cannot be met the run stops at min(m, n, kmax) with
    TOL_NOT_MET; at k = n every column is a skeleton and X is a permutation."""
    m, n, b = 50, 30, 8
    A = np.random.default_rng(17).standard_normal((m, n))
    Om = W.gaussian_omega(18, orc.rows_needed(n, b), m)
    r = orc.id_adaptive(A, Om, b, 0.0, kmax=20)
    assert r["k"] == 20 and r["status"] == orc.TOL_NOT_MET
    r = orc.id_adaptive(A, Om, b, 0.0)
    assert r["k"] == n and r["status"] == orc.OK
    assert sorted(r["J"].tolist()) == list(range(n))
    np.testing.assert_array_equal(r["X"][:, r["J"]], np.eye(n))


def test_nonfinite_input_rejected(orc):
    A = np.ones((5, 4))
    A[2, 3] = np.nan
    with pytest.raises(ValueError):
        orc.id_fixed_rank(A, np.ones((3, 5)), 2)


def test_kahan_and_fast_decay_estimate_tracks_error(orc):
    """Sec. 5.1 test matrices (reduced size): the Schur estimate overlaps the
    true ID error and the ID error is at least the stable ID error."""
    for A in (W.kahan(160), W.spectral_matrix(160, 160, W.spectrum("fast_decay", 160), seed=19)):
        m, n = A.shape
        b = 8
        Om = W.gaussian_omega(20, orc.rows_needed(n, b), m)
        ad = orc.id_adaptive(A, Om, b, 1e-8 * np.linalg.norm(A))
        true = orc.id_residual(A, ad["J"], ad["X"])
        st = orc.stable_residual(A, ad["J"])
        assert st <= true * (1 + 1e-9)
        if ad["k"] < n:
            assert 0.1 < ad["trace"][-1] / true < 10


# ------------------------------------------------------------ stable X, U_r estimates, certificate
def test_stable_x_is_the_least_squares_solution(orc):
    """X = A(:,J)^+ A (Eq. sID, column form): LAPACK's SVD-based least squares
    gives the same X, X(:,J) = I, its residual is the C oracle's Householder
    stable ID error, and no other X on the same skeleton does better."""
    m, n, k = 90, 60, 12
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=31)
    Om = W.gaussian_omega(32, k, m)
    r = orc.id_fixed_rank(A, Om, k)
    Xs = orc.stable_x(A, r["J"])
    Xl = np.linalg.lstsq(A[:, r["J"]], A, rcond=None)[0]
    np.testing.assert_allclose(Xs, Xl, rtol=0, atol=1e-9 * np.abs(Xl).max())
    np.testing.assert_allclose(Xs[:, r["J"]], np.eye(k), rtol=0, atol=1e-10)
    es = orc.id_residual(A, r["J"], Xs)
    assert es == pytest.approx(orc.stable_residual(A, r["J"]), rel=1e-9)
    assert es <= orc.id_residual(A, r["J"], r["X"]) * (1 + 1e-12)


def test_stable_x_equals_the_id_on_exactly_rank_k_input(orc):
    """A = B C of rank k: A(:,J) spans the range, and both interpolation
    matrices are C_J^{-1} C."""
    A, _, Cf = W.low_rank(70, 50, 6, seed=33)
    r = orc.id_fixed_rank(A, W.gaussian_omega(34, 6, 70), 6)
    want = np.linalg.solve(Cf[:, r["J"]], Cf)
    np.testing.assert_allclose(orc.stable_x(A, r["J"]), want, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r["X"], want, rtol=0, atol=1e-9)


def test_ur_block_is_lapacks_trailing_block_and_gives_the_schur_estimate(orc):
    """Remark 1: LUPP of [Y Y_r]^T continued for p more steps.  On Gaussian
    data (no ties) LAPACK's getrf gives the same permutation and the same
    trailing p x p block U_r; L_r U_r is the Schur complement of the p extra
    rows, so ||L_r U_r||_F / sqrt(p) is the fixed-rank Schur estimate
    (Eq. errSch), and |L_r| <= 1 gives the bound sqrt(n-k) ||U_r||_F."""
    m, n, k, p = 120, 80, 15, 6
    A = W.spectral_matrix(m, n, W.spectrum("poly", n), seed=35)
    Om = W.gaussian_omega(36, k + p, m)
    u = orc.ur_estimates(A, Om, k)
    P, L, U = sla.lu((Om @ A).T)
    assert np.array_equal(np.argmax(P, axis=0)[: k + p], u["perm"][: k + p])
    np.testing.assert_allclose(u["U_r"], U[k:, k:], rtol=0, atol=1e-12 * np.abs(U).max())
    np.testing.assert_allclose(u["L_r"], L[k:, k:], rtol=0, atol=1e-12)
    assert np.all(np.abs(u["L_r"]) <= 1.0)
    assert u["est"] == pytest.approx(orc.id_fixed_rank(A, Om, k)["est"], rel=1e-12)
    assert u["est"] * np.sqrt(p) <= u["bound"]
    assert u["u_fro"] == pytest.approx(np.linalg.norm(U[k:, k:]), rel=1e-12)
    assert u["u_max"] == pytest.approx(np.abs(U[k:, k:]).max(), rel=1e-12)
    assert u["u_max"] <= u["u_fro"] <= p * u["u_max"]  # p x p triangle


@pytest.mark.parametrize("kind", ["fast_decay", "geometric", "poly"])
def test_normUest_bounds_the_best_rank_k_error(orc, kind):
    """The paper's appendix: with Gaussian sketches, (4 log k / k) sqrt(m-k)
    ||U_r||_F (Eq. normUest) stays above the best rank-k error in every case it
    tried.  The oracle returns ||U_r||_F; the factor is the paper's, written
    here.  (How close Eq. maxUest comes is shown only in a figure the text
    does not carry, so neither side computes that estimate.)"""
    m = n = 400
    s = W.spectrum(kind, n)
    A = W.spectral_matrix(m, n, s, seed=37)
    for k in (20, 60, 120):
        for seed in range(3):
            u = orc.ur_estimates(A, W.gaussian_omega(40 + seed, k + 10, m), k)
            normUest = 4.0 * np.log(k) / k * np.sqrt(n - k) * u["u_fro"]  # the paper's Eq. normUest
            assert normUest >= np.sqrt(np.sum(s[k:] ** 2))


def test_certificate_identity_and_unbiasedness(orc):
    """The a-posteriori estimate ||Omega'(A - A(:,J)X)||_F / sqrt(q): with
    Omega' = I_m it is the error over sqrt(m) exactly; with fresh Gaussian rows
    its square averages to the squared error (Sec. 4.2)."""
    m, n, k = 60, 45, 8
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=41)
    r = orc.id_fixed_rank(A, W.gaussian_omega(42, k, m), k)
    e = orc.id_residual(A, r["J"], r["X"])
    assert orc.certificate(A, r["J"], r["X"], np.eye(m)) == pytest.approx(e / np.sqrt(m), rel=1e-12)
    q, trials = 4, 400
    sq = [orc.certificate(A, r["J"], r["X"], W.gaussian_omega(1000 + t, q, m)) ** 2 for t in range(trials)]
    # E^2 is e^2 times a chi-square with q * (effective rank) degrees over q: its
    # relative spread is at most sqrt(2/q); the mean of 400 is within 4 sigma
    assert abs(np.mean(sq) / e ** 2 - 1.0) <= 4 * np.sqrt(2.0 / q) / np.sqrt(trials)


# ------------------------------------------------------------ two-sided ID and CUR
def test_row_id_of_the_skeleton_columns(orc):
    """W from LUPP of C = A(:,J): W(I,:) = I, C = W C(I,:), and with LAPACK's
    getrf on C (no ties on this data) the same I and W = P^T [I; L2 L1^{-1}]."""
    m, n, k = 80, 60, 9
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=51)
    J = orc.id_fixed_rank(A, W.gaussian_omega(52, k, m), k)["J"]
    I, Wm = orc.row_id_of_columns(A, J)
    C = A[:, J]
    np.testing.assert_array_equal(Wm[I], np.eye(k))
    assert np.linalg.norm(C - Wm @ C[I]) <= 1e-12 * np.linalg.norm(C)
    P, L, _ = sla.lu(C)
    perm = np.argmax(P, axis=0)
    assert np.array_equal(I, perm[:k])
    T = sla.solve_triangular(L[:k, :k], L[k:, :k].T, trans="T", lower=True, unit_diagonal=True).T
    np.testing.assert_allclose(Wm[perm[k:]], T, rtol=0, atol=1e-12 * max(1.0, np.abs(T).max()))


def test_two_sided_and_cur_on_exactly_rank_k(orc):
    """A = B C of rank k: the two-sided ID W A(I,J) X and the CUR C U R both
    reproduce A to rounding."""
    A, _, _ = W.low_rank(70, 55, 7, seed=53)
    r = orc.id_fixed_rank(A, W.gaussian_omega(54, 7, 70), 7)
    I, Wm = orc.row_id_of_columns(A, r["J"])
    nA = np.linalg.norm(A)
    assert orc.two_sided_residual(A, I, r["J"], Wm, r["X"]) <= 1e-11 * nA
    assert orc.cur_residual(A, I, r["J"], orc.cur_middle(A, I, r["J"])) <= 1e-11 * nA


def test_two_sided_error_equals_column_id_error_and_cur_is_optimal(orc):
    """C = W A(I,J) makes the two-sided ID error the column ID error (Sec. 2.2.1:
    equivalent in exact arithmetic).  U = C^+ A R^+ is the least-squares middle
    factor: the normal equations C^T (A - C U R) R^T = 0 hold, and perturbing U
    only raises the error."""
    m, n, k = 90, 70, 12
    A = W.spectral_matrix(m, n, W.spectrum("poly", n), seed=55)
    r = orc.id_fixed_rank(A, W.gaussian_omega(56, k, m), k)
    J = r["J"]
    I, Wm = orc.row_id_of_columns(A, J)
    e1 = orc.id_residual(A, J, r["X"])
    assert orc.two_sided_residual(A, I, J, Wm, r["X"]) == pytest.approx(e1, rel=1e-9)
    U = orc.cur_middle(A, I, J)
    C, R = A[:, J], A[I, :]
    G = C.T @ (A - C @ U @ R) @ R.T
    assert np.abs(G).max() <= 1e-10 * np.linalg.norm(A) ** 3
    e = orc.cur_residual(A, I, J, U)
    rng = np.random.default_rng(57)
    for _ in range(5):
        assert orc.cur_residual(A, I, J, U + 1e-3 * np.abs(U).max() * rng.standard_normal(U.shape)) > e


# ------------------------------------------------------------ sparse-sign sketch
def test_sparse_sign_structure(orc):
    """zeta entries +-sqrt(b/zeta) per column of every block, so every column
    of Omega^T Omega's diagonal is exactly b; a block depends only on (seed, t)."""
    b, m, zeta = 64, 3000, 8
    S = orc.sparse_sign_rows(11, 0, 3, b, m, zeta)
    for q in range(3):
        blk = S[q * b:(q + 1) * b]
        nz = blk != 0
        assert np.all(nz.sum(axis=0) == zeta)
        np.testing.assert_array_equal(np.abs(blk[nz]), np.sqrt(b / zeta))
        np.testing.assert_allclose((blk ** 2).sum(axis=0), b, rtol=1e-15)
    np.testing.assert_array_equal(orc.sparse_sign_rows(11, 2, 1, b, m, zeta), S[2 * b:])
    assert not np.array_equal(S[:b], S[b:2 * b])
    assert not np.array_equal(orc.sparse_sign_rows(12, 0, 1, b, m, zeta), S[:b])


def test_sparse_sign_positions_pairs_and_signs_are_uniform(orc):
    """Uniformly random coordinates (Sec. 5.1): over 20000 columns every row is
    chosen equally often and every pair of rows equally often together (chi-square),
    and the Rademacher signs balance."""
    b, m, zeta = 32, 20000, 8
    blk = orc.sparse_sign_rows(13, 0, 1, b, m, zeta)
    nz = blk != 0
    counts = nz.sum(axis=1)
    expected = zeta * m / b
    assert ((counts - expected) ** 2 / expected).sum() < 31 + 6 * np.sqrt(2 * 31)  # 31 dof
    signs = np.sign(blk[nz])
    assert abs(signs.mean()) < 5 / np.sqrt(signs.size)
    co = nz.astype(float) @ nz.T.astype(float)
    off = co[np.triu_indices(b, 1)]
    e2 = m * zeta * (zeta - 1) / (b * (b - 1))
    assert off.sum() == pytest.approx(m * zeta * (zeta - 1) / 2)  # pairs per column are fixed
    dof = off.size - 1
    assert ((off - e2) ** 2 / e2).sum() < dof + 6 * np.sqrt(2 * dof)


def test_sparse_sign_sketch_recovers_rank_k_and_certifies_without_bias(orc):
    """Any sketch of full rank recovers an exactly rank-k matrix (X = C_J^{-1} C),
    and E[Omega^T Omega] = b I makes the certificate's square unbiased."""
    A, _, Cf = W.low_rank(90, 70, 6, seed=61)
    r = orc.id_fixed_rank(A, orc.sparse_sign_rows(14, 0, 1, 16, 90, 8), 6)
    np.testing.assert_allclose(r["X"], np.linalg.solve(Cf[:, r["J"]], Cf), rtol=0, atol=1e-9)
    m, n, k, b = 60, 45, 8, 16
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=41)
    r = orc.id_fixed_rank(A, W.gaussian_omega(42, k, m), k)
    e2 = orc.id_residual(A, r["J"], r["X"]) ** 2
    rat = np.array([orc.certificate(A, r["J"], r["X"], orc.sparse_sign_rows(99, t, 1, b, m, 8)) ** 2 / e2
                    for t in range(400)])
    assert abs(rat.mean() - 1.0) < 5 * rat.std() / np.sqrt(rat.size)


def test_cur_inverse_middle_interpolates_on_the_skeletons(orc):
    """U = A(I,J)^{-1}: C U R agrees with A on the rows I and the columns J (to
    rounding), and equals A exactly (to rounding) when A has rank k."""
    m, n, k = 70, 55, 9
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=8.0), seed=71)
    r = orc.id_fixed_rank(A, W.gaussian_omega(72, k + 4, m), k)
    I, _ = orc.row_id_of_columns(A, r["J"])
    U = orc.cur_inverse_middle(A, I, r["J"])
    CUR = A[:, r["J"]] @ U @ A[I, :]
    np.testing.assert_allclose(CUR[I, :], A[I, :], rtol=0, atol=1e-10 * np.abs(A).max())
    np.testing.assert_allclose(CUR[:, r["J"]], A[:, r["J"]], rtol=0, atol=1e-10 * np.abs(A).max())
    Ak, _, _ = W.low_rank(m, n, k, seed=73)
    rk = orc.id_fixed_rank(Ak, W.gaussian_omega(74, k + 4, m), k)
    Ik, _ = orc.row_id_of_columns(Ak, rk["J"])
    Uk = orc.cur_inverse_middle(Ak, Ik, rk["J"])
    np.testing.assert_allclose(Ak[:, rk["J"]] @ Uk @ Ak[Ik, :], Ak, rtol=0, atol=1e-9 * np.abs(Ak).max())
