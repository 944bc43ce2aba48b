"""GPU tests of the L1 condition estimate and the FP64 solve for X
(opts.x_solve_f64): kappa_1(L1) against numpy on the unit-lower factor of the
skeleton rows of the sketch, and an FP32-LU run whose L1 is exponentially
ill-conditioned and whose X cancels, where only the FP64 solve recovers X."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402

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


def unit_lower_of(M):
    """L of M = L U without pivoting (Doolittle), M square."""
    M = np.array(M, dtype=np.float64)
    k = M.shape[0]
    L = np.eye(k)
    U = M.copy()
    for c in range(k):
        L[c + 1:, c] = U[c + 1:, c] / U[c, c]
        U[c + 1:, c:] -= np.outer(L[c + 1:, c], U[c, c:])
    return L


def kappa1(L):
    return np.linalg.norm(L, 1) * np.linalg.norm(np.linalg.inv(L), 1)


@pytest.mark.parametrize("dtype,tol,rtol", [(torch.float64, 1e-4, 1e-8), (torch.float32, 1e-2, 1e-3)])
def test_cond_estimate_matches_numpy(B, orc, dtype, tol, rtol):
    """kappa_1(L1) of the run equals ||L1||_1 ||L1^{-1}||_1 of the unit-lower factor
    of Y^T(J, 0:k), the skeleton rows of the sketch in pivot order (LUPP restricted
    to those rows pivots in the same order, so no row exchange is needed).  The
    FP32 case stops early, where its pivots are well separated from their runners-up."""
    m, n, b = 700, 400, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=3)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    Om = W.gaussian_omega(4, orc.rows_needed(n, b, m=m), m).astype(npdt)
    g = B.id_adaptive(dev_cm(A.astype(npdt), dtype), tol, block=b, omega=dev(Om, dtype), x_solve_f64=1)
    k = g.k
    J = g.J.cpu().numpy()
    Yt = (Om[:k].astype(np.float64) @ A.astype(npdt).astype(np.float64)).T  # n x k
    L1 = unit_lower_of(Yt[J, :k])
    assert np.abs(L1).max() <= 1.0 + 1e-6  # partial pivoting: |L| <= 1
    assert g.cond_L1 == pytest.approx(kappa1(L1), rel=rtol)
    assert g.x_f64 == 0  # well conditioned: no FP64 re-solve


def test_mode_one_leaves_well_conditioned_x_unchanged(B):
    m, n, b = 900, 500, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=8).astype(np.float32)
    Ad = dev_cm(A, torch.float32)
    g0 = B.id_adaptive(Ad, 1e-4, block=b, seed=2)
    g1 = B.id_adaptive(Ad, 1e-4, block=b, seed=2, x_solve_f64=1)
    assert g0.cond_L1 == 0.0 and g1.cond_L1 >= 1.0
    assert g1.x_f64 == int(g1.cond_L1 > 4096.0)
    assert torch.equal(g0.J, g1.J)
    if not g1.x_f64:
        assert torch.equal(g0.X, g1.X)


def ill_conditioned_panel(n, k, seed):
    """An n x k matrix whose LUPP is itself (U = I, no row exchange): unit lower L1
    (k x k) with multipliers of random sign and magnitude 0.5 .. 0.95 (kappa_1
    grows exponentially in k), over L2 = T L1 with small T (|T| <= 0.01), so that
    T = L2 L1^{-1} is obtained only by cancelling terms of size |L2| |L1^{-1}|: a
    triangular solve in FP32 loses about u_32 kappa of T's accuracy there.  FP32 values."""
    rng = np.random.default_rng(seed)
    sg = rng.choice([-1.0, 1.0], size=(k, k))
    L1 = (np.eye(k) + np.tril(sg * rng.uniform(0.5, 0.95, size=(k, k)), -1)).astype(np.float32).astype(np.float64)
    L2 = rng.uniform(-0.01, 0.01, size=(n - k, k)) @ L1
    return np.vstack([L1, L2]).astype(np.float32).astype(np.float64)


def test_fp64_solve_recovers_x_of_ill_conditioned_l1(B):
    """Y = Omega A with Omega = I (caller rows of the identity) and A = L^T, so the
    sketch's LUPP returns L: J = 0..k-1 and X^T(J^c,:) = L2 L1^{-1}.  kappa_1(L1) is
    about 7e7 and T = L2 L1^{-1} cancels: the FP32 block updates keep only about
    two digits of X, the FP64 solve from the stored multipliers FP32 accuracy."""
    n, k, b = 300, 60, 20
    L = ill_conditioned_panel(n, k, 0)
    A = L.T.copy()          # k x n: Y^T = (I A)^T = L
    Om = np.eye(k)
    T_ref = L[k:] @ np.linalg.inv(L[:k])
    kap = kappa1(L[:k])
    assert kap > 1e7
    assert np.abs(L[k:]).max() < 0.5  # pivots stay on L1's diagonal
    Ad = dev_cm(A, torch.float32)
    Od = dev(Om, torch.float32)
    res = {}
    for mode in (0, 1, 2):
        g = B.id_fixed_rank(Ad, k, k, block=b, omega=Od, x_solve_f64=mode)
        assert np.array_equal(g.J.cpu().numpy(), np.arange(k))
        Xt = g.X.cpu().numpy().astype(np.float64).T[k:]  # rows J^c of X^T
        res[mode] = (np.linalg.norm(Xt - T_ref) / np.linalg.norm(T_ref), g)
    err0, g0 = res[0]
    err1, g1 = res[1]
    err2, g2 = res[2]
    assert g0.x_f64 == 0 and g1.x_f64 == 1 and g2.x_f64 == 1
    assert g1.cond_L1 > 1e6  # estimated from FP32 data: only its size matters here
    assert err1 < 1e-6 and err2 < 1e-6, (err1, err2)
    assert err0 > 100 * err1, (err0, err1)


def test_fp64_path_estimate_on_ill_conditioned_l1(B):
    n, k, b = 300, 60, 20
    L = ill_conditioned_panel(n, k, 1)
    g = B.id_fixed_rank(dev_cm(L.T.copy()), k, k, block=b, omega=dev(np.eye(k)), x_solve_f64=1)
    assert g.x_f64 == 0  # FP64 LU: X is already FP64
    assert g.cond_L1 == pytest.approx(kappa1(L[:k]), rel=1e-6)
