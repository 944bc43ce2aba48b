"""GPU parity of what follows a column ID: the a-posteriori certificate (the
estimate Remark 1 points to, Sec. 3.2) and the residual block U_r of Remark 1,
each against the oracle on the same inputs.

* certificate: E_post = ||Omega'A - (Omega'A)(:,J) X||_F / sqrt(q) against
  oracle.certificate with the same Omega' (caller rows, and the generator's
  rows), in FP64 within 1e-9 relative; FP32 and BF16 inputs within their
  rounding; E_post^2 averages to the squared error (Sec. 4.2); a bad index is
  refused.
* U_r: the continued LUPP's extra pivots and trailing block against
  oracle.ur_estimates (pinned against LAPACK getrf): the extra columns
  identical, U_r within 1e-12 ||A||_F entrywise, ||U_r||_F and max|U_r| within
  1e-9 relative, the estimate equal to the fixed-rank Schur estimate.
"""
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


# ---------------------------------------------------------------- certificate
@pytest.mark.parametrize("m,n,q", [(1500, 900, 40), (333, 517, 7)])
def test_certificate_matches_oracle_f64(B, orc, m, n, q):
    A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n), per_decade=40.0), seed=m + 3)
    Ad = dev_cm(A)
    g = B.id_adaptive(Ad, 1e-5, block=32, seed=5)
    J = g.J.cpu().numpy()
    X = g.X.cpu().numpy()
    Omp = W.gaussian_omega(77, q, m)
    e = B.certificate(Ad, g.J, g.X, q, omega=dev(Omp))
    eo = orc.certificate(A, J, X, Omp)
    assert e == pytest.approx(eo, rel=1e-9, abs=1e-13 * np.linalg.norm(A))
    # the generator's rows: seed 99, rows 10 .. 10+q
    e2 = B.certificate(Ad, g.J, g.X, q, seed=99, row0=10)
    eo2 = orc.certificate(A, J, X, orc.gaussian_rows(99, 10, q, m))
    assert e2 == pytest.approx(eo2, rel=1e-9, abs=1e-13 * np.linalg.norm(A))
    # F64_EMU sketch: Omega' on the grid 2^-11
    from test_gpu_f64emu import on_grid
    e3 = B.certificate(Ad, g.J, g.X, q, omega=dev(Omp), sketch_prec=B.F64_EMU)
    eo3 = orc.certificate(A, J, X, on_grid(Omp))
    assert e3 == pytest.approx(eo3, rel=1e-9, abs=1e-13 * np.linalg.norm(A))


def test_certificate_f32_and_bf16(B, orc):
    m, n, q = 1200, 700, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=60.0), seed=8)
    A32 = A.astype(np.float32)
    Ad = dev_cm(A32, torch.float32)
    g = B.id_adaptive(Ad, 1e-3, block=32, seed=6)
    J = g.J.cpu().numpy()
    X = g.X.cpu().numpy().astype(np.float64)
    Omp = W.gaussian_omega(78, q, m).astype(np.float32)
    e = B.certificate(Ad, g.J, g.X, q, omega=dev(Omp, torch.float32))
    eo = orc.certificate(A32.astype(np.float64), J, X, Omp.astype(np.float64))
    assert e == pytest.approx(eo, rel=1e-3)
    # BF16 storage: the oracle on the decoded values and the BF16-rounded rows
    Ab = torch.from_numpy(A32).to("cuda").to(torch.bfloat16)
    Abd = B.colmajor_padded(Ab, 8)
    Ob = torch.from_numpy(Omp).to("cuda").to(torch.bfloat16)
    Obd = torch.zeros((q, -(-m // 8) * 8), dtype=torch.bfloat16, device="cuda")
    Obd[:, :m] = Ob
    e = B.certificate(Abd, g.J, g.X, q, omega=Obd[:, :m])
    eo = orc.certificate(Ab.double().cpu().numpy(), J, X, Ob.double().cpu().numpy())
    assert e == pytest.approx(eo, rel=1e-3)


def test_certificate_is_unbiased(B, orc):
    """E_post^2 over independent draws averages to ||A - A(:,J)X||_F^2."""
    m, n = 600, 400
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=30.0), seed=12)
    Ad = dev_cm(A)
    g = B.id_fixed_rank(Ad, 40, 50, seed=1)
    true2 = orc.id_residual(A, g.J.cpu().numpy(), g.X.cpu().numpy()) ** 2
    q = 8
    vals = np.array([B.certificate(Ad, g.J, g.X, q, seed=1000 + i) ** 2 for i in range(300)])
    # mean of 300 draws of a scaled chi-square with 8 q degrees of freedom at most:
    # relative standard error <= sqrt(2 / (8 q) / 300) ~ 0.01; 5 sigma
    assert abs(vals.mean() / true2 - 1.0) <= 0.05


def test_certificate_rejects_bad_index(B):
    A = B.colmajor(torch.randn(100, 80, dtype=torch.float64, device="cuda"))
    g = B.id_fixed_rank(A, 10, 12)
    J = g.J.clone()
    J[3] = 80
    with pytest.raises(B.IDError) as e:
        B.certificate(A, J, g.X, 5, seed=3)
    assert e.value.code == -2


# ---------------------------------------------------------------- U_r
@pytest.mark.parametrize("m,n,k,p,b", [(120, 80, 15, 6, 64), (900, 700, 100, 10, 32), (500, 450, 64, 5, 64)])
def test_ur_matches_oracle_f64(B, orc, m, n, k, p, b):
    A = W.spectral_matrix(m, n, W.spectrum("poly", n), seed=35 + m)
    Om = W.gaussian_omega(36 + m, k + p, m)
    r = B.ur_estimates(dev_cm(A), k, p, block=b, omega=dev(Om))
    u = orc.ur_estimates(A, Om, k)
    nA = np.linalg.norm(A)
    assert np.array_equal(r.id.J.cpu().numpy(), u["perm"][:k])
    assert np.array_equal(r.J_extra.cpu().numpy(), u["perm"][k:k + p])
    np.testing.assert_allclose(r.U_r.cpu().numpy(), u["U_r"], rtol=0, atol=1e-12 * nA)
    assert r.u_fro == pytest.approx(u["u_fro"], rel=1e-9, abs=1e-13 * nA)
    assert r.u_max == pytest.approx(u["u_max"], rel=1e-9, abs=1e-13 * nA)
    assert r.est == pytest.approx(u["est"], rel=1e-9, abs=1e-13 * nA)
    assert r.bound == pytest.approx(u["bound"], rel=1e-9, abs=1e-12 * nA)
    assert r.est == pytest.approx(orc.id_fixed_rank(A, Om, k)["est"], rel=1e-9, abs=1e-13 * nA)


def test_ur_f32(B, orc):
    m, n, k, p = 800, 600, 60, 8
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=80.0), seed=41).astype(np.float32)
    Om = W.gaussian_omega(42, k + p, m).astype(np.float32)
    r = B.ur_estimates(dev_cm(A, torch.float32), k, p, omega=dev(Om, torch.float32))
    u = orc.ur_estimates(A.astype(np.float64), Om.astype(np.float64), k)
    assert np.array_equal(r.id.J.cpu().numpy()[:20], u["perm"][:20])
    assert r.u_fro == pytest.approx(u["u_fro"], rel=2e-2)
    assert r.est == pytest.approx(u["est"], rel=2e-2)


def test_ur_argument_checks(B):
    A = B.colmajor(torch.randn(100, 80, dtype=torch.float64, device="cuda"))
    with pytest.raises(B.IDError) as e:
        B.ur_estimates(A, 75, 10)  # k + p > n
    assert e.value.code == -3
    with pytest.raises(B.IDError) as e:
        B.ur_estimates(A, 10, 200)  # p > 128
    assert e.value.code == -3
