"""GPU parity at late-round shapes: ranks in the thousands, where paths that a
small case never reaches take over (tb in the thousands of earlier pivots,
the panel over thousands of remaining columns, the FP32 Schur products split
K 32 ways with few remaining rows).

* FP64 and FP64-accurate tensor-core adaptive runs on a 4500 x 3000 matrix
  with geometric decay 10^(-j/450) at relative tolerance 1e-3: the oracle stops
  at k = 2240 after 35 rounds (Algorithm 1).  J bit-exact, the estimates
  E^(t) within 1e-9 relative (+1e-13 ||A||_F), A(:,J) X within 1e-10 ||A||.
* FP32 fixed rank k = 4200 of n = 4400 (l = 4264): from tb = 4096 on, the
  Schur product has K = tb >= 4096 and 304 remaining rows, which the FP32 path
  splits 32 ways.  FP32 cannot reproduce FP64 skeletons late in the run, so it
  is held to the FP64 oracle's error at the same rank, and its estimate to the
  oracle's evaluation of the same quantity for the GPU's own J and X.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import assert_id_close, dev, dev_cm, oracle_x_spread  # noqa: E402
from test_gpu_f64emu import on_grid  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def late_case(orc):
    m, n, b, tol = 4500, 3000, 64, 1e-3
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=450.0), seed=61)
    Om = W.gaussian_omega(62, orc.rows_needed(n, b, m=m), m)
    return A, Om, b, tol


@pytest.mark.parametrize("precision", ["f64", "f64emu"])
def test_adaptive_late_rounds(B, orc, late_case, precision):
    A, Om, b, tol = late_case
    if precision == "f64emu":
        Om = on_grid(Om)
    thr = tol * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    assert r["k"] >= 2000 and r["k"] < A.shape[1]
    g = B.id_adaptive(dev_cm(A), tol, block=b, omega=dev(Om),
                      sketch_prec=B.F64_EMU if precision == "f64emu" else None)
    assert g.status == r["status"]
    assert g.k == r["k"] and g.rounds == r["rounds"]
    assert_id_close(orc, A, g, r, spread, "adaptive late rounds %s k=%d" % (precision, r["k"]))
    np.testing.assert_allclose(g.trace, r["trace"], rtol=1e-9, atol=1e-13 * orc.fro_norm(A))


def test_fixed_rank_f32_split_k_late(B, orc):
    m, n, k, l, b = 5000, 4400, 4200, 4264, 64
    A = W.spectral_matrix(m, n, W.spectrum("poly", n, power=1.0), seed=63).astype(np.float32)
    Om = W.gaussian_omega(64, l, m).astype(np.float32)
    A64 = A.astype(np.float64)
    g = B.id_fixed_rank(dev_cm(A, torch.float32), k, l, block=b, omega=dev(Om, torch.float32))
    r = orc.id_fixed_rank(A64, Om.astype(np.float64), k)
    J = g.J.cpu().numpy()
    assert len(np.unique(J)) == k
    # the leading pivots are far apart: identical even in FP32
    assert np.array_equal(J[:64], r["J"][:64])
    eg = orc.id_residual(A64, J, g.X.cpu().numpy().astype(np.float64))
    eo = orc.id_residual(A64, r["J"], r["X"])
    assert eg <= 1.2 * eo, (eg, eo)
    # the Schur estimate of the 64 extra rows, formed after the 32-way split products,
    # is ||Omega_e (A - A(:,J) X)||_F / sqrt(l - k) for the GPU's own J and X (the
    # estimation rows Omega_e = Omega[k:l]); the oracle evaluates that in FP64
    ref = orc.certificate(A64, J, g.X.cpu().numpy().astype(np.float64), Om[k:].astype(np.float64))
    assert g.est_err == pytest.approx(ref, rel=1e-3)
