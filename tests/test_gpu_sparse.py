"""GPU parity of the sparse-sign sketch (Sec. 5.1, "Sparse Sign", zeta = 8).

* Omega element by element: the library's rows against the oracle's own
  implementation of the same counter-based definition -- bit-exact (the
  entries are +-sqrt(b/zeta), rounded the same way on both sides).
* the gather-add sketch against the oracle's dense product with the same
  Omega, on ragged shapes (rows of A not a multiple of the 128-row tile,
  columns not a multiple of 32, a last block cut short), in FP64 within 1e-13
  relative to sum |Omega||A| and in FP32 / BF16 within their rounding; two runs
  bit-identical (fixed summation order).
* the adaptive and fixed-rank IDs with the sparse-sign matrix against the oracle
  run on the same rows: J bit-exact, rank, rounds, estimates and X as for the
  Gaussian path; a rank guess (k0) leaves J, X and k unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import assert_id_close, dev_cm, oracle_x_spread  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("b,zeta,blocks,m", [(64, 8, 3, 1000), (16, 3, 5, 257), (128, 128, 1, 300), (5, 5, 2, 50),
                                              (1, 1, 4, 33), (32, 8, 2, 4097)])
def test_sparse_sign_rows_bit_exact(B, orc, b, zeta, blocks, m):
    seed, t0 = 2310_09417 + b, 7
    g = B.sparse_sign_rows(seed, t0, blocks, b, m, zeta).cpu().numpy()
    o = orc.sparse_sign_rows(seed, t0, blocks, b, m, zeta)
    np.testing.assert_array_equal(g, o)
    g32 = B.sparse_sign_rows(seed, t0, blocks, b, m, zeta, dtype=torch.float32).cpu().numpy()
    np.testing.assert_array_equal(g32, o.astype(np.float32))


@pytest.mark.parametrize("m,n,rows,b,zeta", [(1000, 77, 130, 64, 8), (3000, 600, 64, 64, 8), (257, 33, 40, 16, 8),
                                              (5000, 1000, 256, 128, 8), (3000, 150, 176, 16, 8),
                                              (700, 90, 96, 32, 32), (300, 40, 128, 128, 128), (129, 65, 7, 3, 2)])
def test_sparse_sketch_matches_dense_product(B, orc, m, n, rows, b, zeta):
    """Ragged tiles (m not a multiple of 128, n of 32 / 64), the last block cut
    short, one or several K splits, passes of many blocks (11 blocks of 16: three
    groups of four), zeta up to b (dense +-1 blocks: the largest lists)."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-8, 9, size=n))[None, :]
    blocks = -(-rows // b)
    Om = orc.sparse_sign_rows(5, 2, blocks, b, m, zeta)[:rows]
    ref = orc.sketch_t(A, Om)
    bound = (np.abs(Om) @ np.abs(A)).T
    G = B.sparse_sketch(dev_cm(A), rows, b, seed=5, t0=2, zeta=zeta).cpu().numpy()
    assert np.all(np.abs(G - ref) <= 1e-13 * bound + 1e-300)
    G2 = B.sparse_sketch(dev_cm(A), rows, b, seed=5, t0=2, zeta=zeta).cpu().numpy()
    np.testing.assert_array_equal(G, G2)
    # FP32 and BF16 storage: FP32 sums
    A32 = A.astype(np.float32)
    G32 = B.sparse_sketch(dev_cm(A32, torch.float32), rows, b, seed=5, t0=2, zeta=zeta).cpu().numpy()
    ref32 = orc.sketch_t(A32.astype(np.float64), Om)
    assert np.all(np.abs(G32 - ref32) <= 1e-5 * bound + 1e-30)
    Ab = torch.from_numpy(A32).to("cuda").to(torch.bfloat16)
    Gb = B.sparse_sketch(B.colmajor_padded(Ab, 8), rows, b, seed=5, t0=2, zeta=zeta).cpu().numpy()
    refb = orc.sketch_t(Ab.double().cpu().numpy(), Om)
    assert np.all(np.abs(Gb - refb) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("kind,m,n,b,tol", [("geometric", 900, 600, 32, 1e-6), ("poly", 2100, 700, 64, 1e-3),
                                             ("fast_decay", 500, 400, 16, 1e-8)])
def test_adaptive_sparse_sign_parity(B, orc, kind, m, n, b, tol):
    A = W.spectral_matrix(m, n, W.spectrum(kind, min(m, n)), seed=m + 2 * n)
    seed = 91
    rows = orc.rows_needed(n, b, m=m)
    Om = orc.sparse_sign_rows(seed, 0, rows // b, b, m)
    thr = tol * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    g = B.id_adaptive(dev_cm(A), tol, block=b, seed=seed, omega_kind=B.OMEGA_SPARSE_SIGN)
    assert g.status == r["status"]
    assert g.k == r["k"] and g.rounds == r["rounds"]
    assert_id_close(orc, A, g, r, spread, "adaptive sparse sign %s k=%d" % (kind, r["k"]))
    np.testing.assert_allclose(g.trace, r["trace"], rtol=1e-9, atol=1e-13 * orc.fro_norm(A))
    # a rank guess sketches several blocks per pass: the same result
    g2 = B.id_adaptive(dev_cm(A), tol, block=b, seed=seed, omega_kind=B.OMEGA_SPARSE_SIGN, k0=r["k"])
    assert g2.k == g.k and torch.equal(g2.J, g.J) and torch.equal(g2.X, g.X)


def test_fixed_rank_sparse_sign_parity(B, orc):
    m, n, k, l, b = 1500, 1100, 90, 100, 64  # l not a multiple of b: the second block is cut short
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=17)
    seed = 92
    Om = orc.sparse_sign_rows(seed, 0, 2, b, m)[:l]
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_fixed_rank(AA, Om, k))
    g = B.id_fixed_rank(dev_cm(A), k, l, block=b, seed=seed, omega_kind=B.OMEGA_SPARSE_SIGN)
    assert_id_close(orc, A, g, r, spread, "fixed rank sparse sign k=%d" % k)
    assert g.est_err == pytest.approx(r["est"], rel=1e-9)


def test_sparse_sign_with_tensor_core_schur_f64emu(B, orc):
    """F64_EMU with the sparse-sign sketch: the gather-add in FP64 replaces the
    digit-sliced sketch; the FP64-accurate tensor-core Schur GEMM and block update
    remain.  Same bars as the FP64 path."""
    m, n, b, tol = 2100, 700, 64, 1e-3
    A = W.spectral_matrix(m, n, W.spectrum("poly", n), seed=m + 2 * n)
    seed = 91
    Om = orc.sparse_sign_rows(seed, 0, orc.rows_needed(n, b, m=m) // b, b, m)
    thr = tol * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    g = B.id_adaptive(dev_cm(A), tol, block=b, seed=seed, omega_kind=B.OMEGA_SPARSE_SIGN, sketch_prec=B.F64_EMU)
    assert g.k == r["k"] and g.rounds == r["rounds"]
    assert_id_close(orc, A, g, r, spread, "adaptive sparse sign f64emu k=%d" % r["k"])
    np.testing.assert_allclose(g.trace, r["trace"], rtol=1e-9, atol=1e-13 * orc.fro_norm(A))


def test_sparse_sign_unsupported_paths(B):
    A = B.colmajor(torch.randn(200, 100, dtype=torch.float64, device="cuda"))
    Aodd = B.colmajor(torch.randn(257, 40, dtype=torch.float32, device="cuda").to(torch.bfloat16))
    with pytest.raises(B.IDError) as e:  # BF16 with an odd leading dimension
        B.sparse_sketch(Aodd, 64, 64)
    assert e.value.code == B.ERR_UNSUPPORTED
    A8 = B.quantize_fp8(B.colmajor(torch.randn(256, 100, dtype=torch.float32, device="cuda")))
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(A8, 1e-3, omega_kind=B.OMEGA_SPARSE_SIGN)
    assert e.value.code == B.ERR_UNSUPPORTED
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(A, 1e-3, block=16, omega_kind=B.OMEGA_SPARSE_SIGN, zeta=17)
    assert e.value.code == -2


def test_f32_sparse_sign_pass_size_does_not_change_result(B):
    """FP32 A with the sparse-sign sketch: four blocks per pass (the default), one
    block per pass and a rank guess give the same J, X and k bit for bit (the
    split count depends on the problem only, and every entry's gather sums run in
    the same order whatever the pass holds)."""
    A = W.spectral_matrix(2100, 700, W.spectrum("poly", 700), seed=5)
    Ad = dev_cm(A, torch.float32)
    kw = dict(block=64, seed=13, omega_kind=B.OMEGA_SPARSE_SIGN)
    base = B.id_adaptive(Ad, 1e-3, blocks_per_pass=1, **kw)
    assert 64 < base.k < 700
    for extra in (dict(), dict(k0=300), dict(blocks_per_pass=3)):
        g = B.id_adaptive(Ad, 1e-3, **kw, **extra)
        assert g.k == base.k and torch.equal(g.J, base.J) and torch.equal(g.X, base.X), extra
