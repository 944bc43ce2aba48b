"""GPU tests of the FP64-accurate sketch on the tensor cores (sketch precision
F64_EMU): A is split into exact BF16 digit slices, Omega is a Gaussian on the
grid 2^-11, and the digit products are summed exactly.

* the sketch against the exact product (extended-precision reference) within
  2^-52 max_i|A_ij| sum_r |Omega_cr| -- including sums near the FP32 exactness
  limit of the tensor-core accumulators;
* the sketch against an FP64 GEMM on tiled, ragged and split-K shapes;
* the whole ID against the FP64 oracle run on the same grid-rounded Omega:
  J bit-exact, X and the error within the FP64 bars of the plain path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402

from test_gpu_parity import assert_id_close, assert_x_close, dev, dev_cm, oracle_x_spread  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


def on_grid(Om):
    """Omega rounded to the grid 2^-11 and clipped to |q| <= 16383 (the sketch
    precision's definition of its Gaussian)."""
    return np.clip(np.rint(np.asarray(Om) * 2048.0), -16383.0, 16383.0) / 2048.0


def emu_bound(A, Om):
    """2^-52 max_i |A_ij| sum_r |Omega_cr|, as an (n x rows) array: the digit
    remainders (2^-55 per term) and the final rounding."""
    return 2.0 ** -52 * np.outer(np.abs(A).max(axis=0), np.abs(Om).sum(axis=1))


def sketch(B, A, Om):
    return B.id_sketch(dev_cm(A), dev(Om), sketch_prec=B.F64_EMU).cpu().numpy()


@pytest.mark.parametrize("case", ["scaled_columns", "near_accumulator_limit"])
def test_emu_sketch_against_exact_product(B, case):
    rng = np.random.default_rng(17)
    m, n, rows = 4101, 70, 33  # 9 exact chunks of 512, ragged K, n and rows
    if case == "scaled_columns":
        # column exponents from 2^-40 to 2^40, a zero column, a single spike
        A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-40, 41, size=n))[None, :]
        A[:, 3] = 0.0
        A[:, 5] = 0.0
        A[17, 5] = -3.0
        Om = on_grid(rng.standard_normal((rows, m)))
    else:
        # A = -0.99609375 = 2 (-127.5 / 256): digits d0 = -128, d1 = 128; Omega =
        # 16001 / 2048 (q1 = 63, q0 = -127), one sign per row: group 1 sums
        # 512 (127*128 + 63*128) = 0.74 * 2^24 over each chunk
        A = np.full((m, n), -0.99609375)
        A[:, ::3] *= -1.0
        Om = np.full((rows, m), 16001.0 / 2048.0)
        Om[1::2] *= -1.0
    G = sketch(B, A, Om)
    ref = (Om.astype(np.longdouble) @ A.astype(np.longdouble)).T
    err = np.abs(G.astype(np.longdouble) - ref).astype(np.float64)
    bound = emu_bound(A, Om)
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    if case == "scaled_columns":
        # nothing is lost for the zero column and the exactly representable spike
        np.testing.assert_array_equal(G[3], 0.0)
        np.testing.assert_array_equal(G[5], -3.0 * Om[:, 17])


@pytest.mark.parametrize("m,n,rows", [
    (1024, 256, 64),     # whole tiles, one chunk
    (1000, 333, 100),    # ragged K, n and rows (two Omega tiles)
    (8, 5, 3),           # smaller than every tile
    (40000, 300, 64),    # long K: many chunks and split-K partials
    (5000, 1100, 200),   # several column tiles and Omega tiles
])
def test_emu_sketch_matches_fp64_gemm(B, m, n, rows):
    rng = np.random.default_rng(m + n + rows)
    A = rng.standard_normal((m, n))
    Om = on_grid(rng.standard_normal((rows, m)))
    G = sketch(B, A, Om)
    ref = (torch.from_numpy(Om).cuda() @ torch.from_numpy(A).cuda()).t().cpu().numpy()
    # the FP64 GEMM's own rounding (at most m u |Omega||A|) plus the slicing bound
    tol = m * 2.0 ** -53 * (np.abs(Om) @ np.abs(A)).T + emu_bound(A, Om)
    assert np.all(np.abs(G - ref) <= tol)
    # and in practice far inside it: FP64-GEMM-level agreement
    rel = np.abs(G - ref).max() / (np.abs(Om) @ np.abs(A)).max()
    assert rel < 1e-14, rel


# ---------------------------------------------------------------- whole ID vs the oracle
@pytest.mark.parametrize("m,n,k,l,b", [
    (2000, 2000, 100, 120, 64),   # the 2000 x 2000 fixed-rank workload
    (257, 203, 37, 45, 16),       # ragged everything
    (300, 150, 1, 9, 64),         # k = 1
])
def test_emu_fixed_rank_parity(B, orc, m, n, k, l, b):
    A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n)), seed=m + n)
    Om = on_grid(W.gaussian_omega(k + l, l, m))
    g = B.id_fixed_rank(dev_cm(A), k, l, block=b, omega=dev(Om), sketch_prec=B.F64_EMU)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_fixed_rank(AA, Om, k))
    assert g.status == 0
    assert_id_close(orc, A, g, r, spread)
    assert g.est_err == pytest.approx(r["est"], rel=1e-10)


@pytest.mark.parametrize("kind,m,n,b,tol", [
    ("geometric", 600, 500, 32, 1e-6),
    ("poly", 700, 333, 64, 1e-3),
    ("geometric", 3000, 257, 20, 1e-9),   # three exact chunks along K
])
def test_emu_adaptive_parity(B, orc, kind, m, n, b, tol):
    A = W.spectral_matrix(m, n, W.spectrum(kind, min(m, n)), seed=m * 7 + n)
    Om = on_grid(W.gaussian_omega(n, orc.rows_needed(n, b, m=m), m))
    g = B.id_adaptive(dev_cm(A), tol, block=b, omega=dev(Om), sketch_prec=B.F64_EMU)
    thr = tol * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    assert g.status == r["status"]
    assert g.k == r["k"] and g.rounds == r["rounds"]
    assert_id_close(orc, A, g, r, spread)
    np.testing.assert_allclose(g.trace, r["trace"], rtol=1e-9, atol=1e-13 * orc.fro_norm(A))


def test_emu_generated_omega_matches_oracle_generator(B, orc):
    """Omega drawn on the device (Philox4x64-10 + Box-Muller, then the grid):
    the oracle's generator rounded to the same grid gives the same ID."""
    m, n, b = 1500, 400, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=9)
    seed = 777
    g = B.id_adaptive(dev_cm(A), 1e-6, block=b, seed=seed, sketch_prec=B.F64_EMU)
    Om = on_grid(orc.gaussian_rows(seed, 0, orc.rows_needed(n, b), m))
    thr = 1e-6 * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    assert g.k == r["k"]
    assert_id_close(orc, A, g, r, spread)


@pytest.mark.parametrize("seed,row0,rows,m", [(777, 0, 512, 40000), (3, 1000, 37, 9999), (2**63 + 5, 5, 130, 3001)])
def test_emu_grid_rows_equal_oracle_generator(B, orc, seed, row0, rows, m):
    """The FP64-accurate path's own Omega (FP32 Box-Muller, FP64 recomputation near
    a rounding boundary of 2048 z) against the oracle's FP64 generator rounded to
    the grid: every entry identical (20 million samples in the first case; a
    misrounded sample would be 2^-11 off)."""
    g = B.gaussian_rows(seed, row0, rows, m, grid=True).cpu().numpy()
    o = on_grid(orc.gaussian_rows(seed, row0, rows, m))
    bad = np.flatnonzero(g.ravel() != o.ravel())
    assert bad.size == 0, (bad[:5], g.ravel()[bad[:5]], o.ravel()[bad[:5]])


def test_emu_pass_size_does_not_change_result(B):
    m, n, b = 2100, 600, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=30.0), seed=5)
    Ad = dev_cm(A)
    base = B.id_adaptive(Ad, 1e-7, block=b, seed=11, sketch_prec=B.F64_EMU)
    for kw in (dict(k0=100), dict(blocks_per_pass=3)):
        g = B.id_adaptive(Ad, 1e-7, block=b, seed=11, sketch_prec=B.F64_EMU, **kw)
        assert g.k == base.k
        assert torch.equal(g.J, base.J)
        assert_x_close(g.X, base.X.cpu().numpy(), tol=1e-12)


def test_emu_matches_plain_fp64_path_on_same_omega(B):
    """Same grid-rounded Omega through the plain FP64 sketch and the emulated
    one: identical skeletons on a well-separated spectrum."""
    m, n, b = 1200, 500, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=21)
    Om = dev(on_grid(W.gaussian_omega(22, 600, m)))
    Ad = dev_cm(A)
    g0 = B.id_adaptive(Ad, 1e-8, block=b, omega=Om)
    g1 = B.id_adaptive(Ad, 1e-8, block=b, omega=Om, sketch_prec=B.F64_EMU)
    assert g0.k == g1.k and torch.equal(g0.J, g1.J)


def test_emu_rejects_other_input_types(B):
    A = B.colmajor(torch.randn(100, 50, dtype=torch.float32, device="cuda"))
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(A, 1e-3, sketch_prec=B.F64_EMU)
    assert e.value.code == B.ERR_UNSUPPORTED


def test_emu_nonfinite_input_is_rejected(B):
    A = torch.ones(50, 40, dtype=torch.float64, device="cuda")
    A[3, 7] = float("inf")
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(B.colmajor(A), 1e-3, sketch_prec=B.F64_EMU)
    assert e.value.code == B.ERR_NONFINITE


@pytest.mark.parametrize("b", [32, 128])
def test_emu_other_block_sizes(B, orc, b):
    """b = 32 runs the tensor-core Schur GEMM and block update on narrower panels;
    b = 128 is wider than they take (64), so those two steps run in FP64 SIMT
    while the sketch stays on the tensor cores.  Both match the oracle."""
    m, n, tol = 1500, 700, 1e-7
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n), seed=b)
    Om = on_grid(W.gaussian_omega(b, orc.rows_needed(n, b, m=m), m))
    g = B.id_adaptive(dev_cm(A), tol, block=b, omega=dev(Om), sketch_prec=B.F64_EMU)
    thr = tol * orc.fro_norm(A)
    r, spread = oracle_x_spread(orc, A, lambda AA: orc.id_adaptive(AA, Om, b, thr))
    assert g.k == r["k"]
    assert_id_close(orc, A, g, r, spread)


def test_emu_predictor_seeded_run_is_identical(B):
    """A rank guess from the learned predictor only changes how many blocks a
    pass sketches: J, X and k of the emulated path are bit-identical.  The
    network is hand-set to predict the plain loop's rank (all weights zero,
    b3 = 0, the output mean log2(k))."""
    m, n, b = 2000, 800, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=40.0), seed=4)
    Ad = dev_cm(A)
    plain = B.id_adaptive(Ad, 1e-8, block=b, seed=4, sketch_prec=B.F64_EMU)
    p = torch.zeros(B.mlp_param_count(), dtype=torch.float32, device="cuda")
    p[B.MLP_TRAINABLE + 35:B.MLP_TRAINABLE + 70] = 1.0
    p[-2] = float(np.log2(plain.k))
    p[-1] = 1.0
    seeded = B.id_adaptive(Ad, 1e-8, block=b, seed=4, sketch_prec=B.F64_EMU, predictor=p, max_pass_rows=4096)
    assert seeded.k == plain.k and torch.equal(seeded.J, plain.J)
    assert torch.equal(seeded.X, plain.X)
    assert seeded.passes == 2 < plain.passes
