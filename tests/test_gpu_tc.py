"""Tensor-core (tcgen05 + TMA) sketch and the BF16-input ID.

The BF16 path sketches with BF16 x BF16 products accumulated in FP32 in tensor
memory; the references are FP64 products of the same BF16 values (exact
inputs), so the only differences are FP32 accumulation and the FP32 LU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402
from idcheck import oracle_error_at_rank  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


def bf16_pair(rng, m, n, rows):
    """Column-major BF16 A (m x n) and row-major BF16 Omega (rows x m)."""
    A = torch.from_numpy(rng.standard_normal((m, n))).to("cuda", torch.bfloat16)
    Om = torch.from_numpy(rng.standard_normal((rows, m))).to("cuda", torch.bfloat16).contiguous()
    return A, Om


@pytest.mark.parametrize("m,n,rows", [
    (1024, 256, 64),     # whole tiles
    (1000, 333, 100),    # ragged K (not a multiple of 64), ragged n and rows (two N tiles)
    (64, 128, 64),       # one K stage
    (40000, 300, 64),    # long K: many split-K partials
    (8, 5, 3),           # smaller than every tile
    (3000, 700, 600),    # a pass of many blocks: groups of four 64-row sub-tiles, a ragged last group
])
def test_tc_sketch_matches_fp64_product(B, m, n, rows):
    rng = np.random.default_rng(m + n + rows)
    A, Om = bf16_pair(rng, m, n, rows)
    Acm = B.colmajor(A)
    G = B.id_sketch(Acm, Om)
    ref = (Om.double() @ Acm.double()).t()
    # FP32 accumulation of exact BF16 products: error ~ u32 sqrt(m) |Omega||A|
    scale = (Om.double().abs() @ Acm.double().abs()).t()
    err = ((G.double() - ref).abs() / scale).max().item()
    assert err < 4e-6 * max(1.0, np.sqrt(m / 1024)), err


def test_bf16_gaussian_rows_round_the_fp64_generator(B, orc):
    """BF16 rows: the same counters and Box-Muller map evaluated in FP32 on the
    leading 24 bits.  Against the FP64 generator rounded to BF16 (nearest even):
    equal except where the two evaluations straddle a rounding boundary, and
    then one BF16 step apart."""
    g = B.gaussian_rows(7, 0, 64, 4099, dtype=torch.bfloat16).float().cpu().numpy()
    ob = torch.from_numpy(orc.gaussian_rows(7, 0, 64, 4099)).to(torch.bfloat16).float().numpy()
    diff = g != ob
    assert diff.mean() < 1e-3
    assert np.all(np.abs(g[diff] - ob[diff]) <= 2.0 ** -7 * np.abs(ob[diff]) * 1.01)


def test_simt_sketch_matches_fp64_product(B):
    rng = np.random.default_rng(3)
    A = B.colmajor(torch.from_numpy(rng.standard_normal((777, 129))).cuda())
    Om = torch.from_numpy(rng.standard_normal((70, 777))).cuda()
    G = B.id_sketch(A, Om)
    torch.testing.assert_close(G, (Om @ A).t(), rtol=1e-12, atol=1e-12)


def test_tc_rejects_misaligned_leading_dimension(B):
    A = torch.zeros((100, 7), dtype=torch.bfloat16, device="cuda")  # ld = 100 is not a multiple of 8
    Om = torch.zeros((64, 100), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(B.IDError) as e:
        B.id_sketch(B.colmajor(A), Om)
    assert e.value.code == B.ERR_UNSUPPORTED


def test_adaptive_bf16_against_fp64_oracle(B, orc):
    """Low-rank-plus-noise input stored in BF16 (the mixed-precision workload at
    reduced size): the BF16-sketch / FP32-LU run meets the tolerance, its rank is
    within one block of the FP64 oracle's on the same BF16 values, and its
    achieved error is within 1.2x of the oracle's at the smaller of the
    two ranks.  The tolerance sits above the BF16 rounding floor of A (about
    2e-3 relative)."""
    m, n, r, b, tol = 4096, 1024, 150, 32, 1e-2
    rng = np.random.default_rng(31)
    A = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n))) / np.sqrt(r)
    A += 1e-4 * rng.standard_normal((m, n))
    Ab = torch.from_numpy(A).to("cuda", torch.bfloat16)
    A64 = Ab.double().cpu().numpy()
    Om = torch.from_numpy(W.gaussian_omega(32, orc.rows_needed(n, b), m)).to("cuda", torch.bfloat16).contiguous()
    g = B.id_adaptive(B.colmajor(Ab), tol, block=b, omega=Om)
    r_ = orc.id_adaptive(A64, Om.double().cpu().numpy(), b, tol * orc.fro_norm(A64))
    assert g.status == 0
    assert abs(g.k - r_["k"]) <= b
    nA = orc.fro_norm(A64)
    eg = orc.id_residual(A64, g.J.cpu().numpy(), g.X.double().cpu().numpy()) / nA
    eo = oracle_error_at_rank(orc, A64, Om.double().cpu().numpy(), r_, min(g.k, r_["k"]), b) / nA
    assert eg <= 1.2 * eo + 1e-6
    assert eg <= 2 * tol
    kk = min(g.k, r_["k"])
    assert len(set(g.J.cpu().numpy()[:kk]) & set(r_["J"][:kk])) / kk >= 0.9


def test_bf16_generated_omega_runs_and_meets_tolerance(B, orc):
    m, n, r = 3000, 800, 80
    rng = np.random.default_rng(33)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + 1e-4 * rng.standard_normal((m, n))
    Ab = torch.from_numpy(A).to("cuda", torch.bfloat16)
    g = B.id_adaptive(B.colmajor(Ab), 1e-2, block=64, seed=5)
    A64 = Ab.double().cpu().numpy()
    e = orc.id_residual(A64, g.J.cpu().numpy(), g.X.double().cpu().numpy()) / orc.fro_norm(A64)
    assert g.k >= r and e <= 2e-2


# ---------------------------------------------------------------- FP32 sketch by digit slicing
@pytest.mark.parametrize("m,n,rows", [
    (1024, 256, 64),     # whole tiles
    (1000, 333, 100),    # ragged K, n and rows (two 64-column tiles)
    (8, 5, 3),           # smaller than every tile
    (40000, 300, 64),    # long K: many exact chunks and split-K partials
    (3000, 1100, 200),
])
def test_f32emu_sketch_matches_fp64_product(B, m, n, rows):
    """sketch_prec F32_EMU: A and Omega (FP32) in 3 digits of 8 bits each on the
    tensor cores.  Against the FP64 product of the same FP32 values: FP32-level
    error relative to |Omega| |A|."""
    rng = np.random.default_rng(m + 2 * n + rows)
    A = (rng.standard_normal((m, n)) * np.exp2(rng.integers(-6, 7, size=(1, n)))).astype(np.float32)
    Om = rng.standard_normal((rows, m)).astype(np.float32)
    Ad = B.colmajor(torch.from_numpy(A).cuda())
    G = B.id_sketch(Ad, torch.from_numpy(Om).cuda(), sketch_prec=B.F32_EMU).double().cpu().numpy()
    ref = (Om.astype(np.float64) @ A.astype(np.float64)).T
    scale = (np.abs(Om).astype(np.float64) @ np.abs(A).astype(np.float64)).T
    err = (np.abs(G - ref) / scale).max()
    assert err < 2e-6, err


def test_f32emu_adaptive_against_f64_oracle(B, orc):
    """The FP32 sketch on the tensor cores with FP32 LU: the rank matches the FP64
    oracle's within one block, the skeletons overlap almost entirely and the
    achieved error is within 1.2x of the oracle's."""
    m, n, b = 1200, 800, 32
    A = W.spectral_matrix(m, n, W.spectrum("poly", n), seed=12).astype(np.float32)
    Om = W.gaussian_omega(13, orc.rows_needed(n, b), m).astype(np.float32)
    tol = 1e-4
    g = B.id_adaptive(B.colmajor(torch.from_numpy(A).cuda()), tol, block=b, omega=torch.from_numpy(Om).cuda(),
                      sketch_prec=B.F32_EMU)
    A64 = A.astype(np.float64)
    r = orc.id_adaptive(A64, Om.astype(np.float64), b, tol * orc.fro_norm(A64))
    assert abs(g.k - r["k"]) <= b
    kk = min(g.k, r["k"])
    assert len(set(g.J.cpu().numpy()[:kk]) & set(r["J"][:kk])) / kk >= 0.95
    eg = orc.id_residual(A64, g.J.cpu().numpy(), g.X.cpu().numpy().astype(np.float64))
    eo = orc.id_residual(A64, r["J"], r["X"])
    assert eg <= 1.2 * eo and eg <= 3 * tol * orc.fro_norm(A64)


def test_f32emu_pass_size_does_not_change_result(B):
    m, n, b = 2100, 600, 32
    A = W.spectral_matrix(m, n, W.spectrum("geometric", n, per_decade=30.0), seed=5).astype(np.float32)
    Ad = B.colmajor(torch.from_numpy(A).cuda())
    base = B.id_adaptive(Ad, 1e-4, block=b, seed=11, sketch_prec=B.F32_EMU)
    for kw in (dict(k0=100), dict(blocks_per_pass=3)):
        g = B.id_adaptive(Ad, 1e-4, block=b, seed=11, sketch_prec=B.F32_EMU, **kw)
        assert g.k == base.k and torch.equal(g.J, base.J) and torch.equal(g.X, base.X)


def test_tc_sketch_wide_pass_equals_block_passes(B):
    """A pass of many blocks (a CTA runs the MMAs of four 64-row sub-tiles of Omega
    on each stage of A) gives every entry the same bits as passes of one block
    (K = 512: one split for both; rows of Omega 16-byte aligned for TMA)."""
    rng = np.random.default_rng(5)
    m, n, rows = 512, 700, 600
    A, Om = bf16_pair(rng, m, n, rows)
    Acm = B.colmajor(A)
    G = B.id_sketch(Acm, Om)
    for r0 in range(0, rows, 64):
        g = B.id_sketch(Acm, Om[r0:r0 + 64].contiguous())
        assert torch.equal(G[:, r0:r0 + 64], g), r0


def test_bf16_pass_size_does_not_change_result(B):
    """Adaptive BF16 runs with a rank guess or several blocks per pass (wide
    sketch passes) return the one-block-per-pass run's J, X and k bit for bit."""
    m, n, b = 6000, 1500, 64
    rng = np.random.default_rng(8)
    A = (rng.standard_normal((m, 300)) @ rng.standard_normal((300, n))) / np.sqrt(300)
    A += 1e-3 * rng.standard_normal((m, n))
    Ad = B.colmajor(torch.from_numpy(A).to("cuda", torch.bfloat16))
    base = B.id_adaptive(Ad, 3e-2, block=b, seed=4)
    for kw in (dict(k0=400), dict(blocks_per_pass=5)):
        g = B.id_adaptive(Ad, 3e-2, block=b, seed=4, **kw)
        assert g.k == base.k and torch.equal(g.J, base.J) and torch.equal(g.X, base.X)


@pytest.mark.parametrize("m,n", [(4096, 50), (1003, 33), (8, 5)])
def test_bf16_norm_matches_fp64_sum_of_squares(B, m, n):
    """||A||_F of a BF16 matrix (eight values per load, exact FP32 squares summed in
    float-float groups, FP64 across groups) against the FP64 sum of squares, with
    zeros, subnormal, tiny (below 2^-63) and huge (above 2^54) entries that take
    the FP64 branch, and rows not a multiple of eight."""
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-20, 21, size=n))[None, :]
    A[rng.random((m, n)) < 0.05] = 0.0
    A[0, 0], A[1 % m, 1] = 1e-40, 3e-25
    A[2 % m, 2], A[3 % m, 3] = 1e17, -3e17
    Ab = B.colmajor_padded(torch.from_numpy(A).cuda().to(torch.bfloat16), 8)
    ref = float(np.sqrt(np.sum(Ab.double().cpu().numpy() ** 2)))
    g = B.id_adaptive(Ab, 0.9, block=8, k_max=8)
    assert g.norm_A == pytest.approx(ref, rel=1e-12)


def test_bf16_nonfinite_is_rejected(B):
    Ab = B.colmajor_padded(torch.randn(1000, 20, device="cuda").to(torch.bfloat16), 8)
    Ab[999, 7] = float("inf")
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(Ab, 1e-1)
    assert e.value.code == B.ERR_NONFINITE


@pytest.mark.parametrize("m,n,ld_pad", [(4096, 40, 0), (1001, 17, 3)])
def test_f32_norm_matches_fp64_sum_of_squares(B, m, n, ld_pad):
    """||A||_F of an FP32 matrix (four values per load when aligned, FP32 squares
    with their FMA rounding errors summed in float-float groups, FP64 across groups)
    against the FP64 sum of squares, with zeros, tiny, subnormal and huge entries
    (FP64 branch), an unaligned leading dimension and rows not a multiple of four."""
    rng = np.random.default_rng(m + 1)
    A = (rng.standard_normal((m, n)) * np.exp2(rng.integers(-30, 31, size=n))[None, :]).astype(np.float32)
    A[rng.random((m, n)) < 0.05] = 0.0
    A[0, 0], A[1, 1], A[2, 2], A[3, 3] = 1e-40, 3e-25, 1e17, -3e18
    buf = torch.zeros((n, m + ld_pad), dtype=torch.float32, device="cuda")
    buf[:, :m] = torch.from_numpy(A.T.copy()).cuda()
    Ad = buf[:, :m].t()
    ref = float(np.sqrt(np.sum(A.astype(np.float64) ** 2)))
    g = B.id_adaptive(Ad, 0.9, block=8, k_max=8)
    assert g.norm_A == pytest.approx(ref, rel=1e-12)
