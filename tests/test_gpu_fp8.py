"""GPU tests of the FP8 path: A stored in E4M3 with one FP32 scale per 128-row
block of each column, the sketch on the tensor cores (kind::f8f6f4, FP32
accumulation), LUPP and X in FP32, norms in FP64.

The E4M3 format is decoded here from its definition (sign, 4-bit exponent with
bias 7, 3-bit mantissa, subnormals at exponent 0, NaN at S.1111.111, no
infinities, largest finite 448); the oracle runs in FP64 on the decoded values.
"""
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


def e4m3_table():
    v = np.empty(256)
    for c in range(256):
        sgn = -1.0 if c & 0x80 else 1.0
        e, f = (c >> 3) & 0xF, c & 7
        if e == 15 and f == 7:
            v[c] = np.nan
        elif e == 0:
            v[c] = sgn * (f / 8.0) * 2.0 ** -6
        else:
            v[c] = sgn * (1.0 + f / 8.0) * 2.0 ** (e - 7)
    return v


TABLE = e4m3_table()
POS = TABLE[:127]  # codes 0x00..0x7E: the non-negative finite values, increasing


def encode(x):
    """Nearest E4M3 code (ties to the even code), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    hi = np.clip(np.searchsorted(POS, a), 1, 126)
    lo = hi - 1
    dlo, dhi = a - POS[lo], POS[hi] - a
    code = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    code = np.where(a >= 448.0, 126, code)
    code = np.where(a == 0.0, 0, code)
    return (code | np.where(np.signbit(x), 0x80, 0)).astype(np.uint8)  # negatives keep the sign, also at 0


def decode(codes):
    return TABLE[np.asarray(codes, dtype=np.uint8)]


def codes_of(A8):
    """(m x n) uint8 codes of an FP8Matrix (column-major device data)."""
    return A8.data.view(torch.uint8).cpu().numpy()


def dequantize(A8):
    q = decode(codes_of(A8))
    s = A8.scale.cpu().numpy().astype(np.float64)
    return q * np.repeat(s, 128, axis=0)[: q.shape[0]]


def omega_fp8(B, Om_f64):
    """Caller Omega as E4M3 device rows with a 16-byte aligned row stride."""
    rows, m = Om_f64.shape
    codes = encode(Om_f64)
    ld = -(-m // 16) * 16
    buf = torch.zeros((rows, ld), dtype=torch.uint8, device="cuda")
    buf[:, :m] = torch.from_numpy(codes).cuda()
    return buf.view(torch.float8_e4m3fn)[:, :m], decode(codes)


def test_encoder_pins():
    assert TABLE[0x7E] == 448.0 and np.isnan(TABLE[0x7F]) and TABLE[0x01] == 2.0 ** -9
    assert TABLE[0x38] == 1.0 and TABLE[0xB8] == -1.0
    assert encode(1.0625) == 0x38          # tie between 1 (even code) and 1.125
    assert encode(1.1875) == 0x3A          # tie between 1.125 and 1.25 (even code 0x3A)
    assert encode(1e6) == 0x7E and encode(-1e6) == 0xFE
    assert encode(-1e-5) == 0x80 and encode(0.0) == 0x00  # round to a signed zero
    vals = TABLE[~np.isnan(TABLE)]
    assert np.array_equal(decode(encode(vals)), vals)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("pow2", [True, False])
def test_quantize_matches_definition(B, dtype, pow2):
    rng = np.random.default_rng(3)
    m, n = 300, 7  # 3 blocks, the last one ragged
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-20, 21, size=n))[None, :]
    A[128:256, 2] = 0.0  # a zero block
    A[5, 4] = 1e4        # one large entry sets its block's scale
    Ad = B.colmajor(torch.from_numpy(A).to("cuda", dtype))
    A8 = B.quantize_fp8(Ad, pow2=pow2)
    Ah = Ad.double().cpu().numpy()  # the values the kernel read
    nbs = -(-m // 128)
    S = A8.scale.cpu().numpy()
    Q = codes_of(A8)
    for j in range(n):
        for kb in range(nbs):
            blk = Ah[kb * 128:(kb + 1) * 128, j]
            amax = np.float32(np.abs(blk).max())
            if amax == 0:
                assert S[kb, j] == 1.0
                assert np.all(Q[kb * 128:(kb + 1) * 128, j] == 0)
                continue
            s = np.float32(amax / np.float32(448.0))
            if pow2:
                fr, ex = np.frexp(s)
                s = np.float32(2.0 ** (ex - 1 if fr == 0.5 else ex))
            assert S[kb, j] == s, (j, kb, S[kb, j], s)
            if dtype == torch.float64:
                x = blk / np.float64(s)
            else:
                x = (blk.astype(np.float32) / s).astype(np.float64)
            np.testing.assert_array_equal(Q[kb * 128:(kb + 1) * 128, j], encode(x))


@pytest.mark.parametrize("m,n,rows", [
    (1024, 256, 64),     # whole tiles
    (1000, 333, 100),    # ragged K (not a multiple of the 128-row block), n and rows
    (129, 70, 33),       # one full block and one of a single row
    (8, 5, 3),           # smaller than every tile
    (40000, 300, 64),    # long K: many blocks and split-K partials
])
def test_fp8_sketch_matches_product(B, m, n, rows):
    rng = np.random.default_rng(m + n + rows)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-4, 5, size=(1, n)))
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    Om8, Om = omega_fp8(B, rng.standard_normal((rows, m)))
    G = B.id_sketch(A8, Om8).double().cpu().numpy()
    Ad = dequantize(A8)
    ref = (Om @ Ad).T
    scale = (np.abs(Om) @ np.abs(Ad)).T
    # products are exact; the FP32 sums per block and across blocks round
    err = (np.abs(G - ref) / np.maximum(scale, 1e-300)).max()
    assert err < 2.0 ** -12, err


def test_fp8_wide_pass_equals_block_passes(B):
    """A pass of several blocks (one CTA runs one N = 256 MMA per scale block over
    four 64-row blocks of Omega, two accumulators of 256 columns, eight epilogue
    warps) gives every entry the same bits as passes of one block: the block sums,
    their scaling and their order do not change (K = 1024: eight scale blocks, one
    split for both; n and the last group of rows ragged)."""
    rng = np.random.default_rng(9)
    m, n, rows = 1024, 700, 600
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-4, 5, size=(1, n)))
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    Om8, _ = omega_fp8(B, rng.standard_normal((rows, m)))
    G = B.id_sketch(A8, Om8)
    for r0 in range(0, rows, 64):
        g = B.id_sketch(A8, Om8[r0:r0 + 64])
        assert torch.equal(G[:, r0:r0 + 64], g), r0


def test_fp8_pass_size_does_not_change_result(B):
    """Adaptive FP8 runs with eight blocks per pass (the default), one block per
    pass or a rank guess return the same J, X and k bit for bit."""
    m, n, b = 6016, 1500, 64
    A = lowrank(m, n, 300, 1e-3, 8)
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    base = B.id_adaptive(A8, 5e-2, block=b, seed=4, blocks_per_pass=1)
    for kw in (dict(), dict(k0=400), dict(blocks_per_pass=3)):
        g = B.id_adaptive(A8, 5e-2, block=b, seed=4, **kw)
        assert g.k == base.k and torch.equal(g.J, base.J) and torch.equal(g.X, base.X), kw


def test_fp8_gaussian_rows_round_the_fp64_generator(B, orc):
    """E4M3 rows: the same counters and Box-Muller map, evaluated in FP32 on the
    leading 24 bits.  Against the FP64 generator rounded to E4M3: the same codes
    except where the two evaluations straddle a rounding boundary (one step)."""
    g = B.gaussian_rows(99, 3, 64, 4099, dtype=torch.float8_e4m3fn).view(torch.uint8).cpu().numpy()
    o = encode(orc.gaussian_rows(99, 3, 64, 4099))
    diff = decode(g) != decode(o)
    assert diff.mean() < 1e-3
    # a straddled boundary moves the value to a neighbouring code of the same sign
    assert np.all(np.abs(g[diff].astype(int) - o[diff].astype(int)) == 1)


def lowrank(m, n, r, noise, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) + noise * rng.standard_normal((m, n))


@pytest.mark.parametrize("tol", [5e-2, 1e-1])
def test_fp8_adaptive_against_fp64_oracle(B, orc, tol):
    """The low-rank-plus-noise family stored in FP8: the ID of the stored matrix
    (its decoded values, exact in FP64) by the FP8-sketch / FP32-LU path meets the
    tolerance, its rank is within one block of the FP64 oracle's on the same
    values and the same Omega, and its error is within 1.2x of the oracle's at
    the smaller of the two ranks.  The tolerances sit above the E4M3 rounding
    floor (about 2.6e-2 relative)."""
    m, n, r, b = 4096, 1024, 150, 32
    A = lowrank(m, n, r, 1e-4, 31)
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    Ad = dequantize(A8)
    Om8, Om = omega_fp8(B, W.gaussian_omega(32, orc.rows_needed(n, b, m=m), m))
    g = B.id_adaptive(A8, tol, block=b, omega=Om8)
    assert g.status == 0
    r0 = orc.id_adaptive(Ad, Om, b, tol * orc.fro_norm(Ad))
    assert abs(g.k - r0["k"]) <= b
    nA = orc.fro_norm(Ad)
    eg = orc.id_residual(Ad, g.J.cpu().numpy(), g.X.cpu().numpy().astype(np.float64)) / nA
    eo = oracle_error_at_rank(orc, Ad, Om, r0, min(g.k, r0["k"]), b) / nA
    assert eg <= 1.2 * eo + 1e-6
    assert eg <= 3 * tol
    assert g.norm_A == pytest.approx(nA, rel=1e-12)
    # against the unquantised matrix the FP8 storage error adds on top
    e_orig = orc.id_residual(A, g.J.cpu().numpy(), g.X.cpu().numpy().astype(np.float64)) / orc.fro_norm(A)
    assert e_orig <= eg + 0.05


def test_fp8_generated_omega_matches_oracle_generator(B, orc):
    """Omega drawn on the device in E4M3 (the FP64 Philox/Box-Muller rows rounded
    to nearest even): the oracle on the oracle generator's rows, rounded here the
    same way, finds the rank within one block, and the GPU's error is within 1.2x of
    the oracle's at the smaller of the two ranks."""
    m, n, b, tol, seed = 2048, 512, 32, 1e-1, 5
    A = lowrank(m, n, 60, 1e-4, 7)
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    g = B.id_adaptive(A8, tol, block=b, seed=seed)
    Ad = dequantize(A8)
    Om = decode(encode(orc.gaussian_rows(seed, 0, orc.rows_needed(n, b, m=m), m)))
    r0 = orc.id_adaptive(Ad, Om, b, tol * orc.fro_norm(Ad))
    nA = orc.fro_norm(Ad)
    e = orc.id_residual(Ad, g.J.cpu().numpy(), g.X.cpu().numpy().astype(np.float64)) / nA
    eo = oracle_error_at_rank(orc, Ad, Om, r0, min(g.k, r0["k"]), b) / nA
    assert g.status == 0 and abs(g.k - r0["k"]) <= b
    assert e <= 1.2 * eo + 1e-6 and e <= 3 * tol


def test_fp8_requires_scales_and_alignment(B):
    A = torch.zeros((100, 20), dtype=torch.uint8, device="cuda").view(torch.float8_e4m3fn)
    Ac = B.colmajor(A)  # ld = 100: not a multiple of 16
    sc = torch.ones((20, 1), dtype=torch.float32, device="cuda").t()
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(B.FP8Matrix(Ac, sc), 1e-1)
    assert e.value.code == B.ERR_UNSUPPORTED
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(B.colmajor_padded(A, 16), 1e-1)  # no block scales
    assert e.value.code == -1


def test_fp8_nonfinite_scale_is_rejected(B):
    A = B.colmajor(torch.randn(256, 40, dtype=torch.float32, device="cuda"))
    A[3, 7] = float("nan")
    A8 = B.quantize_fp8(A)
    assert torch.isnan(A8.scale[0, 7])
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(A8, 1e-1)
    assert e.value.code == B.ERR_NONFINITE


def test_fp8_fixed_rank_against_oracle(B, orc):
    """randLUPP at fixed rank on the FP8 path: the first pivots (well separated)
    equal the FP64 oracle's on the decoded values and the same Omega, and the
    rank-k error is within 1.2x of the oracle's."""
    m, n, k, l = 2048, 700, 40, 48
    A = lowrank(m, n, 30, 1e-3, 12)
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
    Ad = dequantize(A8)
    Om8, Om = omega_fp8(B, W.gaussian_omega(8, l, m))
    g = B.id_fixed_rank(A8, k, l, block=16, omega=Om8)
    r = orc.id_fixed_rank(Ad, Om, k)
    assert np.array_equal(g.J.cpu().numpy()[:10], r["J"][:10])
    nA = orc.fro_norm(Ad)
    eg = orc.id_residual(Ad, g.J.cpu().numpy(), g.X.cpu().numpy().astype(np.float64)) / nA
    eo = orc.id_residual(Ad, r["J"], r["X"]) / nA
    assert eg <= 1.2 * eo + 1e-6


@pytest.mark.parametrize("path", ["f64", "f32", "bf16", "fp8", "f64emu"])
def test_sketch_into_padded_rows(B, path):
    """id_sketch writes G with a row stride larger than its row count on every
    path (the split-K partials keep their own stride)."""
    rng = np.random.default_rng(5)
    m, n, rows, ldg = 3000, 300, 40, 56
    A = rng.standard_normal((m, n))
    Om = rng.standard_normal((rows, m))
    kw = {}
    if path == "f64":
        Ad, Od = B.colmajor(torch.from_numpy(A).cuda()), torch.from_numpy(Om).cuda()
    elif path == "f64emu":
        Om = np.clip(np.rint(Om * 1024.0), -8127.0, 8127.0) / 1024.0
        Ad, Od = B.colmajor(torch.from_numpy(A).cuda()), torch.from_numpy(Om).cuda()
        kw = dict(sketch_prec=B.F64_EMU)
    elif path == "f32":
        Ad = B.colmajor(torch.from_numpy(A).to("cuda", torch.float32))
        Od = torch.from_numpy(Om).to("cuda", torch.float32)
    elif path == "bf16":
        Ad = B.colmajor(torch.from_numpy(A).to("cuda", torch.bfloat16))
        Od = torch.from_numpy(Om).to("cuda", torch.bfloat16).contiguous()
    else:
        Ad = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()))
        Od, Om = omega_fp8(B, Om)
    ref = B.id_sketch(Ad, Od, **kw)
    G = torch.full((n, ldg), float("nan"), dtype=ref.dtype, device="cuda")
    lib = B.load()
    import ctypes
    prec = (B.F64_EMU if path == "f64emu" else B._TORCH_TO_ID[Ad.dtype])
    nb = ctypes.c_size_t(0)
    assert lib.id_sketch_workspace_size(ctypes.byref(B._matrix(Ad)), rows, prec, ctypes.byref(nb)) == 0
    ws = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device="cuda")
    rc = lib.id_sketch(ctypes.byref(B._matrix(Ad)), Od.data_ptr(), Od.stride(0), rows, prec, G.data_ptr(), ldg,
                       ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(G[:, :rows], ref)
    assert torch.isnan(G[:, rows:]).all()  # the padding is not written


@pytest.mark.parametrize("m,n", [(1000, 37), (4099, 20), (16, 3)])
def test_fp8_norm_matches_fp64_sum_of_squares(B, m, n):
    """||A||_F of the stored FP8 matrix (vectors of 16 codes summed in float-float,
    scaled in FP64) against the FP64 sum of squares of the decoded values; rows
    not a multiple of 16 (the last vector masked), scales spanning 2^-40 .. 2^40."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-40, 41, size=n))[None, :]
    A[rng.random((m, n)) < 0.05] = 0.0
    A8 = B.quantize_fp8(B.colmajor(torch.from_numpy(A).cuda()), pow2=1)
    Ad = dequantize(A8)
    g = B.id_adaptive(A8, 0.5, block=16, k_max=16)
    ref = np.sqrt(np.sum(Ad * Ad))
    assert g.norm_A == pytest.approx(ref, rel=1e-12)


def test_fp8_nan_code_is_rejected(B):
    A8 = B.quantize_fp8(B.colmajor(torch.randn(300, 20, dtype=torch.float32, device="cuda")))
    codes = A8.data.view(torch.uint8)
    codes[257, 5] = 0x7F  # S.1111.111: NaN, in the masked last vector of the column
    with pytest.raises(B.IDError) as e:
        B.id_adaptive(A8, 1e-1)
    assert e.value.code == B.ERR_NONFINITE
