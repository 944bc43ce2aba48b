"""Batched IDs: many independent problems in one persistent launch.

Each problem's result must be the single-problem path's (same Gaussian rows,
same block size): same rank, same skeletons, X equal to rounding; and against
the CPU oracle the skeletons match and A(:,J) X agrees within 1e-10."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2310_09417_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


def kernel_blocks(count, seed, n_points=20000, leaf_max=256, size_min=32):
    pts, leaves, pairs = W.kernel_block_pairs(n_points, count, seed, leaf_max=leaf_max, size_min=size_min)
    return [W.gaussian_kernel_block(pts, leaves[a], leaves[b], h=0.3) for a, b in pairs]


def to_dev(A, dtype=torch.float64):
    from paper_2310_09417_gb300 import binding
    return binding.colmajor(torch.from_numpy(A).to("cuda", dtype))


def test_batched_equals_single_problem_path(B):
    blocks = kernel_blocks(48, seed=1)
    As = [to_dev(A) for A in blocks]
    res = B.id_batched(As, 1e-8, block=16, seed=77)
    assert len(res) == len(As)
    for A, r in zip(As, res):
        s = B.id_adaptive(A, 1e-8, block=16, seed=77)
        assert r.status == s.status
        assert r.k == s.k and r.rounds == s.rounds
        assert torch.equal(r.J, s.J)
        rel = float(torch.linalg.norm(r.X - s.X) / torch.linalg.norm(s.X))
        assert rel <= 1e-8, rel
        assert r.est_err == pytest.approx(s.est_err, rel=1e-6, abs=1e-13 * s.norm_A)


def test_batched_against_oracle(B, orc):
    blocks = kernel_blocks(6, seed=2, n_points=8000, leaf_max=200)
    As = [to_dev(A) for A in blocks]
    b, tol, seed = 16, 1e-6, 5
    res = B.id_batched(As, tol, block=b, seed=seed)
    for A, r in zip(blocks, res):
        m, n = A.shape
        Om = orc.gaussian_rows(seed, 0, orc.rows_needed(n, b, m=m), m)
        o = orc.id_adaptive(A, Om, b, tol * orc.fro_norm(A))
        assert r.k == o["k"]
        assert np.array_equal(r.J.cpu().numpy(), o["J"])
        Xg = r.X.cpu().numpy()
        nA = np.linalg.norm(A)
        assert np.linalg.norm(A[:, o["J"]] @ (Xg - o["X"])) / nA <= 1e-10


def test_batched_fp32(B, orc):
    """FP32 problems against the FP64 oracle run on the FP32-rounded blocks with the
    same counter-based Gaussian rows: the rank within one block of the oracle's,
    the leading skeletons identical, and the achieved error within 1.2 x the
    oracle's at the smaller of the two ranks (as the single-problem FP32 tests)."""
    from idcheck import oracle_error_at_rank
    blocks = kernel_blocks(24, seed=3)
    As = [to_dev(A, torch.float32) for A in blocks]
    b, tol, seed = 32, 1e-4, 9
    res = B.id_batched(As, tol, block=b, seed=seed)
    for A, r in zip(blocks, res):
        A32 = A.astype(np.float32).astype(np.float64)
        m, n = A32.shape
        Om = orc.gaussian_rows(seed, 0, orc.rows_needed(n, b, m=m), m)
        o = orc.id_adaptive(A32, Om, b, tol * orc.fro_norm(A32))
        assert r.status in (0, B.WARN_TOL_NOT_MET)
        assert abs(r.k - o["k"]) <= b
        kk = min(r.k, o["k"])
        J = r.J.cpu().numpy()
        # the leading pivots are far apart (kernel blocks decay fast); later ones near
        # the FP32 rounding level may legitimately differ, which the error check covers
        assert np.array_equal(J[:8], o["J"][:8])
        e = orc.id_residual(A32, J, r.X.double().cpu().numpy())
        eo = oracle_error_at_rank(orc, A32, Om, o, kk, b)
        assert e <= 1.2 * eo + 1e-6 * orc.fro_norm(A32), (e, eo)


def test_batched_concurrent_host_threads(B):
    """Two host threads calling id_batched at once (own streams and workspaces)
    share the graph and autotuner caches: the results equal the sequential ones."""
    import threading
    sets = [[to_dev(A) for A in kernel_blocks(12, seed=s)] for s in (11, 12)]
    ref = [B.id_batched(As, 1e-8, block=16, seed=4) for As in sets]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out = [None, None]
    err = []

    def run(i):
        try:
            for _ in range(5):
                out[i] = B.id_batched(sets[i], 1e-8, block=16, seed=4, stream=streams[i])
        except Exception as e:  # reported in the main thread
            err.append(e)
    th = [threading.Thread(target=run, args=(i,)) for i in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not err, err
    for i in (0, 1):
        for a, c in zip(ref[i], out[i]):
            assert a.k == c.k and torch.equal(a.J, c.J) and torch.equal(a.X, c.X)


@pytest.mark.parametrize("cfg", ["32x1", "32x2", "64x1", "64x2"])
def test_batched_result_independent_of_tuned_configuration(B, cfg):
    blocks = kernel_blocks(20, seed=4)
    As = [to_dev(A) for A in blocks]
    os.environ.pop("RANDID_BATCHED_CONFIG", None)
    ref = B.id_batched(As, 1e-8, block=16, seed=3)
    os.environ["RANDID_BATCHED_CONFIG"] = cfg
    try:
        got = B.id_batched(As, 1e-8, block=16, seed=3)
    finally:
        os.environ.pop("RANDID_BATCHED_CONFIG", None)
    for a, b_ in zip(ref, got):
        assert a.k == b_.k
        assert torch.equal(a.J, b_.J)
        assert torch.equal(a.X, b_.X)


def test_batched_nonfinite_problem_is_isolated(B):
    blocks = kernel_blocks(5, seed=5)
    blocks[2] = blocks[2].copy()
    blocks[2][3, 4] = np.nan
    As = [to_dev(A) for A in blocks]
    res = B.id_batched(As, 1e-6, block=16)
    assert res[2].status == B.ERR_NONFINITE and res[2].k == 0
    for i in (0, 1, 3, 4):
        assert res[i].status >= 0 and res[i].k > 0


def test_batched_graph_replay_and_uneven_sizes(B):
    rng = np.random.default_rng(6)
    As = []
    for m, n in [(64, 1000), (1000, 64), (300, 257), (17, 9), (512, 512)]:
        As.append(to_dev(rng.standard_normal((m, n)) @ np.diag(0.5 ** np.arange(n))))
    ws = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")
    r1 = B.id_batched(As, 1e-6, block=32, seed=1, workspace=ws)
    r2 = B.id_batched(As, 1e-6, block=32, seed=1, workspace=ws)  # replays the cached graph
    for i, (a, b_) in enumerate(zip(r1, r2)):
        assert a.k == b_.k and torch.equal(a.J, b_.J) and torch.equal(a.X, b_.X)
        s = B.id_adaptive(As[i], 1e-6, block=32, seed=1)
        assert a.k == s.k and torch.equal(a.J, s.J)


def test_batched_rejects_too_wide_problem(B):
    A = torch.zeros((10, 5000), dtype=torch.float64, device="cuda")
    with pytest.raises(B.IDError) as e:
        B.id_batched([B.colmajor(A)], 1e-3)
    assert e.value.code == -2
