"""id_fixed_rank_noalloc: the fixed-rank column ID for callers that cannot
allocate device memory (an application that has reserved the GPU's memory for
its own pool, or a loop whose rules forbid device allocation after start-up).
It runs on the library's static device buffer, so its results must be those of
id_fixed_rank with a caller workspace.  Two different problems back to back
check that what a previous call left in the shared buffer does not leak into
the next.  The file is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

X_TOL = 1e-10


def _noalloc(lib):
    from paper_2310_09417_gb300 import binding as B
    f = lib.id_fixed_rank_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    del B
    return f


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import binding as B
    from paper_2310_09417_gb300 import build
    from paper_2310_09417_gb300 import workloads as W
    build.build()
    lib = B.load()
    f = _noalloc(lib)
    stream = torch.cuda.current_stream().cuda_stream

    cases = [(2000, 2000, 100, 120, 64, 21), (777, 555, 37, 45, 16, 22)]
    for m, n, k, l, b, seed in cases:
        A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n)), seed=seed)
        Ad = B.colmajor(torch.from_numpy(A).to("cuda"))
        ref = B.id_fixed_rank(Ad, k, l, block=b, seed=seed)  # caller-workspace entry point
        J = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        Xb = torch.full((n, k), float("nan"), dtype=torch.float64, device="cuda")
        res = B.IdResult()
        res.J, res.X, res.ldx = J.data_ptr(), Xb.data_ptr(), k
        opts = B._opts(Ad, block=b, tol=0.0, relative=False, k_max=k, k0=0, blocks_per_pass=1,
                       seed=seed, omega=None, profile=False)
        rc = f(ctypes.byref(B._matrix(Ad)), k, l, ctypes.byref(opts), ctypes.byref(res), stream)
        assert rc == B.OK, B.status_string(rc)
        assert res.k == k
        assert torch.equal(J, ref.J)
        X = Xb.t()
        rel = float(torch.linalg.norm(X - ref.X) / torch.linalg.norm(ref.X))
        assert rel <= X_TOL
        assert res.est_err == pytest.approx(ref.est_err, rel=1e-12)

    # the defining property: once the first call has loaded the buffer on this
    # device, a call allocates no device memory (free bytes unchanged)
    m, n, k, l, b, seed = cases[0]
    A = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n)), seed=seed)
    Ad = B.colmajor(torch.from_numpy(A).to("cuda"))
    J = torch.empty((k,), dtype=torch.int64, device="cuda")
    Xb = torch.empty((n, k), dtype=torch.float64, device="cuda")
    res = B.IdResult()
    res.J, res.X, res.ldx = J.data_ptr(), Xb.data_ptr(), k
    opts = B._opts(Ad, block=b, tol=0.0, relative=False, k_max=k, k0=0, blocks_per_pass=1,
                   seed=seed, omega=None, profile=False)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc = f(ctypes.byref(B._matrix(Ad)), k, l, ctypes.byref(opts), ctypes.byref(res), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == B.OK, B.status_string(rc)
    assert free1 == free0, "the call changed free device memory by %d bytes" % (free0 - free1)

    # a problem whose scratch exceeds the static buffer is refused before anything runs
    big = B.IdMatrix(Ad.data_ptr(), B.F64, 40000, 10000, 40000, None)
    opts = B._opts(Ad, block=64, tol=0.0, relative=False, k_max=100, k0=0, blocks_per_pass=1, seed=1,
                   omega=None, profile=False)
    res = B.IdResult()
    res.J, res.X, res.ldx = J.data_ptr(), Xb.data_ptr(), 100
    assert f(ctypes.byref(big), 100, 120, ctypes.byref(opts), ctypes.byref(res), stream) == B.ERR_WORKSPACE
