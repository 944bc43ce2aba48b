"""The failure handling on the GPU: a device wait that nothing can satisfy
gives up after its bounded time, the call returns ID_ERR_TIMEOUT, and the CUDA
context stays usable.  The waits are the library's own: the LUPP panel's grid
barrier and the tensor-core kernels' mbarrier wait.  Each gives up after 4 s of
the GPU's global timer.  No fault, trap or unbounded wait is involved.  The
file is named to be collected last."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("which", [0, 1], ids=["grid_barrier", "mbarrier"])
def test_unsatisfied_wait_times_out_and_the_context_survives(B, which):
    t0 = time.perf_counter()
    assert B.selftest_timeout(which) == B.ERR_TIMEOUT
    waited = time.perf_counter() - t0
    assert 3.0 < waited < 60.0, waited
    # the context still runs an ID afterwards
    from paper_2310_09417_gb300 import workloads as W
    A = W.spectral_matrix(300, 200, W.spectrum("geometric", 200), seed=5)
    r = B.id_adaptive(B.colmajor(torch.from_numpy(A).cuda()), 1e-6, block=16, seed=1)
    assert r.status == B.OK and 0 < r.k < 200
    err = np.linalg.norm(A - A[:, r.J.cpu().numpy()] @ r.X.cpu().numpy()) / np.linalg.norm(A)
    assert err < 1e-5
