"""CPU checks of the binding's argument validation: buffers that the library
would write or read past are refused in Python, before anything reaches the
device.  The checks read only tensor metadata, so CPU tensors stand in for
device ones here (with the CPU as the expected device)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2310_09417_gb300 import binding as B  # noqa: E402

CPU = torch.device("cpu")


def test_out_buffers_of_the_right_size_pass():
    n, kmax = 50, 12
    J = torch.empty(kmax, dtype=torch.int64)
    B._check_out(J, torch.empty((n, kmax), dtype=torch.float64), n, kmax, torch.float64, CPU, "t")
    # larger buffers and a wider row stride are fine
    B._check_out(torch.empty(kmax + 3, dtype=torch.int64), torch.empty((n + 2, kmax + 5), dtype=torch.float64),
                 n, kmax, torch.float64, CPU, "t")
    wide = torch.empty((n, kmax + 7), dtype=torch.float32)[:, :kmax]
    B._check_out(J, wide, n, kmax, torch.float32, CPU, "t")


@pytest.mark.parametrize("case", ["short_J", "J_dtype", "X_rows", "X_cols", "X_transposed", "X_dtype",
                                  "J_strided"])
def test_out_buffers_too_small_or_misshaped_are_refused(case):
    n, kmax = 50, 12
    J = torch.empty(kmax, dtype=torch.int64)
    X = torch.empty((n, kmax), dtype=torch.float64)
    if case == "short_J":
        J = J[: kmax - 1]
    elif case == "J_dtype":
        J = J.to(torch.int32)
    elif case == "X_rows":
        X = X[: n - 1]
    elif case == "X_cols":
        X = X[:, : kmax - 1]
    elif case == "X_transposed":
        X = torch.empty((kmax, n), dtype=torch.float64).t()
    elif case == "X_dtype":
        X = X.float()
    elif case == "J_strided":
        J = torch.empty(2 * kmax, dtype=torch.int64)[::2]
    with pytest.raises(ValueError):
        B._check_out(J, X, n, kmax, torch.float64, CPU, "t")


def test_tensor_check():
    B._check_tensor(torch.zeros(10, dtype=torch.float32), "v", CPU, torch.float32, 10)
    with pytest.raises(ValueError):
        B._check_tensor(torch.zeros(9, dtype=torch.float32), "v", CPU, torch.float32, 10)
    with pytest.raises(ValueError):
        B._check_tensor(torch.zeros(10, dtype=torch.float64), "v", CPU, torch.float32, 10)
    with pytest.raises(ValueError):
        B._check_tensor([0.0] * 10, "v", CPU, torch.float32, 10)


def test_mlp_arguments():
    p = torch.zeros(B.mlp_param_count(), dtype=torch.float32)
    B._check_mlp(p, torch.zeros((4, B.MLP_IN), dtype=torch.float32))
    for x in (torch.zeros((4, B.MLP_IN - 1)), torch.zeros((0, B.MLP_IN)), torch.zeros(B.MLP_IN),
              torch.zeros((4, B.MLP_IN), dtype=torch.float64)):
        with pytest.raises(ValueError):
            B._check_mlp(p, x)
    with pytest.raises(ValueError):
        B._check_mlp(p[:-1], torch.zeros((4, B.MLP_IN)))


def test_workspace_reuse_needs_contiguous_bytes():
    ws = torch.empty(4096, dtype=torch.uint8)
    assert B._workspace(1000, CPU, ws) is ws
    strided = ws[::2]  # 2048 entries, not contiguous: a fresh buffer instead
    assert B._workspace(1000, CPU, strided) is not strided
    assert B._workspace(1000, CPU, torch.empty(1024, dtype=torch.float64)) is not ws
