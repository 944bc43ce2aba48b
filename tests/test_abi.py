"""CPU-side checks of the boundary: the library builds for sm_103a, loads
without a GPU, exports every function include/randid.h declares, and the
ctypes structures match the header's field lists."""
import ctypes
import re

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2310_09417_gb300 import build
    build.build()
    from paper_2310_09417_gb300 import binding
    return binding.load()


def test_exports_every_declared_function(lib):
    from paper_2310_09417_gb300 import binding
    names = binding.header_functions()
    assert set(names) >= {"id_workspace_size", "id_fixed_rank", "id_adaptive", "id_batched",
                          "cur_from_id", "id_status_string"}
    for n in names:
        assert hasattr(lib, n), "missing export %s" % n


def test_every_declared_function_has_a_signature(lib):
    """Each entry point's ctypes signature has as many arguments as the header
    prototype (an undeclared one would truncate 64-bit pointers to C ints)."""
    from paper_2310_09417_gb300 import binding
    protos = binding.header_prototypes()
    assert protos["id_quantize_fp8"] == 6 and protos["id_mlp_param_count"] == 0
    for name, nargs in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None and len(f.argtypes) == nargs, name


def _header_struct_fields(name):
    from paper_2310_09417_gb300 import binding
    text = open(binding.HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*%s;" % name, text, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)
        for part in decl.split(","):
            fields.append(re.findall(r"\w+", part)[-1])
    return fields


@pytest.mark.parametrize("cname,pyname", [("id_matrix", "IdMatrix"), ("id_opts", "IdOpts"),
                                          ("id_result", "IdResult")])
def test_struct_fields_match_header(cname, pyname):
    from paper_2310_09417_gb300 import binding
    py = [f[0] for f in getattr(binding, pyname)._fields_]
    assert py == _header_struct_fields(cname)


def test_status_strings(lib):
    from paper_2310_09417_gb300 import binding
    assert binding.status_string(0) == "ok"
    assert "NaN" in binding.status_string(binding.ERR_NONFINITE)
    assert "timed out" in binding.status_string(binding.ERR_TIMEOUT)


def test_workspace_query_without_gpu(lib):
    """Argument validation and the workspace query run on the host only."""
    from paper_2310_09417_gb300 import binding as B
    A = B.IdMatrix(1, B.F64, 1000, 300, 1000, None)
    o = B.IdOpts()
    o.sketch_prec = o.lu_prec = B.F64
    o.block = 64
    o.tol = 1e-8
    o.tol_relative = 1
    n = ctypes.c_size_t(0)
    assert lib.id_workspace_size(ctypes.byref(A), ctypes.byref(o), 0, ctypes.byref(n)) == 0
    assert n.value > 300 * 64 * 8
    o.block = 1000  # b above the supported 128
    assert lib.id_workspace_size(ctypes.byref(A), ctypes.byref(o), 0, ctypes.byref(n)) == -2
    o.block = 64
    o.lu_prec = B.F32  # F64 input with an F32 LU is not a built combination
    assert lib.id_workspace_size(ctypes.byref(A), ctypes.byref(o), 0, ctypes.byref(n)) == B.ERR_UNSUPPORTED
    bad = B.IdMatrix(1, B.F64, 1000, 300, 999, None)  # ld < m
    o.lu_prec = B.F64
    assert lib.id_workspace_size(ctypes.byref(bad), ctypes.byref(o), 0, ctypes.byref(n)) == -1
