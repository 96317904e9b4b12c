"""The C-ABI library loads on a machine without a GPU and exports every
function include/airgs.h declares; the Python binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(path):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(airgs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2512_20943_b300 import build
    return build.build()


def test_library_exports_every_declared_function(lib_path):
    names = header_functions(os.path.join(ROOT, "include", "airgs.h"))
    assert len(names) >= 20
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_header(lib_path):
    from paper_2512_20943_b300 import _abi
    names = header_functions(os.path.join(ROOT, "include", "airgs.h"))
    assert sorted(_abi.SIGNATURES) == names
    _abi.load_library()  # resolves every symbol with its signature


def test_binding_constants_equal_the_header():
    """Every integer constant the header defines has the same value in the binding."""
    from paper_2512_20943_b300 import _abi
    text = open(os.path.join(ROOT, "include", "airgs.h")).read()
    consts = dict(re.findall(r"#define\s+(AIRGS_[A-Z0-9_]+)\s+(\(?-?[0-9][0-9 <()-]*\)?)", text))
    assert {"AIRGS_E_ARG", "AIRGS_PROFILE_BLEND", "AIRGS_MAX_VIEWS"} <= set(consts)
    for name, expr in consts.items():
        assert getattr(_abi, name) == eval(expr, {}), name  # plain integer literals and shifts only


def test_shape_table_without_gpu(lib_path):
    """Shape 0 is the default; every shape has a distinct name naming its
    forward and backward (batch/warps), the sort's keys per thread and the
    emission's instances per thread."""
    from paper_2512_20943_b300 import _abi
    lib = _abi.load_library()
    n = lib.airgs_shape_count()
    names = [lib.airgs_shape_name(i).decode() for i in range(n)]
    assert n == 225 and len(set(names)) == n
    assert names[0] == "fwd 32/28 bwd 32/32 keys 8 run 8"
    assert lib.airgs_shape_name(n) == b"" and lib.airgs_shape_name(-1) == b""


def test_create_without_gpu_fails_cleanly(lib_path):
    """Without a device airgs_create reports an error code instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2512_20943_b300 import _abi
    lib = _abi.load_library()
    ctx = ctypes.c_void_p()
    assert lib.airgs_create(ctypes.byref(ctx), None, None) != 0
