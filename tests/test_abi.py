"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function include/zq.h declares (no compute call: no GPU here)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "zq.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zq_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_08427_gb300 import build

    return ctypes.CDLL(str(build.build()))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("zq_create", "zq_destroy", "zq_build_tree", "zq_build_tree_batched",
                     "zq_build_transforms", "zq_apply_Q", "zq_apply_QT", "zq_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.zq_status_string.restype = ctypes.c_char_p
    for code in range(7):
        assert lib.zq_status_string(code)


def test_null_arguments_rejected_without_gpu(lib):
    lib.zq_build_tree_batched.restype = ctypes.c_int
    assert lib.zq_build_tree_batched(None, 1, None, None, None, None, 0) == 1  # ZQ_EINVAL
    assert lib.zq_sync(None) == 1
    assert lib.zq_apply_Q(None, 0, 1, None, 0, None, 0) == 1
    lib.zq_apply_rotated.restype = ctypes.c_int
    assert lib.zq_apply_rotated(None, 0, None, None, None, None, None) == 1
    lib.zq_qgen.restype = ctypes.c_int
    lib.zq_qgen_nnz.restype = ctypes.c_int
    assert lib.zq_qgen(None, 0, None, None, None, None) == 1
    assert lib.zq_qgen_nnz(None, None) == 1
    lib.zq_set_vector_order.restype = ctypes.c_int
    assert lib.zq_set_vector_order(None, 0) == 1
    assert lib.zq_set_vector_order(None, 1) == 1


def test_binding_constants_match_the_header():
    """Every enum value and integer #define of include/zq.h has the same
    value in the binding."""
    from paper_1708_08427_gb300 import zq

    text = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "zq.h").read_text(), flags=re.S)
    values = {}
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"\b(ZQ_[A-Z0-9_]+)\s*=\s*(\d+)", body):
            values[name] = int(val)
    for name, val in re.findall(r"#define\s+(ZQ_[A-Z0-9_]+)\s+(\d+)\b", text):
        values[name] = int(val)
    assert len(values) >= 20
    for name, val in values.items():
        assert getattr(zq, name) == val, name


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1708_08427_gb300 import zq

    monkeypatch.setattr(zq, "_LIB_PATH", tmp_path / "missing.so")
    monkeypatch.setattr(zq, "_L", None)
    with pytest.raises(ImportError):
        zq._lib()
