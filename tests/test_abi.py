"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
and exports every function include/idtx.h declares.  No compute calls."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "idtx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(idtx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1807_10459_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("idtx_ctx_create", "idtx_ctx_destroy", "idtx_last_error", "idtx_cmi_ksg",
                     "idtx_cmi_batch", "idtx_mte_step", "idtx_mte_select_target"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(lib):
    lib.idtx_version.restype = ctypes.c_int
    assert lib.idtx_version() >= 100
    lib.idtx_last_error.restype = ctypes.c_char_p
    assert lib.idtx_last_error() is not None


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1807_10459_gb300 as m
    monkeypatch.setattr(m, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(m, "_lib", None)
    with pytest.raises(RuntimeError):
        m.load()
