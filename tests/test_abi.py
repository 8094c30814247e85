"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every function include/idtx.h declares, and rejects NULL arguments
before any CUDA call.  No compute calls."""
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


_CTYPES = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double, "float": ctypes.c_float}


def declared_prototypes():
    """name -> list of ctypes argument types, from the header's prototypes."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\bint\s+(idtx_[a-z0-9_]+)\s*\(([^;]*?)\)\s*;", text, flags=re.S):
        args = " ".join(m.group(2).split())
        types = []
        if args != "void":
            for a in args.split(","):
                a = a.strip()
                if "*" in a:
                    types.append(ctypes.c_void_p)
                else:
                    base = a.replace("const ", "").split()[0]
                    types.append(_CTYPES[base])
        out[m.group(1)] = types
    return out


def test_every_entry_point_rejects_null_arguments_without_touching_the_gpu(lib):
    """Argument checks come before any CUDA call: with a NULL context (or
    NULL settings for the context-free call) every entry point returns
    IDTX_EINVAL with a message; destroying a NULL context is a no-op."""
    protos = declared_prototypes()
    assert len(protos) >= 25
    lib.idtx_last_error.restype = ctypes.c_char_p
    for name, types in protos.items():
        if name == "idtx_version":
            continue
        fn = getattr(lib, name)
        fn.argtypes = types
        fn.restype = ctypes.c_int
        args = [None if t is ctypes.c_void_p else t(0) for t in types]
        rc = fn(*args)
        if name == "idtx_ctx_destroy":
            assert rc == 0
            continue
        assert rc == 1, (name, rc)                   # IDTX_EINVAL
        assert lib.idtx_last_error(), name
