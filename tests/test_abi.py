"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/sem.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_05136_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2205_05136_gb300 import capi
    assert sorted(capi.EXPORTS) == _declared()
    for n in capi.EXPORTS:
        assert callable(getattr(capi, n))


def test_version_string(lib):
    lib.sem_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sem_version()


def test_argument_errors_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    from paper_2205_05136_gb300 import capi
    L = capi.lib()
    out = ctypes.c_void_p()
    v = (ctypes.c_double * 24)()
    assert L.sem_create(ctypes.byref(out), 0, 1, 1, v, 2, 1, 0) == capi.SEM_ERR_ARG
    assert L.sem_create(ctypes.byref(out), 1, 1, 1, v, 7, 1, 0) == capi.SEM_ERR_ARG
    assert L.sem_create(ctypes.byref(out), 1, 1, 1, v, 2, 5, 0) == capi.SEM_ERR_ARG
    assert L.sem_create(ctypes.byref(out), 1, 1, 1, None, 2, 1, 0) == capi.SEM_ERR_ARG
    assert b"vertices" in L.sem_last_error(None)
    assert L.sem_destroy(None) == capi.SEM_OK
    assert L.sem_num_dofs(None, None) == capi.SEM_ERR_ARG


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2205_05136_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libsem.so the binding raises; it has no CPU fallback."""
    from paper_2205_05136_gb300 import capi
    monkeypatch.setattr(capi, "_LIB", None)
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "libsem.so"))
    with pytest.raises(ImportError):
        capi.lib()


def test_binding_rejects_host_and_mistyped_tensors():
    """The binding checks vectors before any library call: CUDA memory,
    contiguous, the right dtype and length."""
    import torch
    from paper_2205_05136_gb300 import capi
    with pytest.raises(TypeError, match="CUDA tensor"):
        capi._dev(torch.zeros(4, dtype=torch.float64), torch.float64, 4, "u")
    with pytest.raises(TypeError, match="CUDA tensor"):
        capi._dev([0.0] * 4, torch.float64, 4, "u")
    with pytest.raises(ValueError, match="vertices"):
        capi.sem_create(1, 1, 1, [0.0] * 23, 2, 1)
