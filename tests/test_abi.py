"""The C ABI: the library builds, loads without a GPU, and exports every
function that include/fea.h declares; host-side error paths need no device."""
import ctypes
import os
import re

import pytest

from paper_2005_05899_b300 import build, fea

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fea.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fea_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    decl = declared_functions()
    assert len(decl) >= 18
    assert sorted(fea.EXPORTED) == decl


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_create_without_device():
    lib = fea.lib()
    assert b"sm_103a" in lib.fea_version()
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    st = lib.fea_create(0, ctypes.byref(h))
    assert st == fea.ECUDA and not h.value
    with pytest.raises(fea.FeaError):
        fea.Context(0)


def test_null_arguments_rejected_without_device():
    lib = fea.lib()
    assert lib.fea_create(0, None) == fea.EINVAL
    assert lib.fea_sync_status(None, None) == fea.EINVAL
    assert lib.fea_set_wait_limit(None, 5) == fea.EINVAL
    assert lib.fea_last_error(None) == b"null context"
    lib.fea_destroy(None)
