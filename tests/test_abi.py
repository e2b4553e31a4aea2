"""The C ABI library builds, loads, and exports every entry point that
include/eeid.h declares; argument errors are reported without a GPU.  CPU only
(no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2002_04989_gb300 import build as eeid_build
from paper_2002_04989_gb300 import eeid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(eeid_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    return eeid.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("eeid_eigvals", "eeid_minor_eigvals", "eeid_components", "eeid_ctx_create",
                     "eeid_sync", "eeid_components_batched", "eeid_components_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", eeid_build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_every_symbol():
    assert declared_functions() <= set(eeid.SIGNATURES)


def test_invalid_arguments_without_gpu(lib):
    # a NULL context is rejected before any CUDA call
    vp = ctypes.c_void_p
    st = lib.eeid_components(None, None, 4, 4, None, 4, None, 4, None, None, None)
    assert st == eeid.EEID_ERR_INVALID
    assert "context" in eeid.last_error()
    assert lib.eeid_ctx_create(0, 0, None) == eeid.EEID_ERR_INVALID
    assert lib.eeid_sync(None, None) == eeid.EEID_ERR_INVALID
    assert lib.eeid_launch_count(None) == 0


def test_ctx_create_reports_missing_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.eeid_ctx_create(0, 0, ctypes.byref(h))
    assert st == eeid.EEID_ERR_CUDA
    assert h.value is None


def test_server_create_reports_missing_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.eeid_server_create(0, None, ctypes.byref(h)) == eeid.EEID_ERR_CUDA
    assert lib.eeid_server_submit(None, None, 1, 1, None, 1, None, None, 0, None) == eeid.EEID_ERR_INVALID
