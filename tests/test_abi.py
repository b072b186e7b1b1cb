"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports every symbol
declared in include/gsolve.h (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gsolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gs_create", "gs_set_layers", "gs_set_inclusions", "gs_set_incidence", "gs_factor",
                 "gs_translate", "gs_apply", "gs_solve", "gs_bragg", "gs_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1412_7466_gb300 import build, exported_symbols, load_library
    build.build()
    lib = load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(exported_symbols()) <= set(_declared())


def test_errors_without_device_are_reported():
    """Without a GPU the library still loads; gs_create reports a CUDA error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1412_7466_gb300 import GS_ERR_CUDA, load_library
    lib = load_library()
    h = ctypes.c_void_p()
    assert lib.gs_create(ctypes.byref(h), 0, None) == GS_ERR_CUDA
    assert lib.gs_strerror(GS_ERR_CUDA).decode() == "CUDA error"


def test_status_strings_cover_every_code():
    """Every status the C-ABI returns, the bounded-wait timeout included, has its own message (host
    function, no device needed)."""
    from paper_1412_7466_gb300 import load_library
    import paper_1412_7466_gb300 as P
    lib = load_library()
    codes = {name: getattr(P, name) for name in dir(P) if name.startswith("GS_ERR_") or name == "GS_OK"}
    assert "GS_ERR_TIMEOUT" in codes
    msgs = {name: lib.gs_strerror(v).decode() for name, v in codes.items()}
    assert msgs["GS_ERR_TIMEOUT"] == "device wait timed out"
    assert len(set(msgs.values())) == len(msgs), msgs            # distinct messages
    assert "unknown status" not in msgs.values()
    assert lib.gs_strerror(12345).decode() == "unknown status"
