"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/*.h.  No device calls."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gw_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2104_09857_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    declared = _declared()
    assert {"gw_create", "gw_chi_tau", "gw_set_3c_tensor", "gw_set_greens"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_declared_symbols(built):
    from paper_2104_09857_gb300 import _lib

    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert _declared() <= bound | {"gw_last_error"}
    _lib.load(built)


def test_create_without_device_fails_cleanly(built):
    """On a machine without a GPU, gw_create returns an error code."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2104_09857_gb300 import _lib

    with pytest.raises(_lib.GwError):
        _lib.gw_create(0, None)
