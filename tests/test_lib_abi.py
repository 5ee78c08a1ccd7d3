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


C_PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "gwchi.h"

int main(void) {
  double tau[6], a[6], omega[6], b[6], err_t, err_w, gamma[36], delta[36], s[36], fit[3];
  if (gw_minimax_grid(GW_GRID_TIME, 6, 0.3, 2.3, tau, a, &err_t) != GW_OK) return 1;
  if (gw_minimax_grid(GW_GRID_FREQ, 6, 0.3, 2.3, omega, b, &err_w) != GW_OK) return 2;
  if (gw_transform_weights(tau, 6, omega, 6, 0.3, 2.3, gamma, delta, s, fit) != GW_OK) return 3;
  if (gw_minimax_grid(GW_GRID_TIME, 0, 0.3, 2.3, tau, a, &err_t) != GW_ERR_INVALID_ARG) return 4;
  /* 1/E from the time grid at E = 1 */
  double sum = 0.0;
  for (int j = 0; j < 6; ++j) sum += a[j] * exp(-tau[j]);
  printf("%.17g %.17g %.17g %.17g\n", err_t, err_w, fit[0], fabs(sum - 1.0));
  return fabs(sum - 1.0) <= err_t * 1.000001 ? 0 : 5;
}
"""


def test_header_compiles_as_c_and_host_calls_link(built):
    """A C99 program includes gwchi.h, links libgwchi and calls the host-code
    entry points (grids and transform weights) without a GPU."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    work = os.path.join(ROOT, "paper_2104_09857_gb300", "_build")
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "abi_check.c")
    exe = os.path.join(work, "abi_check")
    with open(src, "w") as f:
        f.write(C_PROGRAM)
    libdir = os.path.dirname(built)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        src, "-o", exe, "-L", libdir, "-lgwchi", "-lm", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    err_t, err_w, fit0, dev = (float(v) for v in r.stdout.split())
    assert 0 < err_t < 1e-5 and 0 < err_w < 1e-5 and 0 < fit0 < 1e-2 and dev <= err_t * 1.000001
