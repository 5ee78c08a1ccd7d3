"""The library's minimax grids (gw_minimax_grid, host code: runs without a
GPU) against the oracle of oracle/grids.py: nodes, weights and maximum error
on the unit interval and in physical units, the equioscillation of the
library's own result, and the argument and convergence errors."""

import ctypes

import numpy as np
import pytest

from oracle import grids as og

CASES = [("T", 1, 10.0), ("T", 4, 7.66), ("T", 6, 7.66), ("T", 8, 100.0), ("T", 12, 1e3),
         ("T", 12, 1e5), ("F", 1, 10.0), ("F", 4, 7.66), ("F", 8, 100.0), ("F", 12, 1e3),
         ("F", 16, 1e4)]


@pytest.fixture(scope="module")
def lib():
    from paper_2104_09857_gb300 import _lib, build

    _lib.load(build.build())
    return _lib


def _kind(lib, k):
    return lib.GW_GRID_TIME if k == "T" else lib.GW_GRID_FREQ


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}_R{c[2]:g}")
def test_unit_grid_matches_oracle(lib, case):
    kind, n, R = case
    nodes, w, err = lib.gw_minimax_grid(_kind(lib, kind), n, 1.0, R)
    with np.errstate(all="ignore"):
        p, a, E = og.minimax_unit(kind, n, R)
    assert err == pytest.approx(E, rel=1e-8)
    np.testing.assert_allclose(nodes, p, rtol=1e-7, atol=0)
    np.testing.assert_allclose(w, a, rtol=1e-7, atol=0)


@pytest.mark.parametrize("case", [("T", 6, 7.66), ("F", 12, 1e3)], ids=["T6", "F12"])
def test_library_grid_equioscillates(lib, case):
    """Checked on the library's output alone: max |eta| equals the reported
    error and is reached at 2n + 1 points of alternating sign."""
    kind, n, R = case
    nodes, w, err = lib.gw_minimax_grid(_kind(lib, kind), n, 1.0, R)
    x = np.exp(np.linspace(0.0, np.log(R), 40001))
    if kind == "T":
        e = 1.0 / x - np.exp(-np.outer(x, nodes)) @ w
    else:
        e = 1.0 / x - (x[:, None] ** 2 / (x[:, None] ** 2 + nodes[None, :] ** 2) ** 2) @ w
    assert np.abs(e).max() == pytest.approx(err, rel=1e-6)
    s = np.sign(e[np.abs(e) >= (1 - 1e-5) * err])
    runs = [s[0]] + [v for u, v in zip(s[:-1], s[1:]) if v != u]
    assert len(runs) >= 2 * n + 1 and runs[0] > 0
    assert np.all(np.diff(nodes) > 0) and np.all(w > 0)


@pytest.mark.parametrize("kind", ["T", "F"])
def test_physical_grid_matches_oracle(lib, kind):
    """Transition energies of the synthetic molecules: [0.3, 2.3] Ha."""
    nodes, w, err = lib.gw_minimax_grid(_kind(lib, kind), 6, 0.3, 2.3)
    with np.errstate(all="ignore"):
        p, a, E = og.minimax_grid(kind, 6, 0.3, 2.3)
    np.testing.assert_allclose(nodes, p, rtol=1e-7, atol=0)
    np.testing.assert_allclose(w, a, rtol=1e-7, atol=0)
    assert err == pytest.approx(E, rel=1e-8)


def test_argument_errors(lib):
    f = lib.lib().gw_minimax_grid
    buf = np.zeros(8)
    e = ctypes.c_double()
    p = buf.ctypes.data
    assert f(2, 4, 1.0, 10.0, p, p, ctypes.byref(e)) == -1          # kind
    assert f(0, 0, 1.0, 10.0, p, p, ctypes.byref(e)) == -1          # n < 1
    assert f(0, 65, 1.0, 10.0, p, p, ctypes.byref(e)) == -1         # n > GW_GRID_MAX_N
    assert f(0, 4, 0.0, 10.0, p, p, ctypes.byref(e)) == -1          # e_min <= 0
    assert f(0, 4, 2.0, 2.0, p, p, ctypes.byref(e)) == -1           # one energy only
    assert f(0, 4, 1.0, float("nan"), p, p, ctypes.byref(e)) == -4  # non-finite
    assert f(0, 4, 1.0, 10.0, None, p, ctypes.byref(e)) == -1       # null output
    assert f(0, 4, 1.0, 10.0, p, p, None) == -1


@pytest.mark.slow
def test_below_rounding_level_reports_not_converged(lib):
    """Twelve time points for R = 7.66 would fit 1/x far below FP64 rounding:
    the exchange cannot level that and gives up within its work budget."""
    with pytest.raises(lib.GwError) as ei:
        lib.gw_minimax_grid(lib.GW_GRID_TIME, 12, 0.3, 2.3)
    assert ei.value.code == -10


@pytest.mark.parametrize("n", [6, 8])
def test_minimax_grids_fit_the_transforms_better_than_log_grids(lib, n):
    """At equal n, least-squares cosine (tau -> i omega) and sine weights on
    the library's minimax grids fit the closed-form transforms of exp(-x|tau|)
    over the synthetic spectrum [0.3, 2.3] Ha at least twice as well as on the
    log-spaced grid tau in [0.01, 50] with log-spaced omega."""
    from synth.chain_inputs import (fit_error, omega_grid, sine_fit_error, sine_weights,
                                    transform_weights)

    gap, width = 0.3, 2.3
    tl = 0.01 * 5000.0 ** (np.arange(n) / (n - 1))
    ol = omega_grid(n, gap, width)
    tm = lib.gw_minimax_grid(lib.GW_GRID_TIME, n, gap, width)[0]
    om = lib.gw_minimax_grid(lib.GW_GRID_FREQ, n, gap, width)[0]
    errs = []
    for t, o in ((tl, ol), (tm, om)):
        g, d = transform_weights(t, o, gap, width)
        eg, _ = fit_error(t, o, g, d, gap, width)
        es = sine_fit_error(t, o, sine_weights(t, o, gap, width), gap, width)
        errs.append((eg, es))
    (lg, ls), (mg, ms) = errs
    print(f"n={n}: cosine fit {lg:.2e} (log) {mg:.2e} (minimax); sine {ls:.2e} {ms:.2e}")
    assert mg < 0.5 * lg and ms < 0.5 * ls


@pytest.mark.parametrize("n", [4, 6, 8])
def test_transform_weights_match_oracle(lib, n):
    """Library weights (one-sided Jacobi SVD) against the oracle's (numpy
    lstsq) on the log grid and on minimax grids of the synthetic spectrum;
    well-conditioned sizes agree elementwise, and the fit errors agree."""
    gap, width = 0.3, 2.3
    tl = 0.01 * 5000.0 ** (np.arange(n) / (n - 1))
    ol = 0.15 * (9.2 / 0.15) ** (np.arange(n) / (n - 1))
    tm = lib.gw_minimax_grid(lib.GW_GRID_TIME, n, gap, width)[0]
    om = lib.gw_minimax_grid(lib.GW_GRID_FREQ, n, gap, width)[0]
    for tau, omega in ((tl, ol), (tm, om)):
        got = lib.gw_transform_weights(tau, omega, gap, width)
        ref = og.transform_weights(tau, omega, gap, width)
        for g, r in zip(got[:3], ref[:3]):
            assert np.abs(g - r).max() <= 1e-8 * np.abs(r).max()
        np.testing.assert_allclose(got[3], ref[3], rtol=1e-6)


def test_transform_weights_ill_conditioned_fit_as_well(lib):
    """Twenty log-spaced points for R = 7.7: the columns are dependent to
    1e-14, the truncated solutions differ, but they fit equally well."""
    n, gap, width = 20, 0.3, 2.3
    tau = 0.01 * 5000.0 ** (np.arange(n) / (n - 1))
    omega = 0.15 * (9.2 / 0.15) ** (np.arange(n) / (n - 1))
    got = lib.gw_transform_weights(tau, omega, gap, width)
    ref = og.transform_weights(tau, omega, gap, width)
    assert np.all(got[3] <= 1.05 * ref[3]) and np.all(got[3] < 1e-7)


def test_transform_weights_arguments(lib):
    f = lib.lib().gw_transform_weights
    t = np.array([0.5, 1.0])
    w = np.array([0.5, 1.0])
    out = np.zeros(4)
    p = out.ctypes.data
    assert f(None, 2, w.ctypes.data, 2, 0.3, 2.3, p, p, p, None) == -1
    assert f(t.ctypes.data, 0, w.ctypes.data, 2, 0.3, 2.3, p, p, p, None) == -1
    assert f(t.ctypes.data, 2, w.ctypes.data, 2, 2.3, 0.3, p, p, p, None) == -1
    bad = np.array([0.5, -1.0])
    assert f(bad.ctypes.data, 2, w.ctypes.data, 2, 0.3, 2.3, p, p, p, None) == -1
    nan = np.array([0.5, np.nan])
    assert f(t.ctypes.data, 2, nan.ctypes.data, 2, 0.3, 2.3, p, p, p, None) == -4
    assert f(t.ctypes.data, 2, w.ctypes.data, 2, 0.3, 2.3, None, None, None, None) == 0
