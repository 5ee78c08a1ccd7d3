"""Pins of the minimax-grid oracle (oracle/grids.py) against what fixes a best
approximation independently of how it was computed: the equioscillation
(alternation) characterisation on a fine grid, brute force for one term,
local optimality under perturbation, monotonicity in n and R, the half-line
limit, and the scaling to physical energies."""

import numpy as np
import pytest

from oracle import grids as og

CASES = [("T", 1, 10.0), ("T", 4, 7.66), ("T", 6, 7.66), ("T", 8, 100.0), ("T", 12, 1e3),
         ("F", 1, 10.0), ("F", 4, 7.66), ("F", 8, 100.0), ("F", 12, 1e3)]


@pytest.fixture(scope="module")
def solved():
    with np.errstate(all="ignore"):
        return {c: og.minimax_unit(*c) for c in CASES}


def _fine(R, m=40001):
    return np.exp(np.linspace(0.0, np.log(R), m))


def _alternations(e, level):
    """Longest run of alternating signs among the points where |e| reaches
    `level` (consecutive same-sign points count once)."""
    s = np.sign(e[np.abs(e) >= level])
    if len(s) == 0:
        return 0, 0
    runs = [s[0]]
    for v in s[1:]:
        if v != runs[-1]:
            runs.append(v)
    return len(runs), runs[0]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}_R{c[2]:g}")
def test_error_equioscillates_at_2n_plus_1_points(solved, case):
    """Chebyshev's characterisation: the best n-term approximation (2n
    parameters) has an error of constant modulus E at 2n + 1 points of
    alternating sign, positive at both ends; any other approximant with that
    property would have the same E (de la Vallee Poussin)."""
    kind, n, R = case
    p, a, E = solved[case]
    x = _fine(R)
    e = og.error(kind, x, a, p)
    assert np.abs(e).max() == pytest.approx(E, rel=1e-6)
    count, first = _alternations(e, (1.0 - 1e-5) * E)
    assert count >= 2 * n + 1
    assert first > 0
    assert np.all(a > 0) and np.all(p > 0) and np.all(np.diff(p) > 0)


def _brute_one_term(kind, R):
    """min over (a, p) of max |1/x - a b(x; p)| by a nested grid search."""
    x = _fine(R, 4001)
    lo_a, hi_a, lo_p, hi_p = 0.05, 5.0, 0.02, 5.0
    best = (np.inf, 0, 0)
    for _ in range(6):
        A = np.linspace(lo_a, hi_a, 161)
        P = np.linspace(lo_p, hi_p, 161)
        B = og.basis(kind, x, P)                                    # [x, p]
        err = np.abs(1.0 / x[:, None, None] - A[None, :, None] * B[:, None, :]).max(axis=0)
        i, j = np.unravel_index(np.argmin(err), err.shape)
        best = (err[i, j], A[i], P[j])
        da, dp = 4 * (A[1] - A[0]), 4 * (P[1] - P[0])
        lo_a, hi_a = max(1e-3, A[i] - da), A[i] + da
        lo_p, hi_p = max(1e-3, P[j] - dp), P[j] + dp
    return best


@pytest.mark.parametrize("kind", ["T", "F"])
def test_one_term_matches_brute_force(solved, kind):
    p, a, E = solved[(kind, 1, 10.0)]
    e_brute, a_b, p_b = _brute_one_term(kind, 10.0)
    # the search's best pair, measured on the same fine grid as E
    e_brute = np.abs(og.error(kind, _fine(10.0), np.array([a_b]), np.array([p_b]))).max()
    assert E <= e_brute * (1 + 1e-9)
    assert E == pytest.approx(e_brute, rel=2e-4)
    assert a[0] == pytest.approx(a_b, rel=1e-2)
    assert p[0] == pytest.approx(p_b, rel=1e-2)


@pytest.mark.parametrize("case", [("T", 6, 7.66), ("F", 8, 100.0)], ids=["T6", "F8"])
def test_no_nearby_parameters_do_better(solved, case):
    """Small random perturbations of the 2n parameters never lower the
    maximum error (local optimality in the max norm)."""
    kind, n, R = case
    p, a, E = solved[case]
    x = _fine(R, 20001)
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = 10.0 ** rng.uniform(-9, -5)
        ap = a * (1 + s * rng.standard_normal(n))
        pp = p * (1 + s * rng.standard_normal(n))
        assert np.abs(og.error(kind, x, ap, pp)).max() >= E * (1 - 1e-9)


def test_error_falls_with_n_and_grows_with_R(solved):
    with np.errstate(all="ignore"):
        for kind in ("T", "F"):
            e4 = og.minimax_unit(kind, 4, 100.0)[2]
            assert solved[(kind, 8, 100.0)][2] < e4
            e = [og.minimax_unit(kind, 4, R)[2] for R in (5.0, 20.0, 80.0)]
            assert e[0] < e[1] < e[2]


def test_half_line_limit():
    """One term: the half-line solution has its last alternation point near
    x = 12; beyond that R no longer matters."""
    with np.errstate(all="ignore"):
        r1 = og.minimax_unit("T", 1, 1e3)
        r2 = og.minimax_unit("T", 1, 1e6)
    assert r1[2] == pytest.approx(r2[2], rel=1e-9)
    assert r1[0][0] == pytest.approx(r2[0][0], rel=1e-6)


@pytest.mark.parametrize("kind", ["T", "F"])
def test_physical_grid_bounds_the_energy_denominator(kind):
    """The physical grid approximates 1/E for every E in [e_min, e_max]
    within the returned error, which is attained."""
    e_min, e_max = 0.3, 2.3
    with np.errstate(all="ignore"):
        nodes, w, err = og.minimax_grid(kind, 5, e_min, e_max)
    E = np.linspace(e_min, e_max, 20001)
    if kind == "T":
        approx = np.exp(-np.outer(E, nodes)) @ w
    else:
        approx = (E[:, None] ** 2 / (E[:, None] ** 2 + nodes[None, :] ** 2) ** 2) @ w
    dev = np.abs(1.0 / E - approx)
    assert dev.max() <= err * (1 + 1e-6)
    assert dev.max() >= err * (1 - 1e-4)


def test_transform_weights_solve_the_normal_equations():
    """Well-conditioned case (4 points): the weights equal the solution of the
    normal equations A^T A w = A^T f, a second route, and the residual is
    orthogonal to every column."""
    tau = np.array([0.2, 0.9, 3.0, 9.0])
    omega = np.array([0.2, 0.7, 2.0, 5.0])
    gamma, delta, sw, err = og.transform_weights(tau, omega, 0.3, 2.3)
    x = 0.3 * (2.3 / 0.3) ** (np.arange(400) / 399)
    e = np.exp(-np.outer(x, tau))
    c = 2.0 * x[:, None] / (x[:, None] ** 2 + omega ** 2)
    s = omega / (x[:, None] ** 2 + omega ** 2)
    for a, f, w in ((e, c, gamma), (c, e, delta), (e, s, sw)):
        ref = np.linalg.solve(a.T @ a, a.T @ f).T
        np.testing.assert_allclose(w, ref, rtol=1e-6, atol=1e-9 * np.abs(ref).max())
        r = a @ w.T - f
        assert np.abs(a.T @ r).max() <= 1e-9 * np.abs(a).max() * np.abs(f).max() * len(x)
    assert np.all(err > 0) and np.all(err < 0.1)


def test_transform_weights_reproduce_the_closed_form_transform():
    """chi(tau) = exp(-x|tau|) for an energy x inside the range: the cosine
    weights give its full-line transform 2x/(x^2 + omega^2), the sine weights
    omega/(x^2 + omega^2), within the reported fit errors; errors fall as
    points are added."""
    errs = []
    for n in (6, 8, 10):
        tau = 0.01 * 5000.0 ** (np.arange(n) / (n - 1))
        omega = 0.15 * (9.2 / 0.15) ** (np.arange(n) / (n - 1))
        gamma, _, sw, err = og.transform_weights(tau, omega, 0.3, 2.3)
        xs = 0.3 * (2.3 / 0.3) ** (np.arange(997) / 996)
        top_c = np.max(2 * xs[:, None] / (xs[:, None] ** 2 + omega ** 2))
        top_s = np.max(omega / (xs[:, None] ** 2 + omega ** 2))
        for x in (0.31, 0.77, 2.29):
            cos_ft = 2 * x / (x * x + omega ** 2)
            sin_ft = omega / (x * x + omega ** 2)
            assert np.abs(gamma @ np.exp(-x * tau) - cos_ft).max() <= 1.01 * err[0] * top_c
            assert np.abs(sw @ np.exp(-x * tau) - sin_ft).max() <= 1.01 * err[2] * top_s
        errs.append(err)
    assert errs[0][0] > errs[1][0] > errs[2][0]


def test_minimax_grids_transform_chi_of_benzene_more_accurately():
    """chi(i tau) of benzene on 8 log-spaced tau points (0.01-50) and on the 8
    minimax points of its spectrum [0.3, 2.28] Ha, cosine-transformed with
    least-squares weights, against the closed-form chi(i omega) of the MO
    route.  The error, relative to the largest |chi(i omega)|, is lower on
    the minimax grids (the relative error at the largest omega is not: there
    chi is small)."""
    from dataclasses import replace

    from oracle import chain as och
    from oracle import chi as oc
    from synth import make_case

    case = make_case("benzene", n_tau=4)
    s = case.system
    t = oc.dense_three_center(s.n_ao, s.n_ri, case.t3c.blocks, case.t3c.offsets, case.t3c.data, 0.0)
    gap = case.eps[case.n_occ] - case.eps[case.n_occ - 1]
    width = case.eps.max() - case.eps.min()
    n = 8
    log_t = 0.01 * 5000.0 ** (np.arange(n) / (n - 1))
    log_w = 0.5 * gap * (4.0 * width / gap) ** (np.arange(n) / (n - 1))
    with np.errstate(all="ignore"):
        mm_t = og.minimax_grid("T", n, gap, width)[0]
        mm_w = og.minimax_grid("F", n, gap, width)[0]
    errs = []
    for tau, omega in ((log_t, log_w), (mm_t, mm_w)):
        gamma = og.transform_weights(tau, omega, gap, width)[0]
        chi_w = och.chi_to_omega(oc.chi_dense(replace(case, tau=tau)), gamma)
        exact = [och.chi_omega_closed_form(t, case.C, case.eps, case.n_occ, w) for w in omega]
        errs.append(max(np.linalg.norm(chi_w[k] - exact[k]) for k in range(n))
                    / max(np.linalg.norm(x) for x in exact))
    print(f"chi(i omega) error / max |chi|: log {errs[0]:.2e}, minimax {errs[1]:.2e}")
    assert errs[1] < 0.5 * errs[0]
