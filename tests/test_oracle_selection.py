"""Pins of the selection-quality statistic (Sec. 3.2, post-hoc selection bias,
Fig. selectExpect): closed forms, limits, a Monte Carlo draw of the chi
variables it integrates over, and the paper's stated worst case."""
import numpy as np
import pytest

from oracle import selection


@pytest.mark.parametrize("phi,ell,n", [(0.8, 8, 16), (0.95, 4, 12), (0.3, 2, 10)])
def test_probabilities_sum_to_one(phi, ell, n):
    p = selection.select_probabilities(phi, ell, n)
    assert np.all(p >= 0.0)
    assert abs(p.sum() - 1.0) <= 1e-9


@pytest.mark.parametrize("phi", [0.3, 0.7, 0.95])
def test_two_columns_rayleigh_closed_form(phi):
    """n = 2, l = 2: ||b_j||^2 / phi^(2j) are independent exponentials, so
    P(column 1 wins) = 1 / (1 + phi^2) and E = (1 + phi^3) / (1 + phi^2)."""
    e = selection.select_expectation(phi, 2, 2)
    assert abs(e - (1 + phi ** 3) / (1 + phi ** 2)) <= 1e-10


def test_limits():
    assert selection.select_expectation(0.0, 8, 10) == 1.0
    assert selection.select_expectation(1.0, 8, 10) == 1.0


def test_monte_carlo_agrees():
    """Direct simulation: b_j = phi^j g_j with g_j ~ N(0, I_l)."""
    phi, ell, n, trials = 0.9, 8, 16, 200000
    rng = np.random.default_rng(11)
    g = rng.standard_normal((trials, n, ell))
    norms = np.linalg.norm(g, axis=2) * phi ** np.arange(n)
    pick = phi ** np.argmax(norms, axis=1)
    se = pick.std() / np.sqrt(trials)
    assert abs(pick.mean() - selection.select_expectation(phi, ell, n)) <= 5 * se


def test_more_sample_rows_select_better():
    e = [selection.select_expectation(0.9, ell, 16) for ell in (4, 8, 16)]
    assert e[0] < e[1] < e[2]


def test_worst_case_above_ninety_percent():
    """Fig. selectExpect: with a sample of 8 or more rows the expected norm of
    the selected column stays above 90 % of the optimum over phi."""
    for ell in (8, 16):
        worst = min(selection.select_expectation(phi, ell, 32) for phi in (0.8, 0.9, 0.95, 0.98))
        assert worst > 0.9, (ell, worst)


def test_golden_file_matches_oracle():
    """The stored expectations read by the benchmark are the oracle's."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "select_expectation.json")
    cases = json.load(open(path))["cases"]
    for c in cases[::7]:
        assert abs(selection.select_expectation(c["phi"], c["ell"], c["n"]) - c["exact"]) <= 1e-12


# -------------------------------------------------------------- Sec. 3.3, norm truncation
@pytest.mark.parametrize("dof,tau", [(8, 3.0), (8, 20.0), (3, 0.5), (40, 30.0), (144, 60.0)])
def test_truncated_chi2_expectation_is_the_integral(dof, tau):
    """The paper's closed form for E(x) equals the mean of the truncated
    density, integrated directly; the density has unit mass."""
    from scipy import integrate
    pdf = lambda x: selection.truncated_chi2_pdf(x, dof, tau)  # noqa: E731
    mass = integrate.quad(pdf, 0.0, tau, limit=200)[0]
    mean = integrate.quad(lambda x: x * pdf(x), 0.0, tau, limit=200)[0]
    assert abs(mass - 1.0) <= 1e-9
    assert abs(selection.truncated_chi2_expectation(dof, tau) - mean) <= 1e-8 * max(1.0, mean)


def test_truncated_chi2_expectation_limits_and_monotone():
    """Zero at tau = 0, increasing in tau, the untruncated mean (dof) for a
    large cutoff (Sec. 3.3)."""
    taus = np.linspace(0.01, 200.0, 60)
    e = [selection.truncated_chi2_expectation(16, t) for t in taus]
    assert selection.truncated_chi2_expectation(16, 0.0) == 0.0
    # strictly increasing until it meets dof in floating point
    assert all(b > a or b == 16.0 for a, b in zip(e, e[1:]))
    # small cutoff: x is nearly uniform-weighted by x^(s-1) on [0, tau]:
    # E -> dof tau / (dof + 2)
    assert abs(selection.truncated_chi2_expectation(16, 1e-4) - 16e-4 / 18) <= 1e-8
    assert abs(selection.truncated_chi2_expectation(16, 1e4) - 16.0) <= 1e-9
    assert selection.truncated_chi2_expectation(16, 1e-4) <= 1e-4


@pytest.mark.parametrize("seed", range(6))
def test_trailing_sample_norms_respect_the_truncation_bound(seed):
    """The premise of the Sec. 3.3 theorem: after j pivots of the sample QRCP,
    every remaining column's squared trailing norm stays below
    min_i (s_ii^2 - sum_{k=i}^{j-1} s_kc^2), because the i-th pivot was the
    largest trailing norm at step i.  Checked on the oracle's sample QRCP."""
    from oracle.rqrcp import sample_qrcp
    rng = np.random.default_rng(seed)
    ell, n, j = 24, 90, 12
    B = rng.standard_normal((ell, n)) * rng.uniform(0.5, 2.0, n)[None, :]
    S = B.copy()
    sample_qrcp(S, j)
    bounds, tail2 = selection.truncation_bounds(S, j)
    scale = np.max(np.abs(np.diag(S[:j, :j]))) ** 2
    assert np.all(tail2 <= bounds + 1e-12 * scale)
    # the bound is a real cut: the slack of the column closest to it is small
    assert np.min(bounds - tail2) <= 0.5 * scale
