"""Pins of the selection-quality statistic (Sec. 4, post-hoc selection bias,
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
