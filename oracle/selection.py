"""Selection quality of sample pivoting (the post-hoc selection bias of
Sec. 4 and its Fig. selectExpect).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Setting: A has orthogonal columns with ||a_j|| = phi^(j-1), j = 1..n.  The
sample column b_j = Omega a_j (Omega l x m GIID) has ||b_j|| = phi^(j-1) X_j
with X_1..X_n independent chi-distributed with l degrees of freedom (Omega's
rotational invariance maps the orthogonal columns onto independent Gaussian
vectors).  The sample pivot is j_max = argmax_j ||b_j||; the statistic is
E(||a_{j_max}||), which deterministic QRCP makes exactly 1.

P(j_max = j) = integral over x of f(x) prod_{i != j} F(x phi^(j-i)), with f
and F the chi density and distribution function: X_j = x wins when every
other phi^(i-1) X_i stays below phi^(j-1) x.
"""
import numpy as np
from scipy import integrate, stats


def select_probabilities(phi, ell, n):
    """P(j_max = j) for j = 0..n-1 (0-based: ||a_j|| = phi^j)."""
    if not 0.0 <= phi <= 1.0:
        raise ValueError("phi must lie in [0, 1]")
    if phi == 0.0:
        p = np.zeros(n)
        p[0] = 1.0
        return p
    if phi == 1.0:
        return np.full(n, 1.0 / n)
    chi = stats.chi(ell)
    lphi = np.log(phi)
    idx = np.arange(n)
    p = np.zeros(n)
    for j in range(n):
        others = idx[idx != j]
        with np.errstate(over="ignore"):
            factors = np.exp((j - others) * lphi)  # phi^(j - i); inf for far-later columns

        def integrand(x):
            return chi.pdf(x) * np.prod(chi.cdf(x * factors))

        hi = chi.ppf(1.0 - 1e-16)
        p[j] = integrate.quad(integrand, 0.0, hi, limit=400, epsabs=1e-14, epsrel=1e-11)[0]
    return p


def select_expectation(phi, ell, n):
    """E(||a_{j_max}||) for the sample pivot (Fig. selectExpect)."""
    p = select_probabilities(phi, ell, n)
    return float(np.sum(p * phi ** np.arange(n)))
