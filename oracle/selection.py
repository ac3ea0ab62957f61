"""Selection quality of sample pivoting (the post-hoc selection bias of
Sec. 3.2 and its Fig. selectExpect).

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
from scipy import integrate, special, stats

# (The norm-truncation section at the end covers the second form of sample
# bias in Sec. 3.3: after pivoting, the trailing sample norms are truncated
# chi-squared variables.)


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


# -------------------------------------------------------------- Sec. 3.3, norm truncation
def truncated_chi2_pdf(x, dof, tau):
    """Density of the squared trailing sample norm ratio x after pivoting
    (Sec. 3.3 theorem): the chi-squared density with `dof` degrees of freedom
    restricted to [0, tau] and renormalised."""
    x = np.asarray(x, dtype=np.float64)
    s = 0.5 * dof
    norm = special.gammainc(s, 0.5 * tau) * special.gamma(s) * 2.0 ** s
    with np.errstate(divide="ignore", invalid="ignore"):
        body = x ** (s - 1.0) * np.exp(-0.5 * x) / norm
    return np.where((x >= 0) & (x <= tau), body, 0.0)


def truncated_chi2_expectation(dof, tau):
    """E(x) of that law, in the closed form the paper gives:
    dof (1 - exp(-tau/2) / f(dof/2, tau/2)), f(s, z) = s gamma(s, z) / z^s
    with gamma the lower incomplete gamma function (f -> 1 as z -> 0)."""
    s, z = 0.5 * dof, 0.5 * tau
    if z == 0.0:
        return 0.0
    # exp(-z) / f(s, z) in logarithms: log f = log s + log gamma(s, z) - s log z
    log_f = np.log(s) + np.log(special.gammainc(s, z)) + special.gammaln(s) - s * np.log(z)
    return float(dof * (1.0 - np.exp(-z - log_f)))


def truncation_bounds(S, j):
    """For a sample after j pivots of partial QRCP (S = Q_b^T B P, upper
    triangular in its first j columns; Alg. 1), the bound each remaining
    column's squared trailing norm must respect: min over i < j of
    s_ii^2 - sum_{k=i}^{j-1} s_{k,c}^2 (Sec. 3.3: the i-th pivot was the largest
    trailing norm at step i).  Returns (bounds, trailing norms squared) for
    the columns c >= j."""
    S = np.asarray(S, dtype=np.float64)
    tail2 = np.sum(S[j:, j:] ** 2, axis=0)
    bounds = np.full(S.shape[1] - j, np.inf)
    for i in range(j):
        partial = np.sum(S[i:j, j:] ** 2, axis=0)
        bounds = np.minimum(bounds, S[i, i] ** 2 - partial)
    return bounds, tail2

