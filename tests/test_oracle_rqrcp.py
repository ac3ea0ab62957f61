"""Pins for the oracle's RQRCP, unpivoted QR, TRQRCP and TUXV.

What pins what:
* unpivoted blocked QR  -- LAPACK dgeqrf via numpy's raw QR (same reflector
  convention, so F and tau agree entrywise).
* RQRCP                 -- A P = Q R, Q^T Q = I, R upper triangular; with an
  orthogonal Omega of full rank (l = m) the sample norms are the true trailing
  norms, so the pivots and R equal LAPACK dgeqp3's (scipy's pivoted QR);
  orthogonal columns with well separated norms come out sorted by norm;
  8x6 brute force over all column subsets.
* sample update         -- Eq. (1)-(3): with Q_b and Q formed explicitly,
  W = Q_b^T Omega Q has W21 = 0 and the updated sample equals the explicit
  re-sample [W12; W22] A^[J] of the trailing matrix, block after block.
* RSRQRCP (Alg. 5)      -- A P = Q R; with every sample drawn through
  orthonormal columns the pivots and R are dgeqp3's; its first block is
  Alg. 4's.
* TRQRCP                -- equals RQRCP truncated to the same rank (Sec. 6:
  same pivots, reflectors and rows of R).
* TUXV                  -- U, V orthonormal, X upper triangular, U X = A V and
  U X V^T = A V V^T; its error lies between the SVD tail (Eckart-Young) and
  the TRQRCP error.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import householder as hh
from oracle.rqrcp import sample_qrcp
import synth


@pytest.mark.parametrize("m,n,b", [(300, 200, 32), (200, 300, 32), (129, 129, 16),
                                   (64, 64, 64), (70, 10, 4), (10, 70, 8)])
def test_qr_blocked_matches_lapack(m, n, b):
    A = synth.gaussian(m, n, seed=m + n)
    F, tau = oracle.qr_blocked(A, b)
    h, t = np.linalg.qr(A, mode="raw")
    np.testing.assert_allclose(F, h.T, atol=2e-13)
    np.testing.assert_allclose(tau, t, atol=1e-14)


@pytest.mark.parametrize("m,n,b,p", [(120, 100, 16, 8), (100, 120, 16, 8), (97, 97, 32, 8),
                                     (50, 50, 7, 3), (40, 200, 8, 0), (200, 30, 64, 8)])
def test_rqrcp_factorization(m, n, b, p):
    A = synth.gaussian(m, n, seed=7)
    F, jpvt, tau, info = oracle.rqrcp(A, b, p, seed=1)
    assert info == 0
    assert sorted(jpvt) == list(range(n))
    k = min(m, n)
    Q = hh.form_q(F, tau, m)
    R = np.triu(F)
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    err = np.linalg.norm(A[:, jpvt] - Q @ R) / np.linalg.norm(A)
    assert err < 1e-14
    assert np.allclose(np.tril(R[:k, :k], -1), 0.0)


@pytest.mark.parametrize("m,n,b", [(30, 24, 4), (40, 40, 8), (25, 60, 5), (60, 20, 7)])
def test_exact_sample_reproduces_qrcp(m, n, b):
    """Omega orthogonal with l = m: sample norms = true trailing norms at every
    block (the updated compression stays orthonormal), so RQRCP's pivots and
    R are those of deterministic QRCP (LAPACK dgeqp3 via scipy)."""
    r = np.random.default_rng(m * n)
    # columns with well separated norms so that no near-tie decides a pivot
    A = r.standard_normal((m, n)) * (0.7 ** np.arange(n))[None, :]
    A = A[:, r.permutation(n)]
    Om, _ = np.linalg.qr(r.standard_normal((m, m)))
    F, jpvt, tau, info = oracle.rqrcp(A, b, 0, omega=Om)
    Rs, piv = sla.qr(A, pivoting=True, mode="r")
    k = min(m, n)
    np.testing.assert_array_equal(jpvt[:k], piv[:k])
    np.testing.assert_allclose(np.triu(F)[:k], Rs[:k], atol=1e-12 * np.abs(Rs).max())


@pytest.mark.parametrize("m,n,graded", [(50, 40, False), (40, 70, False), (90, 30, False),
                                         (120, 120, True), (80, 150, True)])
def test_qrcp_equals_dgeqp3(m, n, graded):
    """The deterministic QRCP oracle against LAPACK dgeqp3 (scipy): same pivots,
    same R entry by entry (same reflector sign convention), A P = Q R.  The
    graded cases (singular values 1 .. 1e-12) exercise the exact norm
    recomputation after cancellation."""
    r = np.random.default_rng(m + 3 * n)
    if graded:
        kk = min(m, n)
        U = np.linalg.qr(r.standard_normal((m, kk)))[0]
        V = np.linalg.qr(r.standard_normal((n, kk)))[0]
        A = (U * np.logspace(0, -12, kk)) @ V.T
    else:
        A = r.standard_normal((m, n)) * (0.8 ** np.arange(n))[None, :]
        A = A[:, r.permutation(n)]
    F, jpvt, tau = oracle.qrcp(A)
    Rs, piv = sla.qr(A, pivoting=True, mode="r")
    k = min(m, n)
    np.testing.assert_array_equal(jpvt[:k], piv[:k])
    R = np.triu(F)[:k]
    np.testing.assert_allclose(R, Rs[:k], atol=1e-12 * np.abs(Rs).max())
    Q = hh.form_q(F, tau, m)
    assert np.linalg.norm(A[:, jpvt] - Q[:, :k] @ R) <= 1e-14 * np.linalg.norm(A)
    d = np.abs(np.diag(R))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))


def test_sample_qrcp_partial_equals_qrcp_on_sample():
    r = np.random.default_rng(9)
    B = r.standard_normal((12, 40)) * (0.8 ** np.arange(40))[None, :]
    B = B[:, r.permutation(40)]
    S = B.copy()
    swaps, Vb, taub = sample_qrcp(S, 8)
    perm = np.arange(40)
    for i, c in enumerate(swaps):
        perm[[i, c]] = perm[[c, i]]
    Rs, piv = sla.qr(B, pivoting=True, mode="r")
    np.testing.assert_array_equal(perm[:8], piv[:8])
    np.testing.assert_allclose(np.abs(np.diag(S[:8, :8])), np.abs(np.diag(Rs[:8, :8])), rtol=1e-12)
    # Q_b^T B P = S on the processed rows: reflectors reproduce S from B P
    BP = B[:, perm].copy()
    for i in range(8):
        hh.apply_reflector_left(Vb[i:, i], taub[i], BP[i:, :])
    np.testing.assert_allclose(BP, S, atol=1e-13)


@pytest.mark.parametrize("ell", [4, 8, 16])
def test_separated_columns_sorted(ell):
    """Fig. selectExpect setup with phi = 1e-2: a flip would need a chi^2
    ratio of 1e4, so the sample pivots recover the true norm order."""
    A, order = synth.separated_columns(60, 24, phi=1e-2, seed=ell)
    b = ell // 2
    F, jpvt, tau, info = oracle.rqrcp(A, b, ell - b, seed=3)
    np.testing.assert_array_equal(jpvt, order)


def _subset_residual(A, cols):
    Q, _ = np.linalg.qr(A[:, list(cols)])
    return np.linalg.norm(A - Q @ (Q.T @ A))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_brute_force_8x6(k):
    """Greedy pivoting maximises |det R11| step by step (Sec. 2.1); on columns
    that are nearly orthogonal with separated norms the k chosen columns are
    the best k-subset of all C(6,k) (smallest projection residual)."""
    r = np.random.default_rng(42 + k)
    Q, _ = np.linalg.qr(r.standard_normal((8, 6)))
    A = Q * (0.05 ** np.arange(6))[None, :] + 1e-6 * r.standard_normal((8, 6))
    A = A[:, r.permutation(6)]
    F, jpvt, tau, info = oracle.rqrcp(A, k, 3, seed=11, k=k)
    res = {c: _subset_residual(A, c) for c in itertools.combinations(range(6), k)}
    best = min(res, key=res.get)
    assert set(jpvt[:k]) == set(best)


def test_brute_force_8x6_general_ratio():
    """On general Gaussian 8x6 input report how far the k-subset chosen from
    the sample is from the best one; it is never better than the best."""
    for s in range(20):
        A = synth.gaussian(8, 6, seed=100 + s)
        F, jpvt, tau, info = oracle.rqrcp(A, 2, 4, seed=s, k=2)
        res = {c: _subset_residual(A, c) for c in itertools.combinations(range(6), 2)}
        best = min(res.values())
        mine = _subset_residual(A, jpvt[:2])
        assert mine >= best * (1 - 1e-12)
        assert mine <= 3.0 * best


def _explicit_q(Y, T):
    return np.eye(Y.shape[0]) - Y @ T @ Y.T


def _explicit_qb(Vb, taub):
    ell = Vb.shape[0]
    Q = np.eye(ell)
    for i in range(len(taub)):
        Q = Q @ (np.eye(ell) - taub[i] * np.outer(Vb[:, i], Vb[:, i]))
    return Q


@pytest.mark.parametrize("m,n,b,p", [(60, 50, 8, 4), (45, 70, 6, 6), (80, 40, 10, 2)])
def test_sample_update_equals_explicit_resample(m, n, b, p):
    """Eq. (1)-(3): W = Q_b^T Omega^[J-1] Q^[J] has W21 = 0, and
    B^[J] = [S12 - S11 R11^-1 R12; S22] equals [W12; W22] A^[J]."""
    A = synth.gaussian(m, n, seed=21)
    trace = []
    ell = b + p
    Om = oracle.gaussian_omega(5, ell, m)
    F, jpvt, tau, info = oracle.rqrcp(A, b, p, seed=5, trace=trace)
    # replay the trailing matrices: A^[J] after block J
    G = A.copy()
    om = Om
    for blk in trace[:-1]:
        j0, bJ = blk["j0"], blk["bJ"]
        for i, c in enumerate(blk["swaps"]):
            G[:, [j0 + i, j0 + c]] = G[:, [j0 + c, j0 + i]]
        Qj = _explicit_q(blk["Y"], blk["T"])           # (m - j0) x (m - j0)
        G[j0:, j0:] = Qj.T @ G[j0:, j0:]
        Qb = _explicit_qb(blk["Vb"], blk["taub"])
        W = Qb.T @ om @ Qj
        scale = np.abs(W).max()
        np.testing.assert_allclose(W[bJ:, :bJ], 0.0, atol=1e-12 * scale)      # W21 = 0
        np.testing.assert_allclose(np.tril(W[:bJ, :bJ], -1), 0.0, atol=1e-12 * scale)
        Atrail = G[j0 + bJ:, j0 + bJ:]
        np.testing.assert_allclose(blk["B_out"], W[:, bJ:] @ Atrail,
                                   atol=1e-11 * np.abs(blk["B_out"]).max())
        om = W[:, bJ:]


def test_sample_update_mistake_is_caught():
    """Planted mistake (CPU only): dropping the S11 R11^-1 R12 term breaks the
    explicit re-sample identity checked above."""
    A = synth.gaussian(40, 40, seed=2)
    trace = []
    oracle.rqrcp(A, 8, 4, seed=5, trace=trace)
    blk = trace[0]
    S = blk["S"]
    wrong = np.vstack([S[:8, 8:], S[8:, 8:]])
    assert np.abs(wrong - blk["B_out"]).max() > 1e-3


def test_zero_columns_resample_path():
    """Exactly dependent columns leave R11 singular; the update formula is
    then replaced by a fresh sample (info = 2) and the factorization stays valid."""
    A = synth.gaussian(40, 30, seed=4)
    A[:, 10:] = 0.0
    F, jpvt, tau, info = oracle.rqrcp(A, 8, 4, seed=2)
    assert info == 2
    Q = hh.form_q(F, tau, 40)
    assert np.linalg.norm(A[:, jpvt] - Q @ np.triu(F)) < 1e-13 * np.linalg.norm(A)
    assert set(jpvt[:10]) == set(range(10))


def test_replay_accepts_own_pivots_and_rejects_wrong():
    A = synth.gaussian(60, 60, seed=8)
    F, jpvt, tau, _ = oracle.rqrcp(A, 8, 4, seed=1)
    F2, jp2, tau2, _ = oracle.rqrcp(A, 8, 4, seed=1, replay_jpvt=jpvt)
    np.testing.assert_array_equal(jp2, jpvt)
    np.testing.assert_array_equal(F2, F)
    bad = jpvt.copy()
    bad[[0, 30]] = bad[[30, 0]]
    with pytest.raises(oracle.PivotMismatch):
        oracle.rqrcp(A, 8, 4, seed=1, replay_jpvt=bad)


@pytest.mark.parametrize("m,n,k,b,p", [(80, 60, 24, 8, 4), (60, 90, 20, 6, 6), (100, 100, 33, 16, 8)])
def test_trqrcp_equals_truncated_rqrcp(m, n, k, b, p):
    A = synth.gaussian(m, n, seed=m + k)
    F, jpvt, tau, _ = oracle.rqrcp(A, b, p, seed=9, k=k)
    jt, tt, Y, R, info = oracle.trqrcp(A, k, b, p, seed=9)
    np.testing.assert_array_equal(jt[:k], jpvt[:k])
    np.testing.assert_array_equal(np.sort(jt[k:]), np.sort(jpvt[k:]))
    np.testing.assert_allclose(tt, tau, atol=1e-13)
    np.testing.assert_allclose(np.tril(Y, -1), np.tril(F[:, :k], -1), atol=1e-12)
    # rows of R agree column by column (trailing columns identified by original index)
    Rf = np.triu(F[:k, :])
    pos_f = np.argsort(jpvt)
    pos_t = np.argsort(jt)
    np.testing.assert_allclose(R[:, pos_t], Rf[:, pos_f], atol=1e-12 * np.abs(Rf).max())
    # A P ~= Q(:, :k) R on the selected columns exactly
    Q = hh.form_q(np.hstack([Y, np.zeros((m, 0))]), tt, k)
    np.testing.assert_allclose(Q @ R[:, :k], A[:, jt[:k]], atol=1e-12 * np.abs(A).max())


def test_tuxv_properties():
    m, n, k = 120, 90, 12
    A = synth.decaying_lowrank(m, n, rank=60, noise=1e-6)
    U, X, V, jpvt, info = oracle.tuxv(A, k, 4, 4, seed=3)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-13)
    assert np.allclose(np.tril(X, -1), 0.0)
    np.testing.assert_allclose(U @ X, A @ V, atol=1e-13)
    # U X V^T is the projection of A's rows onto span(V), and span(V) = row
    # space of the first k rows of Q^T A P^T: check against a pseudo-inverse.
    jt, tt, Y, R, _ = oracle.trqrcp(A, k, 4, 4, seed=3)
    Z0 = np.zeros((k, n))
    Z0[:, jt] = R
    proj = A @ np.linalg.pinv(Z0) @ Z0
    np.testing.assert_allclose(U @ X @ V.T, proj, atol=1e-12)
    s = np.linalg.svd(A, compute_uv=False)
    e_svd = np.sqrt(np.sum(s[k:] ** 2))
    e_tuxv = np.linalg.norm(A - U @ X @ V.T)
    Qk = hh.form_q(Y, tt, k)
    e_tr = np.linalg.norm(A - Qk @ (Qk.T @ A))
    assert e_svd * (1 - 1e-10) <= e_tuxv <= e_tr * (1 + 1e-10)


@pytest.mark.parametrize("jmax", [1, 2, 3, 4])
def test_tuxv_iterations_are_subspace_iteration(jmax):
    """Alg. 7 with j_max iterations: span(V) after the i-th QR step is
    (A^T A)^(i-1) applied to the row space of R P^T, span(U) after an LQ step
    is A times the previous V.  Checked against projections built with
    numpy's QR and pseudo-inverse, not the oracle's Householder routines."""
    m, n, k = 110, 80, 10
    A = synth.decaying_lowrank(m, n, rank=50, noise=1e-7)
    U, X, V, jpvt, info = oracle.tuxv(A, k, 4, 4, seed=5, jmax=jmax)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-13)
    if jmax % 2:
        assert np.allclose(np.tril(X, -1), 0.0)
        np.testing.assert_allclose(U @ X, A @ V, atol=1e-12)
    else:
        assert np.allclose(np.triu(X, 1), 0.0)
        np.testing.assert_allclose(X @ V.T, U.T @ A, atol=1e-12)
    jt, tt, Y, R, _ = oracle.trqrcp(A, k, 4, 4, seed=5)
    Z0 = np.zeros((k, n))
    Z0[:, jt] = R
    W = np.linalg.qr(Z0.T)[0]              # row space of R P^T
    for i in range(jmax):
        if i % 2 == 0:
            W = np.linalg.qr(A @ W)[0]     # column space, after a QR step
        else:
            W = np.linalg.qr(A.T @ W)[0]   # row space, after an LQ step
    if jmax % 2:
        # the last step was a QR step: U spans W
        np.testing.assert_allclose(U @ U.T, W @ W.T, atol=1e-10)
    else:
        # the last step was an LQ step: V spans W
        np.testing.assert_allclose(V @ V.T, W @ W.T, atol=1e-10)


def test_tuxv_error_non_increasing_in_iterations():
    """Each extra iteration of Alg. 7 projects onto a subspace at least as
    good (Alg. 7's QR step gives A V V^T, its LQ step U U^T A with U spanning
    A V), so ||A - U X V^T||_F never grows with j_max and stays above the
    Eckart-Young bound; with a spectral gap it approaches that bound."""
    m, n, k = 150, 120, 8
    rng = np.random.default_rng(4)
    Qa = np.linalg.qr(rng.standard_normal((m, n)))[0]
    Qb = np.linalg.qr(rng.standard_normal((n, n)))[0]
    s = np.concatenate([np.geomspace(1.0, 0.5, k), 0.05 * np.geomspace(1.0, 0.1, n - k)])
    A = (Qa * s) @ Qb.T
    e_svd = np.sqrt(np.sum(s[k:] ** 2))
    errs = []
    for jmax in range(1, 7):
        U, X, V, _, _ = oracle.tuxv(A, k, 4, 4, seed=2, jmax=jmax)
        errs.append(np.linalg.norm(A - U @ X @ V.T))
    for a, b in zip(errs, errs[1:]):
        assert b <= a * (1 + 1e-12)
    assert errs[0] >= e_svd * (1 - 1e-12)
    assert errs[-1] <= e_svd * (1 + 1e-6)


@pytest.mark.parametrize("jmax", [1, 2, 3])
def test_tuxv_svd_properties(jmax):
    """The SVD of X leaves the approximation unchanged and its singular values
    are those of the m x n approximation itself (brute-force SVD); they
    interlace below those of A (the approximation is A projected on one side)."""
    m, n, k = 90, 70, 9
    A = synth.decaying_lowrank(m, n, rank=40, noise=1e-6)
    U, X, V, _, _ = oracle.tuxv(A, k, 4, 4, seed=6, jmax=jmax)
    Us, sig, Vs, _, _ = oracle.tuxv_svd(A, k, 4, 4, seed=6, jmax=jmax)
    approx = U @ X @ V.T
    np.testing.assert_allclose(Us @ np.diag(sig) @ Vs.T, approx, atol=1e-13)
    np.testing.assert_allclose(Us.T @ Us, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Vs.T @ Vs, np.eye(k), atol=1e-13)
    assert np.all(np.diff(sig) <= 0) and sig[-1] >= 0
    s_approx = np.linalg.svd(approx, compute_uv=False)
    np.testing.assert_allclose(sig, s_approx[:k], rtol=1e-12, atol=1e-15)
    s_A = np.linalg.svd(A, compute_uv=False)
    assert np.all(sig <= s_A[:k] * (1 + 1e-12))
    # |diag(X)| are estimates too; the SVD's are at least as large in sum
    # of squares (both give ||X||_F^2) and dominate in the leading value
    np.testing.assert_allclose(np.sum(sig ** 2), np.sum(X ** 2), rtol=1e-12)
    assert sig[0] >= np.abs(np.diag(X)).max() * (1 - 1e-12)


# ---------------------------------------------------------------- RSRQRCP (Alg. 5)
@pytest.mark.parametrize("m,n,b,p", [(120, 100, 16, 8), (100, 120, 16, 8), (97, 97, 32, 8),
                                     (200, 30, 64, 8)])
def test_rsrqrcp_factorization(m, n, b, p):
    """Alg. 5: A P = Q R with Q orthogonal and R upper triangular."""
    A = synth.gaussian(m, n, seed=7)
    F, jpvt, tau, info = oracle.rsrqrcp(A, b, p, seed=1)
    assert info == 0
    assert sorted(jpvt) == list(range(n))
    Q = hh.form_q(F, tau, m)
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-13)
    assert np.linalg.norm(A[:, jpvt] - Q @ np.triu(F)) < 1e-14 * np.linalg.norm(A)


@pytest.mark.parametrize("m,n,b,p", [(60, 50, 8, 4), (45, 70, 6, 6)])
def test_rsrqrcp_samples_are_fresh_compressions(m, n, b, p):
    """Alg. 5 by definition: after block J the next sample is Omega^[J] A^[J],
    a fresh GIID block (Philox stream 0x100 + J) times the trailing matrix
    updated by that block's reflectors, rebuilt here from explicit Q's."""
    from oracle import philox as ph
    A = synth.gaussian(m, n, seed=23)
    trace = []
    ell = b + p
    oracle.rqrcp(A, b, p, seed=7, trace=trace, resample_every_block=True)
    G = A.copy()
    for J, blk in enumerate(trace[:-1], start=1):
        j0, bJ = blk["j0"], blk["bJ"]
        for i, c in enumerate(blk["swaps"]):
            G[:, [j0 + i, j0 + c]] = G[:, [j0 + c, j0 + i]]
        G[j0:, j0:] = _explicit_q(blk["Y"], blk["T"]).T @ G[j0:, j0:]
        trailing = G[j0 + bJ:, j0 + bJ:]
        om = ph.gaussian_block(7, ell, trailing.shape[0], 0x100 + J)
        np.testing.assert_allclose(blk["B_out"], om @ trailing,
                                   atol=1e-11 * np.abs(blk["B_out"]).max())


@pytest.mark.parametrize("m,n,b", [(30, 24, 4), (40, 40, 8), (25, 60, 5), (60, 20, 7)])
def test_rsrqrcp_exact_samples_reproduce_qrcp(m, n, b):
    """With every sample drawn through orthonormal columns (l = m), each
    block's sample norms are the true trailing column norms, so Alg. 5's pivots
    and R are deterministic QRCP's (LAPACK dgeqp3 via scipy)."""
    r = np.random.default_rng(m * n + 1)
    A = r.standard_normal((m, n)) * (0.7 ** np.arange(n))[None, :]
    A = A[:, r.permutation(n)]
    Om, _ = np.linalg.qr(r.standard_normal((m, m)))

    def omega_fn(J, rows):
        Q, _ = np.linalg.qr(r.standard_normal((m, m)))
        return Q[:, :rows]
    F, jpvt, tau, info = oracle.rsrqrcp(A, b, 0, omega=Om, omega_fn=omega_fn)
    Rs, piv = sla.qr(A, pivoting=True, mode="r")
    k = min(m, n)
    np.testing.assert_array_equal(jpvt[:k], piv[:k])
    np.testing.assert_allclose(np.triu(F)[:k], Rs[:k], atol=1e-12 * np.abs(Rs).max())


def test_rsrqrcp_first_block_equals_rqrcp():
    """Alg. 4 and Alg. 5 share Omega^[0] and the first block, so the first b
    pivots, reflectors and rows of R coincide; later blocks differ only
    through the samples (both stay valid factorizations)."""
    A = synth.gaussian(80, 70, seed=3)
    F1, j1, t1, _ = oracle.rqrcp(A, 16, 8, seed=4)
    F2, j2, t2, _ = oracle.rsrqrcp(A, 16, 8, seed=4)
    np.testing.assert_array_equal(j1[:16], j2[:16])
    np.testing.assert_allclose(t1[:16], t2[:16], atol=1e-14)
    np.testing.assert_allclose(np.triu(F1)[:16, :16], np.triu(F2)[:16, :16], atol=1e-12)
