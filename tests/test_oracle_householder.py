"""Pins for the oracle's Householder, panel QR and compact-WY routines.

Each check is independent of the routine it tests: LAPACK's dgeqrf (through
numpy's raw QR) for the reflector convention and storage, explicit products
of reflector matrices for the T factor (Sec. 2.2) and for the block
composition of Sec. 5.1.
"""
import numpy as np
import pytest

from oracle import householder as hh


def _rng(s):
    return np.random.default_rng(s)


@pytest.mark.parametrize("x", [
    np.array([3.0, 4.0]), np.array([-1.0, 2.0, 2.0]), np.array([0.0, 1.0, 0.0]),
    np.array([5.0]), np.array([2.0, 0.0, 0.0]), np.array([-7.0, 0.0])])
def test_house_maps_to_axis(x):
    v, tau, beta = hh.house(x)
    H = np.eye(len(x)) - tau * np.outer(v, v)
    y = H @ x
    assert v[0] == 1.0
    np.testing.assert_allclose(y[1:], 0.0, atol=1e-15 * max(1.0, np.abs(x).max()))
    np.testing.assert_allclose(y[0], beta, rtol=1e-15)
    # H orthogonal, and beta = -sign(alpha) ||x|| unless the tail is zero
    np.testing.assert_allclose(H @ H.T, np.eye(len(x)), atol=1e-15)
    if np.any(x[1:] != 0):
        assert beta == pytest.approx(-np.copysign(np.linalg.norm(x), x[0] if x[0] != 0 else 1.0))
    else:
        assert tau == 0.0 and beta == x[0]


@pytest.mark.parametrize("m,n", [(7, 5), (40, 40), (64, 33), (5, 9), (1, 1), (130, 17)])
def test_panel_qr_matches_lapack(m, n):
    A = _rng(m * 100 + n).standard_normal((m, n))
    P = A.copy()
    tau = hh.panel_qr(P)
    h, t = np.linalg.qr(A, mode="raw")   # LAPACK dgeqrf, Fortran order -> h is A^T
    np.testing.assert_allclose(P, h.T, atol=1e-13, rtol=0)
    np.testing.assert_allclose(tau, t, atol=1e-14, rtol=0)


def _reflector_product(Y, tau):
    m = Y.shape[0]
    Q = np.eye(m)
    for j in range(len(tau)):
        Q = Q @ (np.eye(m) - tau[j] * np.outer(Y[:, j], Y[:, j]))
    return Q


@pytest.mark.parametrize("m,b", [(20, 6), (64, 32), (9, 9)])
def test_t_factor_equals_reflector_product(m, b):
    P = _rng(m + b).standard_normal((m, b))
    tau = hh.panel_qr(P)
    Y = hh.unit_lower(P)
    T = hh.t_factor(Y, tau)
    assert np.allclose(np.tril(T, -1), 0.0)
    np.testing.assert_allclose(np.eye(m) - Y @ T @ Y.T, _reflector_product(Y, tau), atol=1e-14)


def test_form_q_and_reconstruction():
    A = _rng(3).standard_normal((50, 20))
    P = A.copy()
    tau = hh.panel_qr(P)
    Q = hh.form_q(P, tau, 20)
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-14)
    np.testing.assert_allclose(Q @ np.triu(P[:20]), A, atol=1e-13)


def test_block_composition():
    """Sec. 5.1: (I - Y1 T1 Y1^T)(I - Y2 T2 Y2^T) = I - Y T Y^T and
    W^T = T^T Y^T A = [T1^T Y1^T A ; T2^T (Y2^T A - (Y2^T Y1) W1^T)]."""
    m, b1, b2 = 30, 5, 7
    r = _rng(11)
    P1 = r.standard_normal((m, b1))
    t1 = hh.panel_qr(P1)
    Y1 = hh.unit_lower(P1)
    P2 = r.standard_normal((m - b1, b2))
    t2 = hh.panel_qr(P2)
    Y2 = np.zeros((m, b2))
    Y2[b1:] = hh.unit_lower(P2)
    T1 = hh.t_factor(Y1, t1)
    T2 = hh.t_factor(Y2, t2)
    T = hh.compose_t(T1, Y1, T2, Y2)
    Y = np.hstack([Y1, Y2])
    lhs = (np.eye(m) - Y1 @ T1 @ Y1.T) @ (np.eye(m) - Y2 @ T2 @ Y2.T)
    np.testing.assert_allclose(lhs, np.eye(m) - Y @ T @ Y.T, atol=1e-14)
    np.testing.assert_allclose(lhs, _reflector_product(Y, np.concatenate([t1, t2])), atol=1e-14)
    A = r.standard_normal((m, 11))
    Wt = T.T @ Y.T @ A
    W1t = T1.T @ Y1.T @ A
    W2t = T2.T @ (Y2.T @ A - (Y2.T @ Y1) @ W1t)
    np.testing.assert_allclose(Wt, np.vstack([W1t, W2t]), atol=1e-13)


def test_apply_block_transpose_is_qt():
    m, b = 25, 6
    r = _rng(5)
    P = r.standard_normal((m, b))
    tau = hh.panel_qr(P)
    Y = hh.unit_lower(P)
    T = hh.t_factor(Y, tau)
    C = r.standard_normal((m, 4))
    Q = _reflector_product(Y, tau)
    out = hh.apply_block_transpose(Y, T, C.copy())
    np.testing.assert_allclose(out, Q.T @ C, atol=1e-14)
