"""Householder reflectors, unblocked panel QR and the compact-WY form.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages restated here:

* Sec. 2.1 / Alg. 1: a reflection H_j = I - y_j tau_j y_j^T is formed from
  the current column and applied to the trailing columns.
* Sec. 2.2: a block of reflectors is held as Q_j = I - Y_j T_j Y_j^T with T_j
  upper triangular and recoverable from Y and the tau's; the inner products
  W^T = T^T Y^T A give the effect of Q^T on A.
* Sec. 5.1: block reflector composition,
  (I - Y1 T1 Y1^T)(I - Y2 T2 Y2^T) = I - Y T Y^T with
  T = [[T1, -T1 Y1^T Y2 T2], [0, T2]].

Sign / normalisation reading (the paper writes tau = 2 / y^T y with y
unnormalised): the reflector is stored with a unit leading entry, v_0 = 1,
tau = (beta - alpha) / beta, beta = -sign(alpha) * ||x||, sign(0) = +1, so
that H x = beta e_1.  If the part of x below its first entry is exactly zero
the reflector is the identity (tau = 0, beta = alpha).  This is the
convention of LAPACK's dgeqrf / dgeqp3, so R may have negative diagonal
entries.  No scaling against underflow is done.
"""

import numpy as np


def house(x):
    """Reflector for column x: returns (v, tau, beta) with v[0] = 1 and
    (I - tau v v^T) x = beta e_1."""
    x = np.asarray(x, dtype=np.float64)
    alpha = x[0]
    tail = x[1:]
    xnorm = np.sqrt(np.dot(tail, tail)) if tail.size else 0.0
    v = np.zeros_like(x)
    v[0] = 1.0
    if xnorm == 0.0:
        return v, 0.0, alpha
    beta = -np.copysign(np.hypot(alpha, xnorm), alpha if alpha != 0.0 else 1.0)
    tau = (beta - alpha) / beta
    v[1:] = tail / (alpha - beta)
    return v, tau, beta


def apply_reflector_left(v, tau, C):
    """C <- (I - tau v v^T) C, in place (Alg. 1, 'apply reflection')."""
    if tau == 0.0 or C.shape[1] == 0:
        return C
    w = v @ C
    C -= tau * np.outer(v, w)
    return C


def panel_qr(P):
    """Unblocked Householder QR of the panel P (rows x cols), in place.

    On return the upper triangle of P holds R, the strict lower triangle
    holds the reflectors below their unit leading entries, and the returned
    array holds tau.  Column j is reduced, then its reflector is applied to
    columns j+1.. of the panel (Alg. 1 without pivoting).
    """
    rows, cols = P.shape
    kk = min(rows, cols)
    tau = np.zeros(kk)
    for j in range(kk):
        v, t, beta = house(P[j:, j])
        tau[j] = t
        apply_reflector_left(v, t, P[j:, j + 1:])
        P[j, j] = beta
        P[j + 1:, j] = v[1:]
    return tau


def unit_lower(P, cols=None):
    """Explicit reflector block Y from in-place storage: unit diagonal,
    strict lower part of P, zeros above the diagonal."""
    rows = P.shape[0]
    cols = P.shape[1] if cols is None else cols
    Y = np.tril(P[:, :cols], -1)
    Y[np.arange(min(rows, cols)), np.arange(min(rows, cols))] = 1.0
    return Y


def t_factor(Y, tau):
    """Upper-triangular T with H_0 H_1 ... H_{b-1} = I - Y T Y^T (Sec. 2.2).

    Forward, column by column: T[i,i] = tau_i and
    T[:i, i] = -tau_i * T[:i,:i] @ (Y[:, :i]^T y_i).
    """
    b = len(tau)
    T = np.zeros((b, b))
    for i in range(b):
        T[i, i] = tau[i]
        if i > 0:
            T[:i, i] = -tau[i] * (T[:i, :i] @ (Y[:, :i].T @ Y[:, i]))
    return T


def compose_t(T1, Y1, T2, Y2):
    """Block reflector composition of Sec. 5.1:
    T = [[T1, -T1 Y1^T Y2 T2], [0, T2]]."""
    b1, b2 = T1.shape[0], T2.shape[0]
    T = np.zeros((b1 + b2, b1 + b2))
    T[:b1, :b1] = T1
    T[b1:, b1:] = T2
    T[:b1, b1:] = -T1 @ (Y1.T @ Y2) @ T2
    return T


def apply_block_transpose(Y, T, C):
    """C <- Q^T C with Q = I - Y T Y^T, i.e. C - Y (T^T (Y^T C)), in place."""
    if C.shape[1] == 0:
        return C
    W = T.T @ (Y.T @ C)
    C -= Y @ W
    return C


def form_q(P, tau, ncols):
    """Explicit first ``ncols`` columns of Q = H_0 H_1 ... H_{k-1} from
    in-place reflectors (applied to the identity from the last to the first)."""
    rows = P.shape[0]
    k = len(tau)
    Q = np.zeros((rows, ncols))
    Q[np.arange(min(rows, ncols)), np.arange(min(rows, ncols))] = 1.0
    for j in range(k - 1, -1, -1):
        v = np.zeros(rows - j)
        v[0] = 1.0
        v[1:] = P[j + 1:, j]
        apply_reflector_left(v, tau[j], Q[j:, :])
    return Q
