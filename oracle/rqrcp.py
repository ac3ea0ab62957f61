"""RQRCP, TRQRCP, TUXV and unpivoted blocked QR, step by step in float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows, in the paper's order and notation:

* Alg. 1 (QRCP, level-2) halted after b steps, run on the l x n_J sample
  matrix B ("qrcp(B, b)" in Alg. 4 / Alg. 6; Sec. 5 says only a partial
  factorization of the sample is needed).
* Alg. 4 (RQRCP): sketch B = Omega A, then per block J: b pivots from the
  sample, permutation of the whole column of the A/R array, panel QR of
  the b new leading columns, R12 and the trailing update by the block
  reflector, and the sample update of Eq. (3):
  B1 = S12 - S11 R11^{-1} R12,  B2 = S22.
* The unpivoted blocked QR of Table 3's note: RQRCP with every sample
  operation and every pivot removed.
* Alg. 6 (TRQRCP): no trailing update; selected columns are built as
  A - Y W^T, inner products W2^T = T2^T (Y2^T A - (Y2^T Y1) W1^T) (Sec. 5.1)
  and new rows of R from A - Y W^T.
* Alg. 7 (TUXV) with j_max = 1: Z0 = R P^T, [V, X0^T] = qr(Z0^T),
  Z1 = A V(:, 1:k), [U, X] = qr(Z1).

Readings where the paper is silent (each is listed in the design notes):

* Pivot ties: the first maximum in the current column order wins (Sec. 3.3
  notes that QRCP takes the lower index on a tie).
* Trailing-norm update of Alg. 1 (dropping the finished row): trailing sample
  norms are downdated multiplicatively, nrm *= sqrt(max(0, 1 - (|s_ij|/nrm)^2));
  when the downdated norm has lost more than half the digits relative to the
  last exactly computed norm (f * (nrm/nrm0)^2 <= sqrt(eps)), it is
  recomputed from the remaining rows and becomes the new reference.
* The sample-QRCP input in Alg. 6 reads B^{[J-1]} (as in Alg. 4).
* No sample update after the last block.
* If a diagonal entry of R11 is exactly zero the update formula is
  undefined; the sample is then re-drawn for the trailing matrix
  (an RSRQRCP step, Alg. 5) from Philox stream 0x100 + J and the returned
  info is 2.
* TRQRCP builds the selected columns on all m rows; W2 is formed only on
  columns that are still trailing.
* Alg. 4 runs k/b blocks, so b <= k is implied: a block size above the rank
  is clamped to k before the sample rank l = b + p is formed.
"""

import numpy as np

from .householder import (
    house,
    apply_reflector_left,
    panel_qr,
    unit_lower,
    t_factor,
    apply_block_transpose,
    form_q,
)
from .philox import gaussian_omega, gaussian_block

EPS = np.finfo(np.float64).eps
TOL3Z = np.sqrt(EPS)
RESAMPLE_STREAM_BASE = 0x100


class PivotMismatch(AssertionError):
    """Raised in replay mode when a forced pivot disagrees with a
    well-separated oracle choice."""


def _colnorms(X):
    return np.sqrt(np.einsum("ij,ij->j", X, X)) if X.shape[0] else np.zeros(X.shape[1])


def sample_qrcp(Bs, nsteps, ids=None, forced_ids=None, tie_rtol=1e-8, ties=None):
    """Partial QRCP (Alg. 1 halted after ``nsteps`` pivots) on the sample Bs.

    Bs (l x nc) is overwritten by S: its first ``nsteps`` columns become the
    upper-triangular S11 over S12 (zeros below the diagonal), the remaining
    columns hold S12 on rows < nsteps and S22 below.

    ids: optional int array (nc,) of column identities that is permuted along.
    forced_ids: replay mode -- the identity chosen by the device at each step;
      the oracle still computes its own choice and raises PivotMismatch when
      the two differ and the oracle's norms separate them by more than
      ``tie_rtol`` (relative); otherwise it follows the forced choice.
    ties: optional list collecting (step, own, forced, relative gap).

    Returns (swaps, Vb, taub): swap partner of each step (position i <-> swaps[i]),
    the sample reflectors (l x nsteps, unit leading entries) and their taus.
    """
    ell, nc = Bs.shape
    if ids is None:
        ids = np.arange(nc)
    vn = _colnorms(Bs)
    vn0 = vn.copy()
    swaps = np.zeros(nsteps, dtype=np.int64)
    Vb = np.zeros((ell, nsteps))
    taub = np.zeros(nsteps)
    for i in range(nsteps):
        # Alg. 1: index of the maximum trailing norm (first one on a tie).
        c = i + int(np.argmax(vn[i:]))
        if forced_ids is not None:
            hit = np.nonzero(ids[i:] == forced_ids[i])[0]
            if hit.size != 1:
                raise PivotMismatch(f"step {i}: forced column id {forced_ids[i]} is not trailing")
            cf = i + int(hit[0])
            if cf != c:
                top = vn[c]
                gap = (top - vn[cf]) / top if top > 0 else 0.0
                if gap > tie_rtol:
                    raise PivotMismatch(
                        f"step {i}: oracle picks id {ids[c]} (norm {vn[c]:.17g}), "
                        f"forced id {ids[cf]} (norm {vn[cf]:.17g}), gap {gap:.3g}")
                if ties is not None:
                    ties.append((i, int(ids[c]), int(ids[cf]), float(gap)))
                c = cf
        swaps[i] = c
        # Alg. 1: swap column i with the pivot.
        if c != i:
            Bs[:, [i, c]] = Bs[:, [c, i]]
            vn[[i, c]] = vn[[c, i]]
            vn0[[i, c]] = vn0[[c, i]]
            ids[[i, c]] = ids[[c, i]]
        if i >= ell:
            continue
        # Alg. 1: reflector from the new column i, applied to the trailing columns.
        v, t, beta = house(Bs[i:, i])
        Vb[i:, i] = v
        taub[i] = t
        apply_reflector_left(v, t, Bs[i:, i + 1:])
        Bs[i, i] = beta
        Bs[i + 1:, i] = 0.0
        # Alg. 1: remove the contribution of row i from the trailing norms
        # (elementwise over the trailing columns with a nonzero norm).
        cols = i + 1 + np.nonzero(vn[i + 1:] != 0.0)[0]
        r = np.abs(Bs[i, cols]) / vn[cols]
        f = np.maximum(0.0, (1.0 - r) * (1.0 + r))
        redo = f * (vn[cols] / vn0[cols]) ** 2 <= TOL3Z
        rc = cols[redo]
        vn[rc] = _colnorms(Bs[i + 1:, rc])
        vn0[rc] = vn[rc]
        keep = cols[~redo]
        vn[keep] *= np.sqrt(f[~redo])
    return swaps, Vb, taub


def qrcp(A, replay_jpvt=None, tie_rtol=1e-8, ties=None):
    """Deterministic QR with column pivoting, A P = Q R (Alg. 1 run to
    min(m, n) steps on A itself, with the xLAQP2 norm downdate and exact
    recomputation).  Returns (F, jpvt, tau): F holds R on and above the
    diagonal and the reflectors (unit leading entry implied) below it, the
    LAPACK xGEQP3 layout; jpvt[i] is the original index of column i of A P.
    replay_jpvt / tie_rtol / ties: as in ``sample_qrcp`` (follow another
    implementation's choice where the norms tie within tie_rtol)."""
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    k = min(m, n)
    ids = np.arange(n)
    _, Vb, taub = sample_qrcp(F, k, ids=ids, forced_ids=replay_jpvt, tie_rtol=tie_rtol,
                              ties=ties)
    for i in range(k):
        F[i + 1:, i] = Vb[i + 1:, i]
    return F, ids, taub


def _right_upper_solve(S11, R11):
    """W11 = S11 R11^{-1} for upper-triangular R11, column by column
    (W11[:, j] = (S11[:, j] - W11[:, :j] R11[:j, j]) / R11[j, j])."""
    bJ = R11.shape[0]
    W = np.zeros_like(S11)
    for j in range(bJ):
        W[:, j] = (S11[:, j] - W[:, :j] @ R11[:j, j]) / R11[j, j]
    return W


def _sample_update(S, bJ, R11, R12):
    """Eq. (3): [B1; B2] = [S12 - S11 R11^{-1} R12; S22]."""
    S11 = np.triu(S[:bJ, :bJ])
    S12 = S[:bJ, bJ:]
    S22 = S[bJ:, bJ:]
    W11 = _right_upper_solve(S11, np.triu(R11))
    return np.vstack([S12 - W11 @ R12, S22])


def _resample(seed, J, ell, trailing):
    """RSRQRCP step (Alg. 5): fresh GIID compression of the trailing matrix."""
    om = gaussian_block(seed, ell, trailing.shape[0], RESAMPLE_STREAM_BASE + J)
    return om @ trailing


def rqrcp(A, b, p, seed=0, k=None, omega=None, replay_jpvt=None, tie_rtol=1e-8,
          trace=None, ties=None, resample_every_block=False, omega_fn=None):
    """Randomized QR with column pivoting, Alg. 4, on a copy of A.

    resample_every_block: Alg. 5 (RSRQRCP) instead -- before every block after
      the first, a fresh GIID sample of the trailing matrix (Philox stream
      0x100 + J after block J) replaces the sample update of Eq. (3).
    omega_fn: optional omega_fn(J, rows) -> l x rows matrix used for those
      fresh samples instead of the Philox generator (J = 1, 2, ... counts the
      finished blocks).

    Returns (F, jpvt, tau, info): F holds R on and above the diagonal and the
    reflectors below it (rows j0.., columns of each panel); jpvt[c] is the
    original index of column c (0-based); info is 0, or 2 if a re-sample was
    needed (exactly singular R11).

    omega: optional explicit l x m compression matrix (l = omega.shape[0]);
      by default Omega is the seeded Philox GIID matrix with l = b + p.
    replay_jpvt: replay mode (see sample_qrcp); the device's jpvt.
    trace: optional list receiving a dict per block for the sample-update tests.
    """
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    kmax = min(m, n)
    k = kmax if k is None else int(k)
    b = min(b, k)
    if omega is None:
        ell = b + p
        omega = gaussian_omega(seed, ell, m)
    else:
        omega = np.asarray(omega, dtype=np.float64)
        ell = omega.shape[0]
    # Alg. 4: the initial sample B^[0] = Omega^[0] A^[0].
    B = omega @ F
    jpvt = np.arange(n)
    tau = np.zeros(k)
    info = 0
    J = 0
    for j0 in range(0, k, b):
        J += 1
        bJ = min(b, k - j0)
        forced = None if replay_jpvt is None else np.asarray(replay_jpvt)[j0:j0 + bJ]
        ids = jpvt[j0:].copy()
        Bin = B.copy() if trace is not None else None
        # Alg. 4: b column pivots from the sample, [Q_b, S, P_b] = qrcp(B, b).
        swaps, Vb, taub = sample_qrcp(B, bJ, ids=ids, forced_ids=forced,
                                      tie_rtol=tie_rtol, ties=ties)
        # Alg. 4: permute A^[J-1] and the completed rows of R (whole columns).
        for i, c in enumerate(swaps):
            if c != i:
                F[:, [j0 + i, j0 + c]] = F[:, [j0 + c, j0 + i]]
                jpvt[[j0 + i, j0 + c]] = jpvt[[j0 + c, j0 + i]]
        # Alg. 4: b reflectors and R11 from the new leading columns.
        tau[j0:j0 + bJ] = panel_qr(F[j0:, j0:j0 + bJ])
        Y = unit_lower(F[j0:, j0:j0 + bJ])
        T = t_factor(Y, tau[j0:j0 + bJ])
        # Alg. 4: R12 and the trailing matrix A^[J] = Q^T A^[J-1] P_b.
        apply_block_transpose(Y, T, F[j0:, j0 + bJ:])
        S = B
        if j0 + bJ < k:
            R11 = F[j0:j0 + bJ, j0:j0 + bJ]
            R12 = F[j0:j0 + bJ, j0 + bJ:]
            if resample_every_block:
                # Alg. 5: a new GIID compression of the updated trailing matrix.
                trailing = F[j0 + bJ:, j0 + bJ:]
                if omega_fn is None:
                    B = _resample(seed, J, ell, trailing)
                else:
                    B = np.asarray(omega_fn(J, trailing.shape[0]), dtype=np.float64) @ trailing
            elif np.any(np.diag(R11) == 0.0):
                info = 2
                B = _resample(seed, J, ell, F[j0 + bJ:, j0 + bJ:])
            else:
                # Alg. 4: the sample update, Eq. (3).
                B = _sample_update(S, bJ, R11, R12)
        if trace is not None:
            trace.append(dict(j0=j0, bJ=bJ, B_in=Bin, S=S.copy(), swaps=swaps.copy(),
                              Vb=Vb, taub=taub, Y=Y.copy(), T=T.copy(),
                              B_out=B.copy() if j0 + bJ < k else None))
    return F, jpvt, tau, info


def rsrqrcp(A, b, p, seed=0, k=None, replay_jpvt=None, tie_rtol=1e-8, ties=None,
            omega=None, omega_fn=None):
    """Repeated-sampling RQRCP, Alg. 5: Alg. 4 with the sample of every block
    formed anew from the trailing matrix, B^[J] = Omega^[J] A^[J] (Omega^[0]
    as in Alg. 4, then Philox stream 0x100 + J).  Same returns as rqrcp."""
    return rqrcp(A, b, p, seed=seed, k=k, omega=omega, replay_jpvt=replay_jpvt,
                 tie_rtol=tie_rtol, ties=ties, resample_every_block=True, omega_fn=omega_fn)


def qr_blocked(A, b):
    """Unpivoted blocked Householder QR: Alg. 4 with the sample and the
    pivoting removed (Table 3 note).  Returns (F, tau) in in-place storage."""
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    k = min(m, n)
    tau = np.zeros(k)
    for j0 in range(0, k, b):
        bJ = min(b, k - j0)
        tau[j0:j0 + bJ] = panel_qr(F[j0:, j0:j0 + bJ])
        Y = unit_lower(F[j0:, j0:j0 + bJ])
        T = t_factor(Y, tau[j0:j0 + bJ])
        apply_block_transpose(Y, T, F[j0:, j0 + bJ:])
    return F, tau


def trqrcp(A, k, b, p, seed=0, omega=None, replay_jpvt=None, tie_rtol=1e-8, ties=None):
    """Truncated RQRCP without trailing update, Alg. 6.

    A is not modified.  Returns (jpvt, tau, Y, R, info): jpvt (n,) with the
    k selected original indices first; tau (k,); Y (m x k) unit lower
    trapezoidal reflectors; R (k x n) upper trapezoidal in the permuted
    column order, so that A[:, jpvt] ~= Q[:, :k] R.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    k = int(k)
    b = min(b, k)
    if omega is None:
        ell = b + p
        omega = gaussian_omega(seed, ell, m)
    else:
        omega = np.asarray(omega, dtype=np.float64)
        ell = omega.shape[0]
    Ap = A.copy()                 # A^[J]: the permuted (never updated) matrix
    B = omega @ A                 # Alg. 6: B^[0] = Omega^[0] A^[0]
    jpvt = np.arange(n)
    tau = np.zeros(k)
    Y = np.zeros((m, k))
    Wt = np.zeros((k, n))         # W^T, columns in the current order
    R = np.zeros((k, n))
    info = 0
    J = 0
    for j0 in range(0, k, b):
        J += 1
        bJ = min(b, k - j0)
        forced = None if replay_jpvt is None else np.asarray(replay_jpvt)[j0:j0 + bJ]
        ids = jpvt[j0:].copy()
        # Alg. 6: b pivots from the sample.
        swaps, _, _ = sample_qrcp(B, bJ, ids=ids, forced_ids=forced,
                                  tie_rtol=tie_rtol, ties=ties)
        # Alg. 6: permute A, the completed rows of R and the prior inner products.
        for i, c in enumerate(swaps):
            if c != i:
                a, z = j0 + i, j0 + c
                Ap[:, [a, z]] = Ap[:, [z, a]]
                jpvt[[a, z]] = jpvt[[z, a]]
                Wt[:, [a, z]] = Wt[:, [z, a]]
                R[:, [a, z]] = R[:, [z, a]]
        # Alg. 6: construct the selected columns from A^[J] - Y^[J-1] W1^[J]T.
        Ahat = Ap[:, j0:j0 + bJ] - Y[:, :j0] @ Wt[:j0, j0:j0 + bJ]
        # Rows above j0 of A_hat repeat entries of R that earlier blocks
        # already computed and permuted; only rows j0.. are factored.
        # Alg. 6: reflectors Y2 and R11 from qr(A_hat) (rows j0..m-1).
        P = Ahat[j0:, :].copy()
        tau[j0:j0 + bJ] = panel_qr(P)
        Y[j0:, j0:j0 + bJ] = unit_lower(P)
        R[j0:j0 + bJ, j0:j0 + bJ] = np.triu(P[:bJ, :bJ])
        Y1 = Y[:, :j0]
        Y2 = Y[:, j0:j0 + bJ]
        T2 = t_factor(Y2[j0:], tau[j0:j0 + bJ])
        # Alg. 6: W2^T = T2^T (Y2^T A - (Y2^T Y1) W1^T) on the trailing columns.
        tc = slice(j0 + bJ, n)
        Wt[j0:j0 + bJ, tc] = T2.T @ (Y2.T @ Ap[:, tc] - (Y2.T @ Y1) @ Wt[:j0, tc])
        # Alg. 6: new rows of R from A^[J] - Y^[J] W^[J]T.
        R[j0:j0 + bJ, tc] = Ap[j0:j0 + bJ, tc] - Y[j0:j0 + bJ, :j0 + bJ] @ Wt[:j0 + bJ, tc]
        if j0 + bJ < k:
            R11 = R[j0:j0 + bJ, j0:j0 + bJ]
            R12 = R[j0:j0 + bJ, tc]
            if np.any(np.diag(R11) == 0.0):
                info = 2
                trailing = Ap[j0 + bJ:, tc] - Y[j0 + bJ:, :j0 + bJ] @ Wt[:j0 + bJ, tc]
                B = _resample(seed, J, ell, trailing)
            else:
                # Alg. 6: the sample update, Eq. (3).
                B = _sample_update(B, bJ, R11, R12)
    return jpvt, tau, Y, R, info


def tuxv(A, k, b, p, seed=0, omega=None, replay_jpvt=None, tie_rtol=1e-8, ties=None, jmax=1):
    """Approximate truncated SVD, Alg. 7 (j_max LQ-QR iterations; the paper
    sets j_max = 1).

    Returns (U, X, V, jpvt, info) with U (m x k) and V (n x k) having
    orthonormal columns and X (k x k) upper triangular after an odd number
    of iterations and lower triangular after an even number, A ~= U X V^T.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    jpvt, _, _, R, info = trqrcp(A, k, b, p, seed=seed, omega=omega,
                                 replay_jpvt=replay_jpvt, tie_rtol=tie_rtol, ties=ties)
    # Alg. 7: restore the original column order, Z0 = R P^T.
    Z0 = np.zeros((k, n))
    Z0[:, jpvt] = R
    # Alg. 7: LQ of Z0 as the QR of Z0^T; V's leading k columns explicitly.
    Zt = Z0.T.copy()
    tv = panel_qr(Zt)
    V = form_q(Zt, tv, k)
    j = 1
    while True:
        # Alg. 7: Z^(j) = A V(:, 1:k), then [U, X] = qr(Z^(j)).
        Z = A @ V
        tu = panel_qr(Z)
        X = np.triu(Z[:k, :k])
        U = form_q(Z, tu, k)
        if j == jmax:
            break
        # Alg. 7: Z^(j+1) = U(:, 1:k)^T A, LQ of it as the QR of its transpose.
        Zt = U.T @ A
        Zt = Zt.T.copy()
        tv = panel_qr(Zt)
        X = np.triu(Zt[:k, :k]).T
        V = form_q(Zt, tv, k)
        if j + 1 == jmax:
            break
        j += 2
    return U, X, V, jpvt, info


def tuxv_svd(A, k, b, p, seed=0, jmax=1, omega=None, replay_jpvt=None, tie_rtol=1e-8,
             ties=None):
    """Alg. 7 followed by the SVD of the k x k connection matrix X, which the
    paper suggests for better singular value estimates than the diagonal of X:
    X = Ux diag(sigma) Vs^T, returned as (U Ux, sigma, V Vs, jpvt, info) with
    sigma descending, so that A ~= U diag(sigma) V^T.  The SVD of X is LAPACK's
    (numpy), the plain definition of this step."""
    U, X, V, jpvt, info = tuxv(A, k, b, p, seed=seed, omega=omega, replay_jpvt=replay_jpvt,
                               tie_rtol=tie_rtol, ties=ties, jmax=jmax)
    Ux, sigma, VsT = np.linalg.svd(X)
    return U @ Ux, sigma, V @ VsT.T, jpvt, info
