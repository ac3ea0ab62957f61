"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (same b, p and seed):

* 16384^2 graded FP64 RQRCP (b = 64, p = 8, Omega seed 1), native FP64 and
  with the two handle options (the trailing update as FP64-accurate slice
  products on the tensor cores; Alg. 5's fresh sample per block):
  - the whole reconstruction ||A P - Q R||_F / ||A||_F <= 1e-13 over all
    16384 columns, with Q applied in FP64 by plain torch products (compact
    WY blocks built here from the stored reflectors, independent of the CUDA
    path);
  - orthogonality ||Q^T Q e_S - e_S|| on 64 sampled columns;
  - the oracle replays the first 6 blocks (384 pivots): pivots identical
    outside 1e-8 near-ties, the 384 R rows (matched by original column)
    within 1e-10 normwise, tau within 1e-9 where |R_ii| >= 1e-6 |R_00|.
* 16384^2 mixed RQRCP (b = 128, p = 16) on the spiked matrix: the whole
  reconstruction ||A P - Q R||_F / ||A||_F <= 1e-6 in FP64.
* 50000 x 20000, k = 512 TRQRCP + TUXV: orthonormal factors, the TUXV error
  below TRQRCP's own and within 5 % of the Eckart-Young value of the known
  spectrum plus noise.

Each FP64 case takes about 60-90 s (16 s of it the oracle).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _wy_blocks(F, tau, b):
    """Compact-WY blocks (j0, Y, T) of Q = H_0 H_1 ... H_{k-1} from reflectors
    stored below the diagonal of F (float64, on the device): Q_J = I - Y T Y^T
    with T upper triangular from the forward recurrence
    T[:i, i] = -tau_i T[:i, :i] (Y^T Y)[:i, i], T[i, i] = tau_i."""
    k = tau.shape[0]
    out = []
    for j0 in range(0, k, b):
        bJ = min(b, k - j0)
        Y = torch.tril(F[j0:, j0:j0 + bJ], -1)
        Y[torch.arange(bJ), torch.arange(bJ)] = 1.0
        G = (Y.t() @ Y).cpu().numpy()
        t = tau[j0:j0 + bJ].cpu().numpy()
        T = np.zeros((bJ, bJ))
        for i in range(bJ):
            T[:i, i] = -t[i] * (T[:i, :i] @ G[:i, i])
            T[i, i] = t[i]
        out.append((j0, Y, torch.from_numpy(T).to(F.device)))
    return out


def _apply_q(blocks, X, row_hi=None):
    """Q X for X (m x c); rows >= row_hi of X are zero when given."""
    for j0, Y, T in reversed(blocks):
        if row_hi is not None and j0 >= row_hi:
            continue
        X[j0:] -= Y @ (T @ (Y.t() @ X[j0:]))
    return X


def _apply_qt(blocks, X):
    for j0, Y, T in blocks:
        X[j0:] -= Y @ (T.t() @ (Y.t() @ X[j0:]))
    return X


def _full_recon_err(A, F, tau, jpvt, b, chunk=2048):
    """||A[:, jpvt] - Q R||_F / ||A||_F over every column, in FP64 on the
    device, R = triu(F); F may be float32 (converted chunk by chunk)."""
    n = F.shape[1]
    Fd = F if F.dtype == torch.float64 else None
    blocks = _wy_blocks(F.double() if Fd is None else Fd, tau, b)
    rows = torch.arange(F.shape[0], device=F.device)[:, None]
    err2 = 0.0
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        cols = torch.arange(c0, c1, device=F.device)
        X = F[:, c0:c1].double() * (rows <= cols[None, :])
        X = _apply_q(blocks, X, row_hi=c1)
        err2 += ((A[:, jpvt[c0:c1]].double() - X) ** 2).sum().item()
    return (err2 ** 0.5) / torch.linalg.norm(A.double()).item(), blocks


def _orth_err(blocks, m, dev, ncols=64, seed=6):
    g = torch.Generator().manual_seed(seed)
    cols = torch.randperm(m, generator=g)[:ncols].to(dev)
    E = torch.zeros((m, ncols), dtype=torch.float64, device=dev)
    E[cols, torch.arange(ncols, device=dev)] = 1.0
    X = _apply_qt(blocks, _apply_q(blocks, E.clone()))
    return (X - E).norm().item() / ncols ** 0.5


def _replay_first_blocks(A_host, F_top, t_top, jp, b, p, seed, nblk, resample=False):
    """The oracle's first nblk blocks, following the device's pivots through
    near-ties; returns (R error normwise, max tau error on significant rows,
    ties)."""
    k0 = nblk * b
    n = A_host.shape[1]
    ties = []
    fn = oracle.rsrqrcp if resample else oracle.rqrcp
    Fo, jo, to, info_o = fn(A_host, b, p, seed=seed, k=k0, replay_jpvt=jp, ties=ties)
    assert info_o == 0
    np.testing.assert_array_equal(jo[:k0], jp[:k0])
    pos_o = np.empty(n, dtype=np.int64)
    pos_o[jo] = np.arange(n)
    Ro = np.triu(Fo[:k0])[:, pos_o[jp]]
    Rg = np.triu(F_top)
    r_err = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    sig = np.abs(np.diag(Ro[:, :k0])) >= 1e-6 * abs(Ro[0, 0])
    t_err = np.abs(t_top - to[:k0])[sig].max()
    return r_err, t_err, ties


@pytest.mark.parametrize("option", ["native", "fp64_emulation", "resample"])
def test_fullsize_rqrcp_fp64_graded(lib, option):
    n, b, p, seed = 16384, 64, 8, 1
    dev = torch.device("cuda")
    h = lib.Handle()
    if option == "fp64_emulation":
        h.set_fp64_emulation(True)
    elif option == "resample":
        h.set_resample(True)
    A = synth.graded_device(n, dev)
    dA = lib.colmajor(A.clone())
    jpvt, tau = lib.rqrcp_factor(dA, b, p, seed, handle=h)
    assert h.sync_info() == 0
    jp = jpvt.cpu().numpy()
    assert np.array_equal(np.sort(jp), np.arange(n))

    err, blocks = _full_recon_err(A, dA, tau, jpvt, b)
    assert err <= 1e-13, err
    orth = _orth_err(blocks, n, dev)
    assert orth <= 1e-13, orth
    del blocks

    # the oracle's first 6 blocks, replaying the device's pivots through ties
    k0 = 6 * b
    A_host = np.asfortranarray(A.cpu().numpy())
    F_top = dA[:k0].cpu().numpy()
    t_top = tau[:k0].cpu().numpy()
    del dA, A
    torch.cuda.empty_cache()
    r_err, t_err, ties = _replay_first_blocks(A_host, F_top, t_top, jp, b, p, seed, 6,
                                              resample=(option == "resample"))
    assert len(ties) <= 2, ties
    assert r_err <= 1e-10, r_err
    assert t_err <= 1e-9, t_err


def test_fullsize_rqrcp_mixed_spiked(lib):
    n, b, p = 16384, 128, 16
    dev = torch.device("cuda")
    A0 = lib.colmajor(synth.spiked_device(n, n, dev).float())
    A = lib.colmajor(A0.clone())
    jpvt, tau, rdiag = lib.rqrcp_factor_mixed(A, b, p, 1)
    assert lib.sync_info() == 0
    assert torch.equal(torch.sort(jpvt).values, torch.arange(n, device=dev))
    # R's diagonal is returned in FP64; the stored one is its FP32 rounding
    F = A.double()
    F[torch.arange(n, device=dev), torch.arange(n, device=dev)] = rdiag
    err, _ = _full_recon_err(A0, F, tau, jpvt, b)
    assert err <= 1e-6, err


def test_fullsize_trqrcp_tuxv(lib):
    m, n, k, b, p = 50000, 20000, 512, 64, 8
    dev = torch.device("cuda")
    A = lib.colmajor(synth.decaying_lowrank_device(m, n, dev, rank=2048, noise=1e-8))
    jpvt, tau, Y, R = lib.trqrcp(A, k, b, p, 1)
    U, X, V = lib.tuxv(A, k, b, p, 1)
    assert lib.sync_info() == 0
    eye = torch.eye(k, device=dev, dtype=torch.float64)
    assert (U.t() @ U - eye).abs().max().item() <= 1e-13
    assert (V.t() @ V - eye).abs().max().item() <= 1e-13
    assert torch.allclose(torch.tril(X, -1), torch.zeros_like(X))
    a2 = (A ** 2).sum().item()
    # TRQRCP: R = Q_k^T A P, so ||A - Q_k Q_k^T A||^2 = ||A||^2 - ||R||^2
    e_tr = (max(a2 - (R ** 2).sum().item(), 0.0) / a2) ** 0.5
    # TUXV: ||A - U X V^T||^2 = ||A||^2 - 2 <U^T A V, X> + ||X||^2
    e_tx = (max(a2 - 2.0 * ((U.t() @ A @ V) * X).sum().item() + (X ** 2).sum().item(), 0.0)
            / a2) ** 0.5
    # Eckart-Young value of the known spectrum plus the noise energy (1e-8^2
    # per entry), which dominates the tail
    sig = torch.arange(1, 2049, dtype=torch.float64) ** -2.0
    e_opt = (((sig[k:] ** 2).sum().item() + 1e-16 * m * n) / a2) ** 0.5
    assert e_tx <= e_tr * (1 + 1e-9)
    assert 0.99 * e_opt <= e_tx <= 1.05 * e_opt, (e_tx, e_opt)
