"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (default handle, same b, p and seed):

* 16384^2 graded FP64 RQRCP (b = 64, p = 8, Omega seed 1): the oracle runs the
  first 6 blocks (384 pivots) in replay mode; pivots, the 384 R rows (matched
  by original column) and tau are compared with the same tolerances as the
  small cases, and A P = Q R is checked on sampled columns with Q applied in
  FP64 by plain torch operations.
* 16384^2 mixed RQRCP (b = 128, p = 16) on the spiked matrix: reconstruction
  of sampled columns within 1e-6.
* 50000 x 20000, k = 512 TRQRCP + TUXV: orthonormal factors, the TUXV error
  below TRQRCP's own and within 5 % of the Eckart-Young value of the known
  spectrum plus noise.

The FP64 case takes about 70 s (16 s of it the oracle), the others under 20 s.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _apply_q(F, tau, X):
    """Q X with Q = H_0 H_1 ... H_{k-1} from the reflectors stored below the
    diagonal of F (column-major, on the device), X on the device."""
    k = tau.shape[0]
    for i in range(k - 1, -1, -1):
        v = F[i:, i].clone()
        v[0] = 1.0
        X[i:] -= tau[i] * torch.outer(v, v @ X[i:])
    return X


def test_fullsize_rqrcp_fp64_graded(lib):
    n, b, p, seed = 16384, 64, 8, 1
    dev = torch.device("cuda")
    A = synth.graded_device(n, dev)
    dA = lib.colmajor(A.clone())
    jpvt, tau = lib.rqrcp_factor(dA, b, p, seed)
    assert lib.sync_info() == 0
    jp = jpvt.cpu().numpy()
    assert np.array_equal(np.sort(jp), np.arange(n))

    # sampled columns: A(:, jpvt[c]) = Q R(:, c)
    g = torch.Generator().manual_seed(3)
    cols = torch.randperm(n, generator=g)[:16].to(dev)
    rows = torch.arange(n, device=dev)[:, None]
    X = dA[:, cols] * (rows <= cols[None, :])
    X = _apply_q(dA, tau, X)
    ref = A[:, jpvt[cols]]
    err = (ref - X).norm(dim=0).max().item() / torch.linalg.norm(A).item()
    assert err <= 1e-13, err

    # the oracle's first 6 blocks, replaying the device's pivots through ties
    k0 = 6 * b
    A_host = np.asfortranarray(A.cpu().numpy())
    F_dev = dA[:k0].cpu().numpy()
    t_dev = tau[:k0].cpu().numpy()
    del dA, A
    ties = []
    Fo, jo, to, info_o = oracle.rqrcp(A_host, b, p, seed=seed, k=k0, replay_jpvt=jp, ties=ties)
    assert info_o == 0
    assert len(ties) <= 2, ties
    np.testing.assert_array_equal(jo[:k0], jp[:k0])
    # R rows 0..k0-1, columns matched by their original index
    pos_o = np.empty(n, dtype=np.int64)
    pos_o[jo] = np.arange(n)
    Ro = np.triu(Fo[:k0])[:, pos_o[jp]]
    Rg = np.triu(F_dev)
    assert np.linalg.norm(Rg - Ro) <= 1e-10 * np.linalg.norm(Ro)
    sig = np.abs(np.diag(Ro[:, :k0])) >= 1e-6 * abs(Ro[0, 0])
    assert np.abs(t_dev - to[:k0])[sig].max() <= 1e-9


def test_fullsize_rqrcp_mixed_spiked(lib):
    n, b, p = 16384, 128, 16
    dev = torch.device("cuda")
    A0 = lib.colmajor(synth.spiked_device(n, n, dev).float())
    A = lib.colmajor(A0.clone())
    jpvt, tau, rdiag = lib.rqrcp_factor_mixed(A, b, p, 1)
    assert lib.sync_info() == 0
    g = torch.Generator().manual_seed(5)
    cols = torch.randperm(n, generator=g)[:8].to(dev)
    V = A.double()
    rows = torch.arange(n, device=dev)[:, None]
    X = V[:, cols] * (rows <= cols[None, :])
    X[cols, torch.arange(8, device=dev)] = rdiag[cols]
    X = _apply_q(V, tau, X)
    ref = A0[:, jpvt[cols]].double()
    err = ((ref - X).norm(dim=0) / ref.norm(dim=0)).max().item()
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


@pytest.mark.parametrize("option", ["fp64_emulation", "resample"])
def test_fullsize_rqrcp_options(lib, option):
    """The same 16384^2 graded factorization with the trailing update on the
    tensor cores (exact slices) or with Alg. 5's fresh sample per block:
    A P = Q R on sampled columns to the FP64 bound."""
    n, b, p = 16384, 64, 8
    dev = torch.device("cuda")
    h = lib.Handle()
    if option == "fp64_emulation":
        h.set_fp64_emulation(True)
    else:
        h.set_resample(True)
    A = synth.graded_device(n, dev)
    dA = lib.colmajor(A.clone())
    jpvt, tau = lib.rqrcp_factor(dA, b, p, 1, handle=h)
    assert h.sync_info() == 0
    assert torch.equal(torch.sort(jpvt).values, torch.arange(n, device=dev))
    g = torch.Generator().manual_seed(4)
    cols = torch.randperm(n, generator=g)[:16].to(dev)
    rows = torch.arange(n, device=dev)[:, None]
    X = _apply_q(dA, tau, dA[:, cols] * (rows <= cols[None, :]))
    err = (A[:, jpvt[cols]] - X).norm(dim=0).max().item() / torch.linalg.norm(A).item()
    assert err <= 1e-13, err
