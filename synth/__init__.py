"""Seeded synthetic input matrices shaped like the paper's workloads.

This module is shared by the tests, the bench and the oracle checks.  It
holds none of the factorization arithmetic: it only draws matrices.  The
compression matrix Omega is NOT drawn here -- it belongs to the method and
is generated independently on each side from the Philox definition.

The paper times Gaussian i.i.d. matrices (Sec. 7.1, Sec. 7.2) and measures
quality on matrices with decaying spectra (Sec. 7.3).  The generators below give:

* ``gaussian``        -- i.i.d. N(0,1) entries.
* ``graded``          -- U diag(sigma) V^T with Haar U, V (QR of a seeded
                         Gaussian, signs fixed by diag(R)) and
                         sigma_i = 10^(-decades (i-1)/(n-1)).
* ``spiked``          -- N(0,1) plus a rank-r spike of scale s built from
                         orthonormal factors.
* ``decaying_lowrank``-- U_r diag(i^-2) V_r^T of rank r plus N(0, noise^2).
* ``factor_product``  -- X Y^T with Gaussian X (m x k), Y (n x k).
* ``separated_columns`` -- orthogonal columns with norms phi^(j-1) in a
                         shuffled order (the Fig. selectExpect setup).

``*_device`` variants build the large matrices on a torch device in float64;
they are used for sizes whose host construction would take minutes.
"""

import numpy as np


def _rng(seed):
    return np.random.default_rng(int(seed))


def gaussian(m, n, seed=0):
    return _rng(seed).standard_normal((m, n))


def haar(n, seed):
    """Haar-distributed orthogonal n x n matrix: Q of a Gaussian's QR with
    the sign of diag(R) moved into Q."""
    G = _rng(seed).standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def graded_sigma(n, decades=12.0):
    i = np.arange(n, dtype=np.float64)
    return 10.0 ** (-decades * i / max(n - 1, 1))


def graded(n, seed_u=2, seed_v=3, decades=12.0):
    U = haar(n, seed_u)
    V = haar(n, seed_v)
    return (U * graded_sigma(n, decades)[None, :]) @ V.T


def _orthonormal(m, r, seed):
    Q, R = np.linalg.qr(_rng(seed).standard_normal((m, r)))
    return Q * np.sign(np.diag(R))[None, :]


def spiked(m, n, rank=512, scale=1e3, seed_g=0, seed_u=2, seed_v=3):
    G = gaussian(m, n, seed_g)
    return G + scale * (_orthonormal(m, rank, seed_u) @ _orthonormal(n, rank, seed_v).T)


def decaying_lowrank(m, n, rank=2048, noise=1e-8, seed_u=2, seed_v=3, seed_noise=4):
    sig = np.arange(1, rank + 1, dtype=np.float64) ** -2.0
    A = (_orthonormal(m, rank, seed_u) * sig[None, :]) @ _orthonormal(n, rank, seed_v).T
    if noise:
        A += noise * gaussian(m, n, seed_noise)
    return A


def factor_product(m, n, k, seed):
    r = _rng(seed)
    X = r.standard_normal((m, k))
    Y = r.standard_normal((n, k))
    return X @ Y.T


def separated_columns(m, n, phi=1e-2, seed=5):
    """Orthogonal columns with norms phi^(j-1), columns shuffled.
    Returns (A, order) where order[t] is the column holding the t-th largest."""
    r = _rng(seed)
    Q = _orthonormal(m, n, seed + 1000)
    A = Q * (phi ** np.arange(n, dtype=np.float64))[None, :]
    perm = r.permutation(n)
    A = A[:, perm]
    order = np.argsort(perm)
    return A, order


# ---------------------------------------------------------------- device side

def _torch():
    import torch
    return torch


def _dev_gen(device, seed):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian_device(m, n, seed, device, dtype=None):
    """N(0,1) m x n matrix, column-major storage (a transposed row-major
    tensor), drawn with torch's device generator."""
    torch = _torch()
    dtype = dtype or torch.float64
    return torch.randn((n, m), generator=_dev_gen(device, seed), device=device, dtype=dtype).t()


def _orthonormal_device(m, r, seed, device):
    torch = _torch()
    G = torch.randn((m, r), generator=_dev_gen(device, seed), device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    return Q * torch.sign(torch.diagonal(R))[None, :]


def graded_device(n, device, seed_u=2, seed_v=3, decades=12.0):
    """U diag(sigma) V^T on the device; column-major n x n (a .t() view)."""
    torch = _torch()
    U = _orthonormal_device(n, n, seed_u, device)
    V = _orthonormal_device(n, n, seed_v, device)
    sig = torch.as_tensor(graded_sigma(n, decades), device=device)
    At = V @ (U * sig[None, :]).t()          # A^T, row-major == A column-major
    del U, V
    return At.t()


def spiked_device(m, n, device, rank=512, scale=1e3, seed_g=0, seed_u=2, seed_v=3):
    Ut = _orthonormal_device(m, rank, seed_u, device)
    Vt = _orthonormal_device(n, rank, seed_v, device)
    A = gaussian_device(m, n, seed_g, device)
    A.t().add_(scale * (Vt @ Ut.t()))
    return A


def decaying_lowrank_device(m, n, device, rank=2048, noise=1e-8, seed_u=2, seed_v=3, seed_noise=4):
    torch = _torch()
    Ur = _orthonormal_device(m, rank, seed_u, device)
    Vr = _orthonormal_device(n, rank, seed_v, device)
    sig = torch.arange(1, rank + 1, device=device, dtype=torch.float64) ** -2.0
    At = Vr @ (Ur * sig[None, :]).t()
    if noise:
        At.add_(noise * torch.randn((n, m), generator=_dev_gen(device, seed_noise),
                                    device=device, dtype=torch.float64))
    return At.t()


def factor_product_device(m, n, k, seed, device, dtype=None):
    torch = _torch()
    g = _dev_gen(device, seed)
    X = torch.randn((m, k), generator=g, device=device, dtype=torch.float64)
    Y = torch.randn((n, k), generator=g, device=device, dtype=torch.float64)
    At = Y @ X.t()
    return At.t().to(dtype or torch.float64)
