"""Selection quality of the device's sample pivoting (Fig. selectExpect):
the first pivot that the seeded Philox sample and the sample QRCP kernel pick
on a matrix with orthogonal columns of norms phi^j, over many seeds, against
the exact expectation of the oracle."""
import numpy as np
import pytest
import torch

from oracle import selection

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("phi,ell", [(0.9, 8), (0.8, 16), (0.95, 8)])
def test_sample_pivot_expectation(lib, phi, ell):
    m, n, trials = 96, 32, 3000
    g = torch.Generator().manual_seed(17)
    Q = torch.linalg.qr(torch.randn((m, n), generator=g, dtype=torch.float64))[0]
    A = lib.colmajor((Q * phi ** torch.arange(n, dtype=torch.float64)).cuda())
    picks = []
    for seed in range(1, trials + 1):
        B = lib.sketch(A, ell, seed)
        picks.append(lib.sample_qrcp(B, 1)[:1])
    J = torch.cat(picks).cpu().numpy()
    assert lib.sync_info() == 0
    vals = phi ** J.astype(np.float64)
    exact = selection.select_expectation(phi, ell, n)
    se = vals.std() / np.sqrt(trials)
    assert abs(vals.mean() - exact) <= 5 * se, (vals.mean(), exact, se)
    assert exact > 0.9


def test_error_vs_rank_ordering(lib):
    """Error-vs-rank on a matrix whose large columns are nearly collinear:
    the SVD bounds everything (Eckart-Young), TUXV never does worse than the
    truncated RQRCP it starts from, RQRCP stays within a small factor of
    deterministic QRCP, and unpivoted QR after presorting by norm fails to
    reveal the rank (its error stalls while the pivoted methods drop)."""
    n, b, p = 600, 32, 8
    g = torch.Generator().manual_seed(3)
    h = n // 2
    C = torch.randn(n, 5, generator=g, dtype=torch.float64) @ torch.randn(5, h, generator=g,
                                                                          dtype=torch.float64)
    C = C / C.norm(dim=0, keepdim=True) + 1e-8 * torch.randn(n, h, generator=g, dtype=torch.float64)
    U = torch.linalg.qr(torch.randn(n, h, generator=g, dtype=torch.float64))[0]
    V = torch.linalg.qr(torch.randn(h, h, generator=g, dtype=torch.float64))[0]
    D = (U * (0.3 / torch.arange(1, h + 1, dtype=torch.float64))) @ V.T
    A = torch.cat([C, D], dim=1).cuda()
    nrm = torch.linalg.norm(A)

    def tail(F):
        r2 = (torch.triu(F) ** 2).sum(dim=1)
        return torch.sqrt(torch.flip(torch.cumsum(torch.flip(r2, [0]), 0), [0])) / nrm

    F = lib.colmajor(A[:, torch.argsort(A.norm(dim=0), descending=True)].clone())
    lib.qr_factor(F, b)
    e_qr = tail(F)
    F = lib.colmajor(A.clone())
    lib.rqrcp_factor(F, b, p, 1)
    e_rq = tail(F)
    F = lib.colmajor(A.clone())
    lib.qrcp_factor(F, b)
    e_cp = tail(F)
    s = torch.linalg.svdvals(A)
    e_svd = torch.sqrt(torch.flip(torch.cumsum(torch.flip(s ** 2, [0]), 0), [0])) / nrm
    for k in (10, 40, 100, 200):
        Uk, Xk, Vk = lib.tuxv(lib.colmajor(A.clone()), k, b, p, 1)
        e_tx = torch.linalg.norm(A - Uk @ Xk @ Vk.T) / nrm
        assert e_svd[k] <= e_tx * (1 + 1e-10)
        assert e_tx <= e_rq[k] * (1 + 1e-10)
        assert e_rq[k] <= 1.5 * e_cp[k]
        # at k = 10 the unpivoted method spends 5 of its 10 columns on the
        # collinear block (ideal ratio ~3); beyond that it has spent k - 5
        assert e_qr[k] >= (2 if k < 40 else 3) * e_cp[k]
    assert lib.sync_info() == 0
