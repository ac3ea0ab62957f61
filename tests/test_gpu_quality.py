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
