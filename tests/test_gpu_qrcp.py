"""GPU parity of the deterministic QRCP (level-3 reflection blocking) against
the CPU oracle's QRCP (Alg. 1 on A itself, xLAQP2 norm handling).

Tolerances as for RQRCP: pivots equal wherever the oracle's trailing norms
separate the GPU's choice from its own by more than 1e-8 relative (replay
follows the GPU through closer ties); ||R - R_oracle||_F / ||R||_F <= 1e-10;
||A P - Q R||_F / ||A||_F <= 1e-13.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import householder as hh
import synth

pytestmark = pytest.mark.gpu


def to_dev(A):
    import paper_1509_06820_gb300 as rq
    return rq.colmajor(torch.from_numpy(np.asarray(A, dtype=np.float64)).cuda())


def _check_qrcp(lib, A, b, max_ties=2):
    m, n = A.shape
    k = min(m, n)
    dA = to_dev(A)
    jpvt, tau = lib.qrcp_factor(dA, b)
    assert lib.sync_info() == 0
    F, jp, t = dA.cpu().numpy(), jpvt.cpu().numpy(), tau.cpu().numpy()
    assert sorted(jp.tolist()) == list(range(n))
    ties = []
    Fo, jo, to = oracle.qrcp(A, replay_jpvt=jp, ties=ties)
    np.testing.assert_array_equal(jo, jp)
    assert len(ties) <= max_ties, ties
    Ro = np.triu(Fo[:k])
    assert np.linalg.norm(np.triu(F[:k]) - Ro) <= 1e-10 * np.linalg.norm(Ro)
    sig = np.abs(np.diag(Ro)) >= 1e-6 * abs(Ro[0, 0])
    assert np.abs(t - to)[sig].max() <= 1e-9
    Q = hh.form_q(F, t, k)
    assert np.linalg.norm(A[:, jp] - Q @ np.triu(F[:k])) <= 1e-13 * np.linalg.norm(A)
    return F, jp, t


@pytest.mark.parametrize("m,n,b", [(300, 200, 32), (200, 300, 32), (257, 513, 64), (600, 150, 16),
                                   (1, 1, 1), (1, 40, 8), (40, 1, 8), (100, 100, 128),
                                   (130, 90, 7)])
def test_qrcp_matches_oracle(lib, m, n, b):
    A = synth.gaussian(m, n, seed=m + n)
    _check_qrcp(lib, A, b)


def test_qrcp_graded_recomputes_norms(lib):
    """Singular values 1 .. 1e-12: downdated norms lose their digits several
    times, so blocks end early and the norms are recomputed exactly."""
    A = synth.graded(400, decades=12.0)
    _check_qrcp(lib, A, 32, max_ties=4)


def test_qrcp_wide_unchunked(lib):
    """More trailing columns than warps in the grid: the level-2 pass takes one
    warp per whole column (no row chunks)."""
    A = synth.gaussian(300, 3000, seed=5)
    _check_qrcp(lib, A, 64)


def test_qrcp_tall_beyond_staged_rows(lib):
    """m above the rows of the reflector kept in shared memory: the rest of y
    is read from global memory."""
    A = synth.gaussian(30000, 48, seed=6)
    _check_qrcp(lib, A, 16)


def test_qrcp_is_deterministic(lib):
    A = synth.gaussian(500, 400, seed=8)
    d1, d2 = to_dev(A), to_dev(A)
    j1, t1 = lib.qrcp_factor(d1, 32)
    j2, t2 = lib.qrcp_factor(d2, 32)
    assert torch.equal(j1, j2) and torch.equal(t1, t2) and torch.equal(d1, d2)


def test_qrcp_diag_non_increasing(lib):
    """QRCP's R has a non-increasing diagonal in magnitude (Alg. 1 pivots the
    largest trailing norm, which is |R_jj|)."""
    A = synth.gaussian(700, 500, seed=9)
    dA = to_dev(A)
    lib.qrcp_factor(dA, 64)
    d = np.abs(np.diag(dA.cpu().numpy()))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))


def test_qrcp_refuses_capture(lib):
    """The call reads each block's length back on the host: refused while the
    stream is being captured, before anything is enqueued."""
    import paper_1509_06820_gb300 as rq
    A = to_dev(synth.gaussian(64, 64, seed=1))
    h = rq.Handle(A.device)
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g):
        try:
            rq.qrcp_factor(A, 16, handle=h)
        except rq.RqrcpError as e:
            err = e
    assert err is not None and "(1002)" in str(err)
