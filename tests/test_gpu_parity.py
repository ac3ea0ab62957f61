"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (FP64 path): pivots bit-exact wherever the oracle's sample norms
separate the GPU's choice from its own by more than 1e-8 relative (replay
mode follows the GPU through closer ties); ||R_gpu - R_oracle||_F/||R||_F <=
1e-10; ||A P - Q R||_F / ||A||_F <= 1e-13; the Gaussian matrix within
4 ulp-scale (1e-14 absolute on |x| < 10) of the oracle's libm values.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import householder as hh
import synth

pytestmark = pytest.mark.gpu

RTOL_R = 1e-10
RTOL_REC = 1e-13


def to_dev(A):
    import paper_1509_06820_gb300 as rq
    return rq.colmajor(torch.from_numpy(np.asarray(A, dtype=np.float64)).cuda())


def host(x):
    return x.cpu().numpy()


def test_gaussian_matches_oracle(lib):
    for seed, rows, cols, stream in [(1, 72, 1000, 1), (123456789012, 9, 33, 1), (7, 40, 5, 0x101)]:
        g = host(lib.gaussian(seed, stream, rows, cols))
        o = oracle.philox.gaussian_block(seed, rows, cols, stream)
        assert np.abs(g - o).max() <= 1e-14 * max(1.0, np.abs(o).max())


def test_sketch_matches_oracle(lib):
    A = synth.gaussian(300, 77, seed=3)
    B = host(lib.sketch(to_dev(A), 40, 5))
    Bo = oracle.gaussian_omega(5, 40, 300) @ A
    assert np.linalg.norm(B - Bo) <= 1e-14 * np.linalg.norm(Bo) * 10


@pytest.mark.parametrize("m,n,b", [(300, 200, 32), (200, 300, 32), (129, 129, 16), (64, 64, 64),
                                   (1000, 1000, 32), (70, 10, 4), (10, 70, 8), (1, 1, 1), (1, 7, 3),
                                   (7, 1, 3), (5000, 300, 64)])
def test_qr_matches_oracle(lib, m, n, b):
    A = synth.gaussian(m, n, seed=m + 7 * n)
    dA = to_dev(A)
    tau = lib.qr_factor(dA, b)
    assert lib.sync_info() == 0
    F, t = host(dA), host(tau)
    Fo, to = oracle.qr_blocked(A, b)
    scale = np.linalg.norm(A)
    assert np.linalg.norm(np.triu(F) - np.triu(Fo)) <= RTOL_R * np.linalg.norm(np.triu(Fo))
    assert np.abs(np.tril(F, -1) - np.tril(Fo, -1)).max() <= 1e-11
    assert np.abs(t - to).max() <= 1e-12
    Q = hh.form_q(F, t, m)
    assert np.linalg.norm(A - Q @ np.triu(F)) <= RTOL_REC * scale


def _check_rqrcp(lib, A, b, p, seed, expect_info=0):
    m, n = A.shape
    dA = to_dev(A)
    jpvt, tau = lib.rqrcp_factor(dA, b, p, seed)
    info = lib.sync_info()
    assert info == expect_info
    F, jp, t = host(dA), host(jpvt), host(tau)
    assert sorted(jp.tolist()) == list(range(n))
    ties = []
    Fo, jo, to, info_o = oracle.rqrcp(A, b, p, seed=seed, replay_jpvt=jp, ties=ties)
    assert info_o == expect_info
    np.testing.assert_array_equal(jo, jp)
    k = min(m, n)
    Ro = np.triu(Fo[:k])
    assert np.linalg.norm(np.triu(F[:k]) - Ro) <= RTOL_R * np.linalg.norm(Ro)
    # reflectors are determined only where the column is above the rounding
    # floor: compare tau where |R_ii| >= 1e-6 |R_00|
    sig = np.abs(np.diag(Ro)) >= 1e-6 * abs(Ro[0, 0])
    assert np.abs(t - to)[sig].max() <= 1e-9
    Q = hh.form_q(F, t, m)
    assert np.linalg.norm(A[:, jp] - Q @ np.triu(F)) <= RTOL_REC * np.linalg.norm(A)
    return jp, ties


def test_rqrcp_1000_square_b32_p8(lib):
    """1000 x 1000 N(0,1) (seed 0), b = 32, p = 8, Omega seed 1: 32 blocks, last one ragged."""
    A = synth.gaussian(1000, 1000, seed=0)
    jp, ties = _check_rqrcp(lib, A, 32, 8, 1)
    assert len(ties) <= 2


@pytest.mark.parametrize("m,n,b,p", [(50, 30, 8, 4), (30, 50, 8, 4), (200, 200, 64, 8),
                                     (120, 7, 16, 4), (7, 120, 16, 4), (1, 1, 1, 0), (1, 9, 4, 2),
                                     (9, 1, 4, 2), (513, 257, 32, 0), (300, 300, 128, 16),
                                     (2000, 600, 64, 8)])
def test_rqrcp_shapes(lib, m, n, b, p):
    A = synth.gaussian(m, n, seed=m * 31 + n)
    _check_rqrcp(lib, A, b, p, 11)


def test_rqrcp_graded_spectrum(lib):
    """U diag(sigma) V^T with sigma down to 1e-12 (graded), smaller order."""
    A = synth.graded(400, decades=12.0)
    _check_rqrcp(lib, A, 32, 8, 1)


def test_rqrcp_separated_columns_exact_order(lib):
    A, order = synth.separated_columns(200, 64, phi=0.5, seed=9)
    import paper_1509_06820_gb300 as rq
    dA = to_dev(A)
    jpvt, tau = lib.rqrcp_factor(dA, 8, 8, 3)
    np.testing.assert_array_equal(host(jpvt), order)


def test_rqrcp_resample_path(lib):
    A = synth.gaussian(60, 40, seed=4)
    A[:, 12:] = 0.0
    _check_rqrcp(lib, A, 8, 4, 2, expect_info=2)


def test_rqrcp_nonfinite_flagged(lib):
    A = synth.gaussian(40, 40, seed=1)
    A[3, 5] = np.nan
    dA = to_dev(A)
    lib.rqrcp_factor(dA, 8, 4, 1)
    assert lib.sync_info() & 1


def test_rqrcp_deterministic(lib):
    A = synth.gaussian(700, 500, seed=5)
    outs = []
    for _ in range(2):
        dA = to_dev(A)
        jpvt, tau = lib.rqrcp_factor(dA, 32, 8, 1)
        outs.append((host(dA), host(jpvt), host(tau)))
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


def test_argument_errors(lib):
    import paper_1509_06820_gb300 as rq
    A = to_dev(synth.gaussian(10, 10, seed=1))
    with pytest.raises(rq.RqrcpError, match="argument 6"):
        lib.rqrcp_factor(A, 0, 4, 1)
    with pytest.raises(rq.RqrcpError, match="argument 7"):
        lib.rqrcp_factor(A, 4, -1, 1)
    with pytest.raises(rq.RqrcpError, match="argument 6"):
        lib.trqrcp(A, 11, 4, 2, 1)
    with pytest.raises(rq.RqrcpError, match="outside the supported"):
        lib.rqrcp_factor(A, 4, 400, 1)


@pytest.mark.parametrize("m,n,k,b,p", [(300, 200, 64, 16, 8), (200, 300, 50, 16, 8),
                                       (1000, 800, 100, 32, 8), (90, 90, 90, 32, 4)])
def test_trqrcp_matches_oracle(lib, m, n, k, b, p):
    A = synth.decaying_lowrank(m, n, rank=min(m, n) // 2, noise=1e-6)
    jpvt, tau, Y, R = lib.trqrcp(to_dev(A), k, b, p, 3)
    assert lib.sync_info() == 0
    jp, t, Yg, Rg = host(jpvt), host(tau), host(Y), host(R)
    jo, to, Yo, Ro, info = oracle.trqrcp(A, k, b, p, seed=3, replay_jpvt=jp)
    np.testing.assert_array_equal(jo[:k], jp[:k])
    assert sorted(jp.tolist()) == list(range(n))
    assert np.linalg.norm(Rg - Ro) <= RTOL_R * np.linalg.norm(Ro)
    assert np.abs(Yg - Yo).max() <= 1e-10
    assert np.abs(t - to).max() <= 1e-10
    # A P ~= Q_k R with R's first k columns exact
    Q = hh.form_q(Yg, t, k)
    assert np.linalg.norm(Q @ Rg[:, :k] - A[:, jp[:k]]) <= RTOL_REC * np.linalg.norm(A) * 10


@pytest.mark.parametrize("m,n,k,b,p", [(300, 200, 40, 16, 8), (500, 700, 64, 32, 8)])
def test_tuxv_matches_oracle(lib, m, n, k, b, p):
    A = synth.decaying_lowrank(m, n, rank=min(m, n) // 2, noise=1e-8)
    U, X, V = lib.tuxv(to_dev(A), k, b, p, 5)
    assert lib.sync_info() == 0
    Ug, Xg, Vg = host(U), host(X), host(V)
    Uo, Xo, Vo, jo, info = oracle.tuxv(A, k, b, p, seed=5)
    assert np.allclose(np.tril(Xg, -1), 0.0)
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Vg.T @ Vg, np.eye(k), atol=1e-13)
    approx_g = Ug @ Xg @ Vg.T
    approx_o = Uo @ Xo @ Vo.T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-10 * np.linalg.norm(approx_o)
    np.testing.assert_allclose(np.abs(np.diag(Xg)), np.abs(np.diag(Xo)), rtol=1e-9)
