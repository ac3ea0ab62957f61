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


def _check_rqrcp(lib, A, b, p, seed, expect_info=0, handle=None, resample=False):
    m, n = A.shape
    dA = to_dev(A)
    jpvt, tau = lib.rqrcp_factor(dA, b, p, seed, handle=handle)
    info = handle.sync_info() if handle is not None else lib.sync_info()
    assert info == expect_info
    F, jp, t = host(dA), host(jpvt), host(tau)
    assert sorted(jp.tolist()) == list(range(n))
    ties = []
    run = oracle.rsrqrcp if resample else oracle.rqrcp
    Fo, jo, to, info_o = run(A, b, p, seed=seed, replay_jpvt=jp, ties=ties)
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


@pytest.mark.parametrize("m,n,b,p,emul", [(1000, 1000, 32, 8, False), (300, 500, 64, 8, False),
                                          (500, 300, 16, 4, False), (600, 600, 64, 8, True)])
def test_rsrqrcp_matches_oracle(lib, m, n, b, p, emul):
    """Alg. 5 (RQRCP_OPT_RESAMPLE): a fresh sample of the trailing matrix every
    block; pivots, R and the reconstruction against the oracle's Alg. 5 at the
    FP64 tolerances (also with the FP64-emulated products)."""
    h = lib.Handle()
    h.set_resample(True)
    if emul:
        h.set_fp64_emulation(True)
    A = synth.gaussian(m, n, seed=m + n + b)
    _, ties = _check_rqrcp(lib, A, b, p, 3, handle=h, resample=True)
    assert len(ties) <= 2


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


@pytest.mark.parametrize("m,n,k,b,jmax", [(400, 300, 24, 8, 2), (300, 400, 40, 16, 3),
                                           (520, 260, 64, 32, 4), (257, 257, 17, 8, 5)])
def test_tuxv_iter_matches_oracle(lib, m, n, k, b, jmax):
    """Alg. 7 with j_max > 1: the same U X V^T as the oracle's iterations, X
    lower triangular after an even number of iterations, upper after odd."""
    A = synth.decaying_lowrank(m, n, rank=min(m, n) // 2, noise=1e-8)
    U, X, V = lib.tuxv(to_dev(A), k, b, 8, 5, jmax=jmax)
    assert lib.sync_info() == 0
    Ug, Xg, Vg = host(U), host(X), host(V)
    Uo, Xo, Vo, jo, info = oracle.tuxv(A, k, b, 8, seed=5, jmax=jmax)
    if jmax % 2:
        assert np.allclose(np.tril(Xg, -1), 0.0)
    else:
        assert np.allclose(np.triu(Xg, 1), 0.0)
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Vg.T @ Vg, np.eye(k), atol=1e-13)
    approx_g = Ug @ Xg @ Vg.T
    approx_o = Uo @ Xo @ Vo.T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-10 * np.linalg.norm(approx_o)
    np.testing.assert_allclose(np.abs(np.diag(Xg)), np.abs(np.diag(Xo)), rtol=1e-9)


@pytest.mark.parametrize("m,n,k,b,jmax", [(300, 200, 1, 1, 1), (300, 200, 7, 4, 1),
                                           (400, 300, 33, 16, 2), (600, 500, 160, 32, 3)])
def test_tuxv_svd_matches_oracle(lib, m, n, k, b, jmax):
    """Alg. 7 plus the SVD of X (one-sided Jacobi on the device, one CTA for
    k <= 16, cooperative above): singular values and the approximation as
    the oracle's (LAPACK SVD of its X), singular vectors up to sign where the
    singular values are separated."""
    A = synth.decaying_lowrank(m, n, rank=min(m, n) // 2, noise=1e-8)
    U, sig, V = lib.tuxv_svd(to_dev(A), k, b, 8, 5, jmax=jmax)
    assert lib.sync_info() == 0
    Ug, sg, Vg = host(U), sig.cpu().numpy(), host(V)
    Uo, so, Vo, _, _ = oracle.tuxv_svd(A, k, b, 8, seed=5, jmax=jmax)
    assert np.all(np.diff(sg) <= 0)
    assert np.abs(sg - so).max() <= 1e-10 * so[0]
    np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(Vg.T @ Vg, np.eye(k), atol=1e-12)
    approx_g = (Ug * sg) @ Vg.T
    approx_o = (Uo * so) @ Vo.T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-10 * np.linalg.norm(approx_o)
    gap = np.minimum(np.r_[np.inf, so[:-1] - so[1:]], np.r_[so[:-1] - so[1:], np.inf])
    sep = gap > 1e-4 * so[0]
    cu = np.abs(np.sum(Ug * Uo, axis=0))
    cv = np.abs(np.sum(Vg * Vo, axis=0))
    assert np.all(cu[sep] >= 1 - 1e-8) and np.all(cv[sep] >= 1 - 1e-8)


def test_tuxv_svd_zero_matrix(lib):
    """X = 0: every singular value 0 and, as documented, U's columns 0."""
    A = torch.zeros((64, 48), dtype=torch.float64)
    U, sig, V = lib.tuxv_svd(lib.colmajor(A.cuda()), 5, 4, 4, 1)
    # R11 = 0 makes the sample update re-draw the trailing sample
    assert lib.sync_info() & ~lib.INFO_RESAMPLED == 0
    assert np.all(sig.cpu().numpy() == 0.0)
    assert np.all(host(U) == 0.0)
    np.testing.assert_allclose(host(V).T @ host(V), np.eye(5), atol=1e-15)


def test_tuxv_iter_rejects_zero_iterations(lib):
    A = to_dev(synth.gaussian(40, 30, seed=1))
    with pytest.raises(lib.RqrcpError, match="argument 10"):
        lib.tuxv(A, 4, 4, 4, 1, jmax=0)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 200, 150), (64, 700, 1000), (129, 1, 7)])
def test_tc_gemm_bf16x3(lib, ta, tb, m, n, k):
    """Split-BF16 x3 tensor-core GEMM against an FP64 product: FP32-level error
    independent of K (exact three-slice split, the leading product drained
    every 32 k into compensated register sums)."""
    g = torch.Generator().manual_seed(m + n + k)
    Af = torch.randn((m, k) if ta == "N" else (k, m), generator=g, dtype=torch.float64)
    Bf = torch.randn((k, n) if tb == "N" else (n, k), generator=g, dtype=torch.float64)
    A32, B32 = Af.float(), Bf.float()
    A = lib.colmajor(A32.cuda())
    B = lib.colmajor(B32.cuda())
    C0 = lib.colmajor(torch.randn((m, n), generator=g, dtype=torch.float32).cuda())
    C = C0.clone()
    lib.gemm_bf16x(A, B, ta, tb, alpha=-1.0, beta=1.0, C=C, slices=3)
    assert lib.sync_info() == 0
    opA = A32.double() if ta == "N" else A32.double().t()
    opB = B32.double() if tb == "N" else B32.double().t()
    ref = C0.cpu().double() - opA @ opB
    err = (C.cpu().double() - ref).abs().max().item()
    scale = (opA.abs() @ opB.abs()).max().item() + C0.abs().max().item()
    # a few u of sum_k |a||b|: two truncating MMA additions per 32-k chunk,
    # the dropped slice products (below 2^-25 each), the compensated sum and
    # the final FP32 rounding
    assert err <= 8 * 2.0 ** -24 * scale, err / scale


@pytest.mark.parametrize("m,n,k", [(256, 256, 128), (100, 300, 70)])
def test_tc_gemm_bf16x1(lib, m, n, k):
    """One-slice mode: the product of the bf16-rounded operands, FP32 accumulation."""
    g = torch.Generator().manual_seed(7)
    A32 = torch.randn((m, k), generator=g)
    B32 = torch.randn((k, n), generator=g)
    C = lib.gemm_bf16x(lib.colmajor(A32.cuda()), lib.colmajor(B32.cuda()), slices=1)
    assert lib.sync_info() == 0
    ref = A32.bfloat16().double() @ B32.bfloat16().double()
    err = (C.cpu().double() - ref).abs().max().item()
    assert err <= 2.0 ** -22 * (A32.abs().double() @ B32.abs().double()).max().item()


def _mixed_errors(A, A32, jp, t, rdiag):
    """Reconstruction and orthogonality of the mixed-precision factors in FP64."""
    m, n = A.shape
    k = min(m, n)
    F = A32.astype(np.float64)
    Q = hh.form_q(F, t, m)
    R = np.triu(F)
    R[np.arange(k), np.arange(k)] = rdiag
    rec = np.linalg.norm(A[:, jp] - Q @ R) / np.linalg.norm(A)
    orth = np.abs(Q.T @ Q - np.eye(m)).max()
    return rec, orth, R


@pytest.mark.parametrize("m,n,b,p", [(1000, 1000, 128, 16), (700, 400, 64, 8), (300, 900, 128, 16)])
def test_rqrcp_mixed_reconstruction(lib, m, n, b, p):
    """Mixed precision (FP32 storage, BF16 sketch, split-BF16 x3 trailing
    update, FP64 panel/T/R-diagonal) is FP32-level: its reconstruction error
    is within 2x of LAPACK's own FP32 pivoted QR (sgeqp3) on the same matrix,
    Q is orthogonal to FP64 level (tau and T are recomputed from the stored
    FP32 reflectors), and R is stated against the FP64 oracle replayed on the
    same pivots."""
    import scipy.linalg as sla
    A = synth.spiked(m, n, rank=min(m, n) // 4, scale=1e3)
    A32 = A.astype(np.float32)
    dA = lib.colmajor(torch.from_numpy(A32).cuda())
    jpvt, tau, rdiag = lib.rqrcp_factor_mixed(dA, b, p, 1)
    assert lib.sync_info() == 0
    jp = host(jpvt)
    assert sorted(jp.tolist()) == list(range(n))
    A64 = A32.astype(np.float64)
    rec, orth, R = _mixed_errors(A64, host(dA), jp, host(tau), host(rdiag))
    Q32, R32, P32 = sla.qr(A32, pivoting=True)
    rec32 = np.linalg.norm(A64[:, P32] - Q32.astype(np.float64) @ R32.astype(np.float64)) / np.linalg.norm(A64)
    Fo, jo, to, _ = oracle.rqrcp(A64, b, p, seed=1, replay_jpvt=jp, tie_rtol=1.0)
    k = min(m, n)
    rel = np.linalg.norm(R[:k] - np.triu(Fo[:k])) / np.linalg.norm(np.triu(Fo[:k]))
    print(f"mixed {m}x{n}: recon {rec:.2e} (sgeqp3 {rec32:.2e}) orth {orth:.2e} "
          f"R vs FP64 oracle {rel:.2e}")
    assert rec <= 2 * rec32, (rec, rec32)
    assert orth <= 1e-5, orth
    assert rel <= 1e-5


def _swaps_to_ids(swaps, nc):
    perm = np.arange(nc)
    for i, s in enumerate(swaps):
        perm[[i, s]] = perm[[s, i]]
    return perm


@pytest.mark.parametrize("ell,nc,steps,ldpad", [(72, 5000, 64, 0), (40, 333, 32, 5), (9, 20, 9, 0),
                                                (144, 3000, 128, 3)])
def test_sample_qrcp_matches_oracle(lib, ell, nc, steps, ldpad):
    """Alg. 1 halted after `steps` pivots on an l x n sample (row a3 alone)."""
    from oracle.rqrcp import sample_qrcp
    r = np.random.default_rng(ell + nc)
    B = r.standard_normal((ell, nc)) * np.exp(r.standard_normal(nc))[None, :]
    store = torch.zeros((nc, ell + ldpad), dtype=torch.float64)
    store[:, :ell] = torch.from_numpy(B.T)
    dB_full = store.cuda().t()               # (ell + ldpad) x nc column-major
    dB = dB_full[:ell]
    swaps = host(lib.sample_qrcp(dB, steps))
    assert lib.sync_info() == 0
    ids = _swaps_to_ids(swaps, nc)
    S = B.copy()
    sample_qrcp(S, steps, ids=np.arange(nc), forced_ids=ids[:steps])
    Sg = host(dB)
    assert np.abs(Sg - S).max() <= 1e-12 * np.abs(B).max()
    assert np.all(np.tril(Sg[:, :steps], -1) == 0.0)


@pytest.mark.parametrize("m,n,k,b,p", [(512, 384, 64, 64, 8), (1000, 700, 100, 32, 8),
                                       (300, 900, 48, 128, 16)])
def test_trqrcp_mixed_lowrank(lib, m, n, k, b, p):
    """Mixed-precision TRQRCP on a rank-k Gaussian-factor matrix (the served
    workload): the rank-k factorization reproduces A to FP32 level, and its R
    agrees with the FP64 oracle replayed on the same pivots."""
    A = synth.factor_product(m, n, k, seed=m + n + k).astype(np.float32)
    dA = lib.colmajor(torch.from_numpy(A).cuda())
    jpvt, tau, Y, R, rdiag = lib.trqrcp_mixed(dA, k, b, p, 7)
    assert lib.sync_info() == 0
    jp, t, Yg, Rg, rd = host(jpvt), host(tau), host(Y).astype(np.float64), host(R).astype(np.float64), host(rdiag)
    assert sorted(jp.tolist()) == list(range(n))
    Rg[np.arange(k), np.arange(k)] = rd
    Q = hh.form_q(Yg, t, k)
    A64 = A.astype(np.float64)
    approx = np.zeros_like(A64)
    approx[:, jp] = Q @ Rg
    rec = np.linalg.norm(A64 - approx) / np.linalg.norm(A64)
    assert rec <= 1e-5, rec
    jo, to, Yo, Ro, _ = oracle.trqrcp(A64, k, b, p, seed=7, replay_jpvt=jp, tie_rtol=1.0)
    rel = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    print(f"trqrcp_mixed {m}x{n} k={k}: rank-k recon {rec:.2e}, R vs FP64 oracle {rel:.2e}")
    assert rel <= 1e-4


def test_tc_gemm_accumulation_profile(lib):
    """Error of the split-BF16 x3 tensor-core GEMM against K (per entry, in
    units of u = 2^-24 of sum_k |a||b|) next to cuBLAS FP32 SGEMM; prints the
    table and pins the bound: within 8 u at every K, with a mean signed error
    below 1 u (the tensor core truncates inside each 32-k chunk, which on
    all-positive data leaves a bias of under 1 u that does not grow with K)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    g = torch.Generator().manual_seed(0)
    u = 2.0 ** -24
    try:
        for K in [64, 256, 1024, 4096, 16384]:
            for kind in ["gauss", "pos"]:
                A = torch.randn(128, K, generator=g, dtype=torch.float64)
                B = torch.randn(K, 256, generator=g, dtype=torch.float64)
                if kind == "pos":
                    A, B = A.abs(), B.abs()
                A32, B32 = A.float(), B.float()
                ref = A32.double() @ B32.double()
                scale = A32.double().abs() @ B32.double().abs()
                C3 = lib.gemm_bf16x(lib.colmajor(A32.cuda()), lib.colmajor(B32.cuda()),
                                    slices=3).cpu().double()
                Cf = (A32.cuda() @ B32.cuda()).cpu().double()
                e3 = (C3 - ref) / scale
                ef = (Cf - ref) / scale
                print(f"K={K:6d} {kind:5s} bf16x3 max {e3.abs().max().item() / u:8.2f}u "
                      f"mean {e3.abs().mean().item() / u:7.2f}u signed {e3.mean().item() / u:8.2f}u"
                      f" | sgemm max {ef.abs().max().item() / u:6.2f}u "
                      f"mean {ef.abs().mean().item() / u:5.2f}u")
                assert e3.abs().max().item() <= 8 * u
                assert abs(e3.mean().item()) <= 1.0 * u
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (300, 200, 150), (200, 70, 1000), (1, 1, 1)])
def test_gemm_f64x_accuracy(lib, ta, tb, m, n, k):
    """FP64 GEMM emulated on the BF16 tensor cores: the slice products are
    exact and the running sums are double-FP32 (about 48 significant bits;
    each 32-k drain rounds a handful of times), so the error is within
    16 * 2^-48 of sum_k |a||b| (+ |C|), on data spanning 12 decades per row."""
    r = np.random.default_rng(m + 3 * n + 7 * k)
    A = r.standard_normal((m, k) if ta == "N" else (k, m)) * 10.0 ** r.uniform(-6, 6, ((m, k) if ta == "N" else (k, m)))
    B = r.standard_normal((k, n) if tb == "N" else (n, k))
    C0 = r.standard_normal((m, n))
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    C = to_dev(C0)
    lib.gemm_f64x(to_dev(A), to_dev(B), ta, tb, alpha=-1.0, beta=1.0, C=C)
    assert lib.sync_info() == 0
    ref = C0 - opA @ opB
    scale = np.abs(opA) @ np.abs(opB) + np.abs(C0)
    err = (np.abs(host(C) - ref) / scale).max()
    assert err <= 16 * 2.0 ** -48, err


@pytest.mark.parametrize("m,n,b,p", [(300, 200, 32, 8), (1000, 1000, 32, 8), (520, 700, 64, 8)])
def test_rqrcp_fp64_emulated_trailing(lib, m, n, b, p):
    """RQRCP with the trailing update on the BF16 tensor cores (FP64-accurate
    slicing) meets the same FP64 parity bar against the oracle."""
    h = lib.Handle()
    h.set_fp64_emulation(True)
    try:
        A = synth.gaussian(m, n, seed=m + n)
        dA = to_dev(A)
        jpvt, tau = lib.rqrcp_factor(dA, b, p, 1, handle=h)
        assert h.sync_info() == 0
        F, jp, t = host(dA), host(jpvt), host(tau)
        Fo, jo, to, _ = oracle.rqrcp(A, b, p, seed=1, replay_jpvt=jp)
        k = min(m, n)
        Ro = np.triu(Fo[:k])
        assert np.linalg.norm(np.triu(F[:k]) - Ro) <= RTOL_R * np.linalg.norm(Ro)
        Q = hh.form_q(F, t, m)
        assert np.linalg.norm(A[:, jp] - Q @ np.triu(F)) <= RTOL_REC * np.linalg.norm(A)
    finally:
        h.close()


@pytest.mark.parametrize("m,n,b,p,inplace,pinned", [(700, 500, 32, 8, False, True),
                                                    (300, 900, 64, 8, True, True),
                                                    (1000, 1000, 32, 8, False, False),
                                                    (129, 17, 16, 4, True, False)])
def test_rqrcp_factor_host_equals_device_call(lib, m, n, b, p, inplace, pinned):
    """Host buffers, copies overlapped on the handle's copy stream: bit for bit
    the device call's factor, pivots and tau (same kernels on the same data)."""
    A = synth.gaussian(m, n, seed=m + 3 * n)
    dref = to_dev(A)
    jref, tref = lib.rqrcp_factor(dref, b, p, 7)
    hA = torch.from_numpy(np.asfortranarray(A))
    assert hA.stride() == (1, m)
    if pinned:
        hA = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t().copy_(hA)
    out = None
    if inplace:
        out = (hA, torch.empty(n, dtype=torch.int64), torch.empty(min(m, n), dtype=torch.float64))
    F, jp, tau, dA = lib.rqrcp_factor_host(hA, b, p, 7, out=out)
    torch.cuda.synchronize()
    assert lib.sync_info() == 0
    assert torch.equal(jp, jref.cpu())
    assert torch.equal(tau, tref.cpu())
    assert torch.equal(F, dref.cpu())
    assert torch.equal(dA.cpu(), dref.cpu())


def test_max_sms_cap_keeps_parity(lib):
    """RQRCP_OPT_MAX_SMS: a handle whose launches use at most 20 SMs (smaller
    cooperative grids, no split-K beyond 20 CTAs) still matches the oracle."""
    h = lib.Handle()
    h.set_max_sms(20)
    A = synth.gaussian(700, 600, seed=12)
    _check_rqrcp(lib, A, 32, 8, 1, handle=h)
    with pytest.raises(lib.RqrcpError):
        h.set_max_sms(-1)
    h.set_max_sms(0)   # back to all SMs
    _check_rqrcp(lib, A, 32, 8, 1, handle=h)


@pytest.mark.parametrize("mixed", [False, True])
def test_factor_bitwise_reproducible(lib, mixed):
    """Two runs of one factorization are bit for bit equal: every grid reduction
    has a fixed order, including the panel's two-level sum of the column dots
    (4096 rows on 128 CTAs in 16 groups of 8, b = 128, so the grouped form runs
    for the first 73 columns of every panel), whose group sums are added in CTA
    order by whichever CTA of the group publishes last."""
    m, n, b, p = 4096, 768, 128, 16
    A = synth.gaussian(m, n, seed=11)
    runs = []
    for _ in range(2):
        if mixed:
            dA = lib.colmajor(torch.from_numpy(A).float().cuda())
            jp, tau, rd = lib.rqrcp_factor_mixed(dA, b, p, 3)
            runs.append((dA, jp, tau, rd))
        else:
            dA = to_dev(A)
            jp, tau = lib.rqrcp_factor(dA, b, p, 3)
            runs.append((dA, jp, tau))
    assert lib.sync_info() == 0
    for x, y in zip(*runs):
        assert torch.equal(x, y)
