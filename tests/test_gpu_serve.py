"""Serving loop on the GPU: each request's result is the same alone and in
a concurrent mix (same bucket graph, deterministic kernels), the factors are
a valid rank-k factorization of the request's matrix, and a short Poisson
run reports latency percentiles."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SIZES = [(600, 900, 40), (1100, 700, 70), (300, 300, 16), (900, 1200, 100), (512, 512, 32),
         (777, 1500, 64)]


def _run(srv, reqs, together):
    from paper_1509_06820_gb300.serve import factors
    out = {}
    if together:
        for r in reqs:
            srv.submit(r)
        srv.drain()
    else:
        for r in reqs:
            srv.submit(r)
            srv.drain()
    torch.cuda.synchronize()
    for r in reqs:
        jp, tau, Y, R, rd = factors(r)
        out[r.rid] = (jp.cpu().numpy(), R.cpu().numpy().astype(np.float64), Y.cpu().numpy(),
                      tau.cpu().numpy(), rd.cpu().numpy())
    return out


def test_same_alone_and_in_mix(lib):
    from paper_1509_06820_gb300.serve import Request, Server
    srv = Server.on_gpu(slots=4)
    alone = _run(srv, [Request(i, *s) for i, s in enumerate(SIZES)], together=False)
    mixed = _run(srv, [Request(i, *s) for i, s in enumerate(SIZES)], together=True)
    assert srv.max_in_flight > 1
    for i, (m, n, k) in enumerate(SIZES):
        ja, Ra = alone[i][0], alone[i][1]
        jm, Rm = mixed[i][0], mixed[i][1]
        np.testing.assert_array_equal(ja[:k], jm[:k])
        assert np.abs(Ra - Rm).max() <= 1e-6 * np.abs(Ra).max()


def test_served_factors_reconstruct(lib):
    """The served rank-k factors reproduce A = X Y^T (rank k) to FP32 level."""
    from oracle import householder as hh
    from paper_1509_06820_gb300.serve import Request, Server, make_input
    from paper_1509_06820_gb300 import empty_colmajor
    srv = Server.on_gpu(slots=2)
    reqs = [Request(100 + i, *s) for i, s in enumerate(SIZES[:3])]
    res = _run(srv, reqs, together=True)
    for r in reqs:
        A = empty_colmajor(r.m, r.n, "cuda", torch.float32)
        make_input(r, A, torch.cuda.current_stream())
        torch.cuda.synchronize()
        A64 = A.cpu().numpy().astype(np.float64)
        jp, R, Y, tau, rd = res[r.rid]
        k = r.k
        R = R[:k, :].copy()
        R[np.arange(k), np.arange(k)] = rd[:k]
        Q = hh.form_q(Y.astype(np.float64), tau[:k], k)
        approx = np.zeros_like(A64)
        approx[:, jp] = Q @ R
        assert np.linalg.norm(A64 - approx) <= 1e-5 * np.linalg.norm(A64)


def test_poisson_run_reports_latency(lib):
    from paper_1509_06820_gb300.serve import Server
    srv = Server.on_gpu(slots=4)
    stats = srv.run_poisson(rate=300, duration=1.0, warmup=0.2, seed=3,
                            size_range=(256, 1024), k_range=(16, 64))
    assert stats["requests"] > 50
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert stats["throughput_rps"] > 0
