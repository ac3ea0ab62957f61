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


# uneven problems for the batched entry point: (m, n, k, b, p)
BATCH = [(600, 900, 40, 32, 8), (1100, 700, 70, 64, 8), (300, 300, 16, 64, 8),
         (900, 1200, 100, 128, 16), (512, 512, 32, 32, 8), (777, 1500, 64, 64, 16),
         (150, 400, 20, 32, 8), (1200, 1000, 96, 64, 8), (420, 260, 50, 32, 16),
         (1300, 1300, 128, 128, 16)]


def _batch_inputs(seed0=0):
    from paper_1509_06820_gb300 import colmajor
    g = torch.Generator(device="cuda")
    As = []
    for i, (m, n, k, b, p) in enumerate(BATCH):
        g.manual_seed(seed0 + i)
        X = torch.randn((m, k), generator=g, device="cuda")
        Yf = torch.randn((n, k), generator=g, device="cuda")
        As.append(colmajor(X @ Yf.t()))
    return As


def test_trqrcp_batched_same_alone_and_in_batch(lib):
    """The persistent batched launch over uneven problems gives, bit for bit,
    what the same launch gives on each problem alone: a problem's result
    depends only on the problem and the team size."""
    As = _batch_inputs()
    probs = [(A, k, b, p, 11 + i) for i, (A, (m, n, k, b, p)) in enumerate(zip(As, BATCH))]
    got = lib.trqrcp_batched(probs)
    assert lib.sync_info() == 0
    for prob, out in zip(probs, got):
        alone = lib.trqrcp_batched([prob], teams=1)[0]
        assert lib.sync_info() == 0
        for x, y in zip(out, alone):
            assert torch.equal(x, y)


def test_trqrcp_batched_accuracy(lib):
    """Each problem of a batch: the rank-k factors reproduce A = X Y^T to FP32
    level, R agrees with the FP64 oracle's Alg. 6 replayed on the same pivots,
    and the selected columns span what trqrcp_mixed's span."""
    import oracle
    from oracle import householder as hh
    import synth
    probs, hosts = [], []
    for i, (m, n, k, b, p) in enumerate(BATCH):
        A = synth.factor_product(m, n, k, seed=300 + i).astype(np.float32)
        hosts.append(A)
        probs.append((lib.colmajor(torch.from_numpy(A).cuda()), k, b, p, 21 + i))
    got = lib.trqrcp_batched(probs, teams=3)
    assert lib.sync_info() == 0
    for (dA, k, b, p, seed), A, out in zip(probs, hosts, got):
        jp, t, Yg, Rg, rd = (x.cpu().numpy() for x in out)
        Yg, Rg = Yg.astype(np.float64), Rg.astype(np.float64)
        assert sorted(jp.tolist()) == list(range(A.shape[1]))
        Rg[np.arange(k), np.arange(k)] = rd
        Q = hh.form_q(Yg, t, k)
        A64 = A.astype(np.float64)
        approx = np.zeros_like(A64)
        approx[:, jp] = Q @ Rg
        rec = np.linalg.norm(A64 - approx) / np.linalg.norm(A64)
        assert rec <= 1e-5, rec
        _, _, _, Ro, _ = oracle.trqrcp(A64, k, b, p, seed=seed, replay_jpvt=jp, tie_rtol=1.0)
        rel = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
        assert rel <= 1e-4, rel


def test_trqrcp_batched_graph_replay(lib):
    """A whole batch captured as one CUDA graph (one persistent launch)
    replays on new data with the results of an eager launch on that data."""
    h = lib.Handle()
    h.reserve_batched(0, 1300, 1500, 128, 128, 16)
    As = _batch_inputs(100)
    bufs = [A.clone() for A in As]
    probs = [(A, k, b, p, 5) for A, (m, n, k, b, p) in zip(bufs, BATCH)]
    outs = lib.trqrcp_batched(probs, handle=h)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        lib.trqrcp_batched(probs, handle=h, outs=outs)
    new = _batch_inputs(200)
    for buf, A in zip(bufs, new):
        buf.copy_(A)
    graph.replay()
    torch.cuda.synchronize()
    assert h.sync_info() == 0
    ref = lib.trqrcp_batched([(A, k, b, p, 5) for A, (m, n, k, b, p) in zip(new, BATCH)])
    assert lib.sync_info() == 0
    for out, r in zip(outs, ref):
        for x, y in zip(out, r):
            assert torch.equal(x, y)


def test_trqrcp_batched_rejects_before_launch(lib):
    """One invalid problem (k > min(m, n)) fails the whole call with
    RQRCP_ERR_BATCH before anything is enqueued."""
    As = _batch_inputs()[:3]
    ks = [16, 10**6, 16]
    outs = [(torch.full((A.shape[1],), -7, dtype=torch.int64, device="cuda"),
             torch.zeros(16, dtype=torch.float64, device="cuda"),
             lib.empty_colmajor(A.shape[0], 16, "cuda", torch.float32),
             lib.empty_colmajor(16, A.shape[1], "cuda", torch.float32),
             torch.zeros(16, dtype=torch.float64, device="cuda")) for A in As]
    probs = [(A, k, 16, 8, 1) for A, k in zip(As, ks)]
    with pytest.raises(lib.RqrcpError, match="problem 1"):
        lib.trqrcp_batched(probs, teams=2, outs=outs)
    torch.cuda.synchronize()
    assert all(bool((o[0] == -7).all()) for o in outs)


# ---------------------------------------------------------------- ring server
def _ring_run(srv, reqs, together):
    if together:
        for r in reqs:
            srv.submit(r)
        srv.drain()
    else:
        for r in reqs:
            srv.submit(r)
            srv.drain()
    torch.cuda.synchronize()
    return {r.rid: tuple(x.cpu().numpy() for x in r.result) for r in reqs}


def test_ring_server_same_alone_and_in_mix(lib):
    """Requests served through the mapped request ring of one persistent launch:
    each result is bit for bit the same alone and in a concurrent mix, and the
    same as trqrcp_batched gives on that matrix."""
    from paper_1509_06820_gb300.serve import Request, RingServer, make_input
    srv = RingServer(teams=4, capacity=16, keep_results=True)
    try:
        alone = _ring_run(srv, [Request(i, *s) for i, s in enumerate(SIZES)], together=False)
        mixed = _ring_run(srv, [Request(i, *s) for i, s in enumerate(SIZES)], together=True)
        assert srv.max_in_flight > 1
    finally:
        srv.close()
    for i in range(len(SIZES)):
        for x, y in zip(alone[i], mixed[i]):
            np.testing.assert_array_equal(x, y)
    # the batched entry point on the same inputs (same team size, b, p)
    for i, (m, n, k) in enumerate(SIZES):
        r = Request(i, m, n, k)
        A = lib.empty_colmajor(m, n, "cuda", torch.float32)
        make_input(r, A, torch.cuda.current_stream())
        out = lib.trqrcp_batched([(A, k, min(k, 64), 8, i)])[0]
        for x, y in zip(out, alone[i]):
            np.testing.assert_array_equal(x.cpu().numpy(), y)


def test_ring_server_factors_reconstruct(lib):
    """The served rank-k factors reproduce A = X Y^T (rank k) to FP32 level."""
    from oracle import householder as hh
    from paper_1509_06820_gb300.serve import Request, RingServer, make_input
    srv = RingServer(teams=2, capacity=8, keep_results=True)
    try:
        reqs = [Request(200 + i, *s) for i, s in enumerate(SIZES[:4])]
        res = _ring_run(srv, reqs, together=True)
    finally:
        srv.close()
    for r in reqs:
        A = lib.empty_colmajor(r.m, r.n, "cuda", torch.float32)
        make_input(r, A, torch.cuda.current_stream())
        A64 = A.cpu().numpy().astype(np.float64)
        jp, tau, Y, R, rd = res[r.rid]
        k = r.k
        R = R.astype(np.float64)
        R[np.arange(k), np.arange(k)] = rd
        Q = hh.form_q(Y.astype(np.float64), tau, k)
        approx = np.zeros_like(A64)
        approx[:, jp] = Q @ R
        assert np.linalg.norm(A64 - approx) <= 1e-5 * np.linalg.norm(A64)


def test_ring_server_restarts_after_idle(lib):
    """The teams leave the kernel after an idle spell; the next request starts
    it again and is served."""
    import time
    from paper_1509_06820_gb300.serve import Request, RingServer
    srv = RingServer(teams=2, capacity=4, keep_results=True)
    try:
        first = _ring_run(srv, [Request(0, 300, 400, 20)], together=True)
        time.sleep(1.5)  # longer than the kernel's idle bound
        again = _ring_run(srv, [Request(0, 300, 400, 20)], together=True)
    finally:
        srv.close()
    for x, y in zip(first[0], again[0]):
        np.testing.assert_array_equal(x, y)


def test_ring_server_poisson(lib):
    from paper_1509_06820_gb300.serve import RingServer
    srv = RingServer(capacity=64)
    try:
        stats = srv.run_poisson(rate=500, duration=1.0, warmup=0.2, seed=3,
                                size_range=(256, 1024), k_range=(16, 64))
    finally:
        srv.close()
    assert stats["requests"] > 200
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]


EDGE = [(1, 1, 1, 1, 0), (5, 3, 3, 8, 2), (300, 40, 40, 16, 4), (40, 300, 40, 32, 0),
        (257, 129, 100, 32, 8), (64, 64, 64, 64, 8), (1000, 17, 17, 128, 16)]


def test_trqrcp_batched_edge_shapes(lib):
    """Degenerate and ragged problems in one batch (1 x 1, b > k clamped,
    k = n so the last block has no trailing columns, p = 0, m < n, a ragged
    last block): the first k selected columns are reproduced by Q R, R agrees
    with the FP64 oracle's Alg. 6 replayed on the device's pivots, and the
    trailing columns of R are Q_k^T A P."""
    import oracle
    from oracle import householder as hh
    import synth
    probs, hosts = [], []
    for i, (m, n, k, b, p) in enumerate(EDGE):
        A = synth.gaussian(m, n, seed=40 + i).astype(np.float32)
        hosts.append(A)
        probs.append((lib.colmajor(torch.from_numpy(A).cuda()), k, b, p, 3 + i))
    got = lib.trqrcp_batched(probs, teams=2)
    assert lib.sync_info() == 0
    for (dA, k, b, p, seed), A, out in zip(probs, hosts, got):
        jp, t, Yg, Rg, rd = (x.cpu().numpy() for x in out)
        A64 = A.astype(np.float64)
        m, n = A64.shape
        assert sorted(jp.tolist()) == list(range(n))
        Rg = Rg.astype(np.float64)
        Rg[np.arange(k), np.arange(k)] = rd
        Q = hh.form_q(Yg.astype(np.float64), t, k)
        sel = A64[:, jp[:k]]
        assert np.linalg.norm(sel - Q @ Rg[:, :k]) <= 1e-5 * np.linalg.norm(sel)
        if k < n:
            rest = Q.T @ A64[:, jp[k:]]
            assert np.linalg.norm(Rg[:, k:] - rest) <= 1e-5 * np.linalg.norm(A64)
        _, _, _, Ro, _ = oracle.trqrcp(A64, k, min(b, k), p, seed=seed, replay_jpvt=jp,
                                       tie_rtol=1.0)
        assert np.linalg.norm(Rg - Ro) <= 1e-4 * max(np.linalg.norm(Ro), 1e-30)


def test_trqrcp_batched_rejects_oversize_sample(lib):
    """A problem whose sample does not fit the team's shared memory fails the
    whole call before launch, naming the problem."""
    A = lib.colmajor(torch.randn(600, 4096, device="cuda"))
    ok = lib.colmajor(torch.randn(300, 300, device="cuda"))
    with pytest.raises(lib.RqrcpError, match="problem 1"):
        lib.trqrcp_batched([(ok, 16, 16, 8, 1), (A, 128, 128, 64, 1)])
