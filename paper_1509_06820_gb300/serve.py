"""Continuous-batching server for low-rank approximation requests.

Each request asks for the rank-k TRQRCP factorization (Alg. 6, mixed
precision: FP32 storage, split-BF16 tensor-core products, FP64 sample QRCP,
panels and T) of an m x n matrix.  The server keeps a pool of slots; a slot
owns a CUDA stream and an rqrcp handle whose scratch holds the request's
sample, reflector and inner-product state on the device while it runs.

* Admission: requests wait in FIFO order; one is admitted when a slot is free
  and its HBM footprint (input, outputs) fits in what is left of the budget
  after the slots' reserved scratch.  Requests that arrive while others run
  are admitted as soon as a slot and memory free up, so their kernels overlap
  on the device with the ones already in flight (continuous batching).
* Launch: a request is enqueued on its slot's stream as one CUDA graph: the
  first request of each (slot, size bucket) is captured (shapes rounded up to
  the bucket, A zero-padded -- zero columns are never pivoted and zero rows
  leave the reflectors unchanged, and the Philox compression matrix is
  prefix-stable in m), later ones replay it.  With graphs off the calls are
  enqueued eagerly at the request's exact size, into the request's own output
  tensors.
* Each slot's handle caps the SMs its launches spread over (by default a
  quarter of the device's SMs), so requests of different slots run side
  by side instead of each split-K product or cooperative kernel filling the
  GPU.
* Completion is polled with CUDA events; latency = completion - arrival.
* b and p per size bucket come from the autotuner table (autotune.py).

Only host-side scheduling lives here: every numerical step runs in the CUDA
kernels behind the C ABI.
"""
import collections
import gc
import ctypes
import math
import time

import numpy as np
import torch

from . import _ld, _ptr, empty_colmajor, Handle, trqrcp_mixed, load, RQRCP_ERR_BUSY


def request_flops(m, n, k, ell):
    """Algorithmic flops of one TRQRCP request: sketch 2 l m n plus the
    inner products with A, 2 m n k (the same count for every (b, p))."""
    return 2.0 * ell * m * n + 2.0 * m * n * k


class Request:
    __slots__ = ("rid", "m", "n", "k", "seed", "t_arrival", "t_admit", "t_publish", "t_done",
                 "result", "bucket", "b", "p", "slot")

    def __init__(self, rid, m, n, k, seed=None, t_arrival=0.0):
        self.rid = rid
        self.m, self.n, self.k = int(m), int(n), int(k)
        self.seed = rid if seed is None else seed
        self.t_arrival = t_arrival
        self.t_admit = None
        self.t_publish = None
        self.t_done = None
        self.result = None
        self.bucket = None
        self.b = self.p = None
        self.slot = None


def factors(req):
    """(jpvt[:k], tau, Y (m x k), R (k x n), rdiag) of a finished request, on
    the device.  R keeps the columns of the original matrix in pivot order:
    padding columns of the size bucket (index >= n) are dropped."""
    jpvt, tau, Y, R, rdiag = req.result
    keep = jpvt < req.n
    return jpvt[keep][: req.n], tau, Y, R[:, keep], rdiag


def make_input(req, out, stream, gen=None):
    """The request's matrix A = X Y^T (X: m x k, Y: n x k, N(0,1) from the
    request's seed: one draw of (m + n) x k, X its first m rows) written into
    the column-major FP32 view `out`.  gen: a CUDA generator to reseed (one
    per slot saves creating one per request)."""
    with torch.cuda.stream(stream):
        g = gen if gen is not None else torch.Generator(device=out.device)
        g.manual_seed(int(req.seed))
        XY = torch.randn((req.m + req.n, req.k), generator=g, device=out.device,
                         dtype=torch.float32)
        out[: req.m, : req.n].t().copy_(XY[req.m:] @ XY[: req.m].t())


class Slot:
    """One concurrent request: a stream, a handle and cached per-bucket graphs.

    Captured graphs hold the handle's scratch pointers, so the scratch is
    reserved once for the largest bucket and never moves; if a bucket ever
    needs more, the slot's graphs are dropped before the scratch grows.
    """

    def __init__(self, device, max_m, max_n, max_k, use_graphs, bp_choices=((128, 16), (64, 16)),
                 max_sms=0):
        self.device = device
        self.stream = torch.cuda.Stream(device)
        self.handle = Handle(device)
        # cap the SMs one request's launches spread over, so that the slots'
        # requests run side by side instead of each filling the GPU
        self.handle.set_max_sms(max_sms)
        self.event = torch.cuda.Event()
        self.gen = torch.Generator(device=device)
        self.req = None
        self.use_graphs = use_graphs
        self.graphs = {}  # (bucket, b, p) -> (graph, A view, outputs)
        self.max = (max_m, max_n, max_k)
        self.reserved = 0
        for b, p in bp_choices:
            self._reserve(max_m, max_n, max_k, min(b, max_k), p)
        # one buffer set of the largest size; buckets use leading-dimension views
        self.bufA = empty_colmajor(max_m, max_n, device, torch.float32)
        self.bufs = (torch.empty(max_n, dtype=torch.int64, device=device),
                     torch.empty(max_k, dtype=torch.float64, device=device),
                     empty_colmajor(max_m, max_k, device, torch.float32),
                     empty_colmajor(max_k, max_n, device, torch.float32),
                     torch.empty(max_k, dtype=torch.float64, device=device))

    def _reserve(self, M, N, K, b, p):
        need = int(load().rqrcp_workspace_bytes(b"V", M, N, K, b, p))
        if need > self.reserved:
            self.graphs.clear()   # their scratch pointers are about to move
            with torch.cuda.stream(self.stream):
                self.handle.reserve("V", M, N, K, b, p)
            self.reserved = need

    def _buffers(self, bucket):
        M, N, K = bucket
        jp, tau, Y, R, rd = self.bufs
        return self.bufA[:M, :N], (jp[:N], tau[:K], Y[:M, :K], R[:K, :N], rd[:K])

    def launch(self, req):
        M, N, K = req.bucket
        if not self.use_graphs:
            self._launch_eager(req)
            return
        entry = self.graphs.get((req.bucket, req.b, req.p))
        if entry is None:
            A, outs = self._buffers(req.bucket)
            graph = None
            self._reserve(M, N, K, req.b, req.p)
            if self.use_graphs:
                with torch.cuda.stream(self.stream):
                    A.zero_()
                    # eager run first: sets kernel attributes and sizes the scratch
                    trqrcp_mixed(A, K, req.b, req.p, 1, handle=self.handle, out=outs)
                self.stream.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=self.stream):
                    trqrcp_mixed(A, K, req.b, req.p, 1, handle=self.handle, out=outs)
            entry = (graph, A, outs)
            self.graphs[(req.bucket, req.b, req.p)] = entry
        graph, A, outs = entry
        self.req = req
        req.slot = self
        k, m = req.k, req.m
        with torch.cuda.stream(self.stream):
            if req.m < M or req.n < N:
                A.zero_()
            make_input(req, A, self.stream, self.gen)
            if graph is not None:
                graph.replay()
            else:
                trqrcp_mixed(A, K, req.b, req.p, 1, handle=self.handle, out=outs)
            # the slot's buffers are reused by the next request: the request
            # keeps its own copy of the factors
            jpvt, tau, Y, R, rdiag = outs
            req.result = (jpvt.clone(), tau[:k].clone(), Y[:m, :k].clone(), R[:k, :].clone(),
                          rdiag[:k].clone())
            self.event.record(self.stream)

    def _launch_eager(self, req):
        """Eager launches at the request's own size (no bucket padding, which
        only serves graph reuse), written straight into the request's own
        output tensors (no copies)."""
        M, N, K = req.bucket
        self._reserve(M, N, K, req.b, req.p)
        A = self.bufA[:M, :N]
        self.req = req
        req.slot = self
        with torch.cuda.stream(self.stream):
            if req.m < M or req.n < N:
                A.zero_()
            make_input(req, A, self.stream, self.gen)
            own = (torch.empty(N, dtype=torch.int64, device=self.device),
                   torch.empty(K, dtype=torch.float64, device=self.device),
                   empty_colmajor(M, K, self.device, torch.float32),
                   empty_colmajor(K, N, self.device, torch.float32),
                   torch.empty(K, dtype=torch.float64, device=self.device))
            trqrcp_mixed(A, K, req.b, req.p, 1, handle=self.handle, out=own)
            jpvt, tau, Y, R, rdiag = own
            k, m = req.k, req.m
            req.result = (jpvt, tau[:k], Y[:m, :k], R[:k, :], rdiag[:k])
            self.event.record(self.stream)

    def done(self):
        return self.req is not None and self.event.query()


class Server:
    """Continuous-batching TRQRCP server on one GPU.

    `slots` are Slot objects (or any object with launch(req), done() and a
    `req` attribute); `Server.on_gpu` builds real ones.
    """

    def __init__(self, slots, hbm_budget=16 << 30, tuner=None, bucket=512, kbucket=32,
                 footprint_fn=None, clock=time.perf_counter):
        self.bucket = bucket
        self.kbucket = kbucket
        self.tuner = tuner
        self.slots = list(slots)
        self.free = collections.deque(self.slots)
        self.pending = collections.deque()
        self.running = []
        self.done = []
        self.hbm_budget = hbm_budget
        self.in_flight_bytes = 0
        self.max_in_flight = 0
        self.footprint_fn = footprint_fn
        self.clock = clock

    @classmethod
    def on_gpu(cls, device="cuda", slots=8, use_graphs=True, max_m=4096, max_n=4096, max_k=128,
               max_sms=None, **kw):
        """max_sms: SMs per request's launches (None: a quarter of the
        device's SMs, at least 16; 0: all)."""
        dev = torch.device(device)
        # size buckets only serve graph reuse: eager slots solve exact sizes
        kw.setdefault("bucket", 512 if use_graphs else 1)
        kw.setdefault("kbucket", 32 if use_graphs else 1)
        if max_sms is None:
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            max_sms = max(16, nsm // 4)
        return cls([Slot(dev, max_m, max_n, max_k, use_graphs, max_sms=max_sms)
                    for _ in range(slots)], **kw)

    # ---------------------------------------------------------------- sizing
    def plan(self, req):
        M = int(math.ceil(req.m / self.bucket) * self.bucket)
        N = int(math.ceil(req.n / self.bucket) * self.bucket)
        K = int(min(math.ceil(req.k / self.kbucket) * self.kbucket, min(M, N)))
        req.bucket = (M, N, K)
        b, p = (self.tuner.choose(M, N, K) if self.tuner else (min(K, 64), 8))
        req.b, req.p = b, p
        return req

    def footprint(self, req):
        """HBM bytes the request holds while in flight: its padded input and
        outputs plus the handle scratch of its bucket."""
        if self.footprint_fn is not None:
            return self.footprint_fn(req)
        M, N, K = req.bucket
        io = M * N * 4 + N * 8 + K * 16 + (M * K + K * N) * 4
        ws = load().rqrcp_workspace_bytes(b"V", M, N, K, req.b, req.p)
        return io + int(ws)

    # ---------------------------------------------------------------- loop
    def submit(self, req):
        self.pending.append(self.plan(req))

    def poll(self):
        """Retire finished requests, then admit waiting ones (FIFO) while a
        slot is free and the budget allows."""
        still = []
        for req in self.running:
            if req.slot.done():
                req.t_done = self.clock()
                self.in_flight_bytes -= self.footprint(req)
                req.slot.req = None
                self.free.append(req.slot)
                self.done.append(req)
            else:
                still.append(req)
        self.running = still
        while self.pending and self.free:
            req = self.pending[0]
            fp = self.footprint(req)
            if self.in_flight_bytes + fp > self.hbm_budget and self.running:
                break
            self.pending.popleft()
            slot = self.free.popleft()
            req.t_admit = self.clock()
            self.in_flight_bytes += fp
            req.slot = slot
            slot.launch(req)
            self.running.append(req)
            self.max_in_flight = max(self.max_in_flight, len(self.running))

    def drain(self):
        while self.pending or self.running:
            self.poll()
            if self.running and not any(r.slot.done() for r in self.running):
                time.sleep(20e-6)

    # ---------------------------------------------------------------- workload
    def run_poisson(self, rate, duration, warmup=0.0, seed=7, size_range=(256, 4096),
                    k_range=(16, 128)):
        """Serve a Poisson stream at `rate` req/s for warmup + duration seconds;
        statistics cover requests that arrived after the warm-up."""
        return run_poisson(self, rate, duration, warmup, seed, size_range, k_range)


def poisson_arrivals(rate, total, seed, size_range, k_range):
    """(arrival time, Request) pairs of a Poisson stream over `total` seconds:
    m, n uniform in size_range, k uniform in k_range (at most min(m, n))."""
    rng = np.random.default_rng(seed)
    t = 0.0
    arrivals = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > total:
            break
        m = int(rng.integers(size_range[0], size_range[1] + 1))
        n = int(rng.integers(size_range[0], size_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        arrivals.append((t, Request(rid, m, n, min(k, m, n))))
        rid += 1
    return arrivals


def run_poisson(server, rate, duration, warmup=0.0, seed=7, size_range=(256, 4096),
                k_range=(16, 128)):
    """Drive `server` (submit / poll / pending / running / done) with a Poisson
    stream; latency = completion seen by the host - arrival.  The host loop is
    the only thread that admits, publishes and observes completions, so the
    cyclic garbage collector is held off while it runs (reference counting
    still frees every request's tensors): a collection pass over the
    thousands of finished requests stalls every request in flight."""
    arrivals = poisson_arrivals(rate, warmup + duration, seed, size_range, k_range)
    server.done = []
    i = 0
    def busy():
        return bool(server.pending or server.running or getattr(server, "staged", None))

    gc_was_enabled = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        while i < len(arrivals) or busy():
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                req = arrivals[i][1]
                req.t_arrival = t0 + arrivals[i][0]
                server.submit(req)
                i += 1
            server.poll()
            if i < len(arrivals) and not busy():
                wait = arrivals[i][0] - (time.perf_counter() - t0)
                if wait > 50e-6:
                    time.sleep(min(wait, 200e-6))
        t_end = time.perf_counter()
    finally:
        if gc_was_enabled:
            gc.enable()
    measured = [r for r in server.done if r.t_arrival - t0 >= warmup]
    lat = np.array([r.t_done - r.t_arrival for r in measured]) * 1e3
    span = max(r.t_done for r in measured) - min(r.t_arrival for r in measured)
    flops = sum(request_flops(r.m, r.n, r.k, r.b + r.p) for r in measured)
    parts = {}
    if measured and measured[0].t_publish is not None:
        # where a request's latency goes: waiting for admission, its input
        # being produced, and the device serving it after publication
        def pct(xs):
            xs = np.array(xs) * 1e3
            return {"mean": float(xs.mean()), "p50": float(np.percentile(xs, 50)),
                    "p99": float(np.percentile(xs, 99))}
        parts = {"latency_parts_ms": {
            "admission_wait": pct([r.t_admit - r.t_arrival for r in measured]),
            "input": pct([r.t_publish - r.t_admit for r in measured]),
            "service": pct([r.t_done - r.t_publish for r in measured])}}
    return {
        **parts,
        "requests": len(measured), "offered_rate": rate,
        "throughput_rps": len(measured) / span, "gflops": flops / span / 1e9,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "wall_s": t_end - t0, "slots": getattr(server, "nslots", len(getattr(server, "slots", []))),
    }


class RingServer:
    """Continuous batching on the persistent kernel (rqrcp_server_*).

    One long-running launch of the batched TRQRCP kernel serves every request:
    its teams (groups of CTAs) claim requests from a ring in page-locked,
    mapped host memory as the host publishes them, so no capture, graph
    replay or per-request launch sits on a request's path.  The host side:

    * admission: FIFO; a request is admitted when its HBM footprint (input and
      outputs) fits the budget and the ring has a free slot;
    * input: the request's matrix A = X Y^T is produced on a side stream by
      SMs the teams leave free (`reserve_sms`); once it is ready the request
      is published to the ring;
    * completion: the ring's done word of the request (written by the team
      with system-scope release) is polled; latency = completion - arrival.

    Outputs are the request's own tensors (freed when it retires unless
    `keep_results`); the kernel no longer touches them once the done word is
    set, so they go back to the allocator without waiting on the server's
    stream.
    """

    def __init__(self, device="cuda", team=16, teams=None, capacity=512, max_m=4096, max_n=4096,
                 max_k=128, max_b=64, max_p=16, hbm_budget=16 << 30, tuner=None, reserve_sms=16,
                 keep_results=False, clock=time.perf_counter):
        from . import Problem  # noqa: F401  (the ring's descriptor type)
        self.device = torch.device(device)
        nsm = torch.cuda.get_device_properties(self.device).multi_processor_count
        if teams is None:
            teams = max(1, (nsm - reserve_sms) // team)
        self.nslots = teams
        self.team = team
        self.capacity = capacity
        self.limits = (max_m, max_n, max_k, max_b, max_p)
        self.tuner = tuner
        self.hbm_budget = hbm_budget
        self.keep_results = keep_results
        self.clock = clock
        self.handle = Handle(self.device)
        self.handle.set_batch_team(team)
        self.stream = torch.cuda.Stream(self.device)      # the server's launch
        self.in_stream = torch.cuda.Stream(self.device)   # request inputs
        self.gen = torch.Generator(device=self.device)
        self.handle.bind(self.stream)
        from . import _check
        _check(load().rqrcp_server_start(self.handle.h, capacity, teams, max_m, max_n, max_k,
                                         max_b, max_p), self.handle.h)
        self.pending = collections.deque()   # waiting for admission
        self.staged = collections.deque()    # input being produced
        self.running = []                    # published to the ring
        self.done = []
        self.in_flight_bytes = 0
        self.max_in_flight = 0

    def plan(self, req):
        b, p = self.tuner.choose(req.m, req.n, req.k) if self.tuner else (min(req.k, 64), 8)
        # within the sizes the server was started for
        req.b, req.p = min(b, req.k, self.limits[3]), min(p, self.limits[4])
        req.bucket = (req.m, req.n, req.k)
        return req

    @staticmethod
    def footprint(req):
        m, n, k = req.m, req.n, req.k
        return m * n * 4 + n * 8 + k * 16 + (m * k + k * n) * 4

    def submit(self, req):
        self.pending.append(self.plan(req))

    def _admit(self, req):
        from . import trqrcp_outputs
        with torch.cuda.stream(self.in_stream):
            A = empty_colmajor(req.m, req.n, self.device, torch.float32)
            out = trqrcp_outputs(req.m, req.n, req.k, self.device)
            make_input(req, A, self.in_stream, self.gen)
            ev = torch.cuda.Event()
            ev.record(self.in_stream)
        req.t_admit = self.clock()
        req.slot = (A, out, ev, None)
        self.in_flight_bytes += self.footprint(req)
        self.staged.append(req)

    def _publish(self, req):
        from . import problem_struct
        A, out, ev, _ = req.slot
        prob = problem_struct(A, req.k, req.b, req.p, int(req.seed), out)
        ticket = ctypes.c_int64(0)
        rc = load().rqrcp_server_submit(self.handle.h, ctypes.byref(prob), ctypes.byref(ticket))
        if rc == RQRCP_ERR_BUSY:
            return False
        if rc != 0:
            raise RuntimeError(f"rqrcp_server_submit: {rc}")
        req.slot = (A, out, ev, ticket.value)
        req.t_publish = self.clock()
        return True

    def poll(self):
        info = ctypes.c_int(0)
        info_ref = ctypes.byref(info)
        server_poll = load().rqrcp_server_poll
        h = self.handle.h
        still = []
        for req in self.running:
            rc = server_poll(h, req.slot[3], info_ref)
            if rc < 0:
                raise RuntimeError(f"rqrcp_server_poll: {rc}")
            if rc == 1:
                req.t_done = self.clock()
                if info.value:
                    raise RuntimeError(f"request {req.rid}: device status {info.value}")
                A, out, _, _ = req.slot
                jpvt, tau, Y, R, rdiag = out
                req.result = (jpvt, tau, Y, R, rdiag) if self.keep_results else None
                req.slot = None
                self.in_flight_bytes -= self.footprint(req)
                self.done.append(req)
            else:
                still.append(req)
        self.running = still
        while self.staged and self.staged[0].slot[2].query():
            req = self.staged[0]
            if not self._publish(req):
                break
            self.staged.popleft()
            self.running.append(req)
        while self.pending:
            req = self.pending[0]
            inflight = len(self.staged) + len(self.running)
            if inflight >= self.capacity:
                break
            if self.in_flight_bytes + self.footprint(req) > self.hbm_budget and inflight:
                break
            self.pending.popleft()
            self._admit(req)
        self.max_in_flight = max(self.max_in_flight, len(self.running))

    @property
    def busy(self):
        return bool(self.pending or self.staged or self.running)

    def drain(self):
        while self.busy:
            self.poll()
            if self.running:
                time.sleep(20e-6)

    def run_poisson(self, rate, duration, warmup=0.0, seed=7, size_range=(256, 4096),
                    k_range=(16, 128)):
        return run_poisson(self, rate, duration, warmup, seed, size_range, k_range)

    def close(self):
        """Stop the server's launch and wait for it."""
        if self.handle is not None:
            load().rqrcp_server_stop(self.handle.h)
            self.stream.synchronize()
            self.handle.close()
            self.handle = None
