"""Host-side logic of the serving loop (no GPU): bucketing, FIFO admission by
HBM footprint, slot reuse, latency bookkeeping, autotuner table lookup."""
import pytest

torch = pytest.importorskip("torch")

from paper_1509_06820_gb300.serve import Request, Server, request_flops
from paper_1509_06820_gb300.autotune import Tuner


class FakeSlot:
    """Completes a request after `polls` calls to done()."""

    def __init__(self, polls=2):
        self.req = None
        self.polls = polls
        self.left = 0
        self.launched = []

    def launch(self, req):
        self.req = req
        self.left = self.polls
        self.launched.append(req.rid)

    def done(self):
        if self.req is None:
            return False
        self.left -= 1
        return self.left <= 0


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def make_server(nslots=2, budget=10, fp=lambda r: 4, **kw):
    slots = [FakeSlot() for _ in range(nslots)]
    return Server(slots, hbm_budget=budget, footprint_fn=fp, clock=Clock(), **kw), slots


def test_unit_buckets_keep_exact_sizes():
    """Eager slots solve each request at its own size: with buckets of 1 the
    plan is the request itself (the graph mode rounds up for reuse)."""
    srv, _ = make_server(bucket=1, kbucket=1)
    r = srv.plan(Request(0, 300, 1000, 40))
    assert r.bucket == (300, 1000, 40)
    r = srv.plan(Request(1, 257, 129, 200))
    assert r.bucket == (257, 129, 129)   # k capped at min(m, n)


def test_bucketing_rounds_up_and_caps_k():
    srv, _ = make_server()
    r = srv.plan(Request(0, 300, 1000, 40))
    assert r.bucket == (512, 1024, 64)
    r = srv.plan(Request(1, 256, 256, 128))
    assert r.bucket == (512, 512, 128)
    r = srv.plan(Request(2, 100, 700, 90))
    assert r.bucket == (512, 1024, 96)
    assert r.b <= r.bucket[2]


def test_fifo_admission_respects_slots_and_budget():
    # footprint 4 each, budget 10 -> at most 2 in flight even with 3 slots
    srv, slots = make_server(nslots=3, budget=10)
    for i in range(5):
        srv.submit(Request(i, 512, 512, 32))
    srv.poll()
    assert [r.rid for r in srv.running] == [0, 1]
    assert srv.in_flight_bytes == 8
    srv.drain()
    assert sorted(r.rid for r in srv.done) == list(range(5))
    assert srv.max_in_flight == 2
    assert srv.in_flight_bytes == 0
    # FIFO: admission order follows arrival order
    admitted = sorted(srv.done, key=lambda r: r.t_admit)
    assert [r.rid for r in admitted] == list(range(5))


def test_oversized_request_runs_alone():
    # a request larger than the budget is admitted only when nothing else runs
    srv, _ = make_server(nslots=2, budget=10, fp=lambda r: 20 if r.rid == 1 else 4)
    for i in range(3):
        srv.submit(Request(i, 512, 512, 32))
    srv.poll()
    assert [r.rid for r in srv.running] == [0]
    srv.drain()
    assert len(srv.done) == 3


def test_latency_bookkeeping():
    srv, _ = make_server(nslots=1)
    r = Request(0, 512, 512, 16, t_arrival=0.0)
    srv.submit(r)
    srv.drain()
    assert r.t_done > r.t_admit > r.t_arrival


def test_request_flops():
    assert request_flops(100, 200, 10, 18) == 2.0 * 18 * 100 * 200 + 2.0 * 100 * 200 * 10


def test_tuner_lookup_and_roundtrip(tmp_path):
    t = Tuner({"1024x1024x64": {"b": 32, "p": 8, "ms": 1.0},
               "4096x4096x128": {"b": 128, "p": 16, "ms": 3.0}})
    assert t.choose(1024, 1024, 64) == (32, 8)
    assert t.choose(3584, 4096, 128) == (128, 16)   # nearest bucket
    assert t.choose(1024, 1024, 16) == (16, 8)      # b clamped to K
    path = tmp_path / "tune.json"
    t.save(path)
    assert Tuner.load(path).table == t.table
    assert Tuner().choose(512, 512, 32) == (32, 8)
