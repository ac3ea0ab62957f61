"""Autotuner for the block size b and oversampling p of the served TRQRCP
(the stream-slot path through trqrcp_mixed, or the persistent batched
kernel through trqrcp_batched).

For each size bucket (M, N, K) it times the mixed-precision TRQRCP on a
rank-K Gaussian-factor matrix of that size for every candidate (b, p) with
CUDA events and keeps the fastest; the table is JSON and the server looks up
the nearest bucket (log-distance in M, N, K).  Candidates keep p >= 4 so the
sample rank l = b + p stays above b.
"""
import json
import math

import torch

from . import empty_colmajor, Handle, trqrcp_batched, trqrcp_mixed, RqrcpError

CANDIDATES = [(16, 8), (32, 8), (64, 8), (128, 8), (32, 4), (64, 16), (128, 16)]


class Tuner:
    def __init__(self, table=None, default=(64, 8)):
        self.table = dict(table or {})
        self.default = default

    @staticmethod
    def key(M, N, K):
        return f"{M}x{N}x{K}"

    def choose(self, M, N, K):
        if not self.table:
            return (min(self.default[0], K), self.default[1])
        k = self.key(M, N, K)
        if k in self.table:
            b, p = self.table[k]["b"], self.table[k]["p"]
        else:
            def dist(entry):
                m2, n2, k2 = (int(x) for x in entry.split("x"))
                return (math.log(m2 / M) ** 2 + math.log(n2 / N) ** 2 + math.log(k2 / K) ** 2)
            best = min(self.table, key=dist)
            b, p = self.table[best]["b"], self.table[best]["p"]
        return (min(b, K), p)

    def save(self, path):
        with open(path, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)

    @classmethod
    def load(cls, path):
        with open(path) as f:
            return cls(json.load(f))

    @classmethod
    def tune(cls, buckets, device="cuda", candidates=CANDIDATES, reps=3):
        dev = torch.device(device)
        h = Handle(dev)
        table = {}
        for (M, N, K) in buckets:
            g = torch.Generator(device=dev)
            g.manual_seed(M * 7 + N * 3 + K)
            X = torch.randn((M, K), generator=g, device=dev)
            Y = torch.randn((N, K), generator=g, device=dev)
            A = empty_colmajor(M, N, dev, torch.float32)
            A.t().copy_(Y @ X.t())
            best = None
            for (b, p) in candidates:
                if b > K:
                    continue
                h.reserve("V", M, N, K, b, p)
                trqrcp_mixed(A, K, b, p, 1, handle=h)
                times = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    trqrcp_mixed(A, K, b, p, 1, handle=h)
                    e1.record()
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
                t = sorted(times)[len(times) // 2]
                if best is None or t < best[2]:
                    best = (b, p, t)
            table[cls.key(M, N, K)] = {"b": best[0], "p": best[1], "ms": best[2]}
        h.close()
        return cls(table)

    @classmethod
    def tune_batched(cls, buckets, device="cuda", team=16, candidates=CANDIDATES, reps=3):
        """The same search for the persistent batched kernel: each candidate
        (b, p) is timed on one problem run by one team of `team` CTAs (the
        time a serving team spends on such a request); candidates whose sample
        or panel does not fit the team are skipped."""
        dev = torch.device(device)
        h = Handle(dev)
        h.set_batch_team(team)
        table = {}
        for (M, N, K) in buckets:
            g = torch.Generator(device=dev)
            g.manual_seed(M * 7 + N * 3 + K)
            X = torch.randn((M, K), generator=g, device=dev)
            Y = torch.randn((N, K), generator=g, device=dev)
            A = empty_colmajor(M, N, dev, torch.float32)
            A.t().copy_(Y @ X.t())
            best = None
            for (b, p) in candidates:
                if b > K:
                    continue
                try:
                    outs = trqrcp_batched([(A, K, b, p, 1)], teams=1, handle=h)
                except RqrcpError:
                    continue
                times = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    trqrcp_batched([(A, K, b, p, 1)], teams=1, handle=h, outs=outs)
                    e1.record()
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
                t = sorted(times)[len(times) // 2]
                if best is None or t < best[2]:
                    best = (b, p, t)
            if best is not None:
                table[cls.key(M, N, K)] = {"b": best[0], "p": best[1], "ms": best[2]}
        h.close()
        return cls(table)
