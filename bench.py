#!/usr/bin/env python
"""Benchmark: randomized QR with column pivoting (Alg. 4) on a GB300.

Workload: one 16384 x 16384 FP64 matrix A = U diag(sigma) V^T with Haar U, V
(QR of seeded Gaussians) and sigma_i = 10^(-12 (i-1)/(n-1)); block b = 64,
oversampling p = 8, Omega from Philox seed 1.  A step is one full
factorization (sketch, and per block: sample QRCP, column permutation,
panel + T, trailing update, sample update) after restoring A from a
resident copy.  The same matrix is also factored by the project's own
unpivoted blocked QR, the paper's baseline for the cost of pivoting.

Flop convention (LAPACK dgeqrf count, used for both routines so that the
rate ratio is the time ratio): 2 m n^2 - 2 n^3 / 3.

Multi-GPU: every rank factors its own matrix (replicas, no collective on
the data path); value = all ranks' flops / the slowest rank's time.

--impl reference times the CPU oracle (numpy float64) on the host cores on
a bounded sample of the same workload: the first blocks of the same
factorization, scaled by their algorithmic flops.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RQRCP GFLOP/s & time vs own unpivoted QR at 16384^2 FP64"
UNIT = "GFLOP/s"


def flops_geqrf(m, n):
    k = min(m, n)
    if m >= n:
        return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
    return 2.0 * n * m * m - 2.0 * m ** 3 / 3.0


def block_flops(m, n, b, p, nblocks):
    """Algorithmic flops of the first `nblocks` blocks of Alg. 4 (sketch,
    sample QRCP, panel + T, trailing update, sample update)."""
    ell = b + p
    k = min(m, n)
    fl = 2.0 * ell * m * n
    j0 = 0
    for _ in range(nblocks):
        if j0 >= k:
            break
        bJ = min(b, k - j0)
        mJ, nc = m - j0, n - j0
        n2 = nc - bJ
        fl += sum(4.0 * (ell - i) * (nc - i - 1) for i in range(min(bJ, ell)))
        fl += 2.0 * mJ * bJ * bJ - 2.0 * bJ ** 3 / 3.0
        fl += 4.0 * mJ * n2 * bJ
        fl += 2.0 * bJ * bJ * n2
        j0 += bJ
    return fl


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--cpu-blocks", type=int, default=6,
                    help="blocks of the factorization in the oracle's bounded sample")
    ap.add_argument("--no-extras", action="store_true",
                    help="run the FP64 step only (no extra legs; same as --legs '')")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--only-emulated", action="store_true",
                    help="same as --legs emulated")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--legs", default="qr,e2e,cpu,emulated,rsrqrcp,qrcp,quality,mixed,truncated,serving",
                    help="comma-separated extra legs to run after the FP64 step")
    ap.add_argument("--case", choices=["panel", "gemm_bf16x", "gemm_f64x", "qrcp", "sample", "mixed",
                                       "rqrcp", "qr", "fp64peak", "batched", "serve"],
                    default=None,
                    help="run one small kernel case (for profiling) instead of the benchmark")
    ap.add_argument("--shape", default=None,
                    help="--case gemm_*: transA,transB,M,N,K (e.g. T,N,128,8000,8192)")
    ap.add_argument("--m", type=int, default=16384, help="--case panel: rows")
    ap.add_argument("--emulated", action="store_true",
                    help="--case rqrcp / qr: FP64 trailing update as tensor-core slice products")
    ap.add_argument("--reps", type=int, default=1, help="--case: timed repetitions")
    ap.add_argument("--team", type=int, default=16,
                    help="--case batched / serve: CTAs per team (serve: 0 = autotuned)")
    ap.add_argument("--max-sms", type=int, default=0,
                    help="--case: cap on the CTAs per wave of the handle's launches (0: all)")
    args = ap.parse_args()
    legs = set(x for x in args.legs.split(",") if x)
    if args.no_extras:
        legs = set()
    if args.only_emulated:
        legs = {"emulated"}
    args.legs = legs
    return args


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle legs
def cpu_sample(A_host, b, p, nblocks):
    """Time the oracle on the first `nblocks` blocks of the factorization."""
    import numpy as np
    import oracle
    k = nblocks * b
    t0 = time.perf_counter()
    oracle.rqrcp(A_host, b, p, seed=1, k=k)
    dt = time.perf_counter() - t0
    m, n = A_host.shape
    fl = block_flops(m, n, b, p, nblocks)
    return fl / dt / 1e9, dt


def host_matrix(n):
    import torch
    import synth
    if torch.cuda.is_available():
        A = synth.graded_device(n, "cuda")
        return A.cpu().numpy().T.copy().T  # column-major host copy
    return synth.graded(n)


def workload_config(n, b, p, world=1):
    """The `config` object of the JSON line; identical in both arms."""
    return {"workload": f"rqrcp_graded_{n}x{n}_b{b}_p{p}", "m": n, "n": n, "b": b, "p": p,
            "sigma": "10^(-12 (i-1)/(n-1))", "omega_seed": 1,
            "l2": "inputs larger than L2 (2.1 GB matrix)", "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    n, b, p = args.n, args.b, args.p
    A = np.asfortranarray(host_matrix(n))
    for _ in range(args.warmup):
        cpu_sample(A, b, p, max(1, args.cpu_blocks // 2))
    rates, secs = [], []
    for _ in range(args.steps):
        r, dt = cpu_sample(A, b, p, max(1, args.cpu_blocks // 2))
        rates.append(r)
        secs.append(dt)
    value = statistics.mean(rates)
    full_s = flops_geqrf(n, n) / (value * 1e9)
    nb = max(1, args.cpu_blocks // 2)
    sample = (f"first {nb} blocks (b={b}) of the {n}x{n} factorization per step "
              f"({statistics.mean(secs):.2f} s measured per step), rate from their "
              f"algorithmic flops")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # a step is the bounded sample, timed; the whole factorization at the
        # same rate is an extrapolation, reported under its own name
        "ms_per_step": 1e3 * statistics.mean(secs),
        "sample_blocks_per_step": nb,
        "full_factorization_ms_extrapolated": 1e3 * full_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(n, b, p, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample, "threads": "numpy BLAS default (all host cores)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measured_peaks():
    """MEASURED_PEAKS.json as a dict ({} when absent)."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def probe_peaks(dev, kinds=("fp64_fma", "fp64_fma_outer", "fp64_dmma_m8n8k4", "fp64_dmma_m16n8k16"),
                target_ms=60.0, reps=3):
    """Measured arithmetic peaks of this GPU (rqrcp_peak_probe): per kind the
    best TFLOP/s of `reps` launches of about `target_ms` each, with 4 CTAs of
    256 threads per SM."""
    import torch
    import paper_1509_06820_gb300 as rq
    grid = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    for kind in kinds:
        iters = 64
        ms, fl = rq.peak_probe(kind, iters, grid, dev)
        for _ in range(3):   # scale the launch to about target_ms
            iters = max(64, int(iters * target_ms / max(ms, 1e-3)))
            ms, fl = rq.peak_probe(kind, iters, grid, dev)
        best = 0.0
        for _ in range(reps):
            ms, fl = rq.peak_probe(kind, iters, grid, dev)
            best = max(best, fl / (ms / 1e3) / 1e12)
        out[kind] = {"tflops": best, "ms": ms, "iters": iters, "grid": grid}
    return out


# ------------------------------------------------------------------ extra legs
def mixed_leg(args, dev, fp64_ms, stream):
    """Mixed-precision RQRCP on a 16384^2 FP32 matrix N(0,1) + 1e3 x rank-512
    spike, b = 128, p = 16: time, speedup over the FP64 step, and the
    reconstruction error on sampled columns (checked in FP64 with torch)."""
    import torch
    import paper_1509_06820_gb300 as rq
    import synth
    n, b, p = args.n, 128, 16
    A0 = synth.spiked_device(n, n, dev).float()
    A0 = rq.colmajor(A0)
    A = rq.empty_colmajor(n, n, dev, torch.float32)
    h = rq.Handle(dev)
    h.reserve("M", n, n, n, b, p)

    def step():
        A.t().copy_(A0.t())
        return rq.rqrcp_factor_mixed(A, b, p, 1, handle=h)
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    h.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        jpvt, tau, rdiag = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    prof = h.profile_read()
    h.profile(False)
    info = h.sync_info()
    # sampled-column reconstruction: A(:, jpvt[c]) vs Q R(:, c), Q applied in FP64
    g = torch.Generator().manual_seed(5)
    cols = torch.randperm(n, generator=g)[:8].to(dev)
    V = A.double()
    k = n
    rows = torch.arange(n, device=dev)[:, None]
    X = V[:, cols] * (rows <= cols[None, :])          # R(:, c): rows 0..c
    X[cols, torch.arange(8, device=dev)] = rdiag[cols]
    for i in range(k - 1, -1, -1):
        v = V[i:, i].clone()
        v[0] = 1.0
        X[i:] -= tau[i] * torch.outer(v, v @ X[i:])
    ref = A0[:, jpvt[cols]].double()
    err = ((ref - X).norm(dim=0) / ref.norm(dim=0)).max().item()
    tr_ms, tr_fl, tr_l = prof["trailing_update"]
    del A, A0, V, X
    return {"workload": f"rqrcp_mixed_spiked_{n}x{n}_b{b}_p{p}", "ms_per_step": ms,
            "gflops": flops_geqrf(n, n) / (ms / 1e3) / 1e9, "speedup_vs_f64": fp64_ms / ms,
            "recon_err_sampled_cols": err, "device_info": info,
            "trailing_update": {"ms": tr_ms, "bf16_tflops": 6 * tr_fl / (tr_ms / 1e3) / 1e12,
                                "tf32_equiv_tflops": tr_fl / (tr_ms / 1e3) / 1e12},
            "phases": {kk: {"ms": v[0], "launches": v[2]} for kk, v in prof.items()}}


def emulated_leg(args, dev, A0, fp64_ms, qr_ms, stream):
    """The same FP64 factorization with the trailing update on the BF16
    tensor cores (FP64-accurate slicing, rqrcp_set_option), and the same for
    the unpivoted QR."""
    import torch
    import paper_1509_06820_gb300 as rq
    n, b, p = args.n, args.b, args.p
    h = rq.Handle(dev)
    h.set_fp64_emulation(True)
    h.reserve("R", n, n, n, b, p)
    A = rq.empty_colmajor(n, n, dev)
    out = {}
    for name, call in (("rqrcp", lambda: rq.rqrcp_factor(A, b, p, 1, handle=h)),
                       ("qr", lambda: rq.qr_factor(A, b, handle=h))):
        for _ in range(max(1, args.warmup)):
            A.copy_(A0)
            call()
        torch.cuda.synchronize(dev)
        h.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            A.copy_(A0)
            call()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        prof = h.profile_read()
        h.profile(False)
        tr_ms, tr_fl, tr_l = prof["trailing_update"]
        out[name] = {"ms_per_step": ms, "gflops": flops_geqrf(n, n) / (ms / 1e3) / 1e9,
                     "trailing_update_fp64_equiv_tflops": tr_fl / (tr_ms / 1e3) / 1e12,
                     "trailing_update_bf16_tflops": 28 * tr_fl / (tr_ms / 1e3) / 1e12,
                     "phases": {k: round(v[0] / args.steps, 2) for k, v in prof.items()}}
    out["device_info"] = h.sync_info()
    out["rqrcp_over_qr_time"] = out["rqrcp"]["ms_per_step"] / out["qr"]["ms_per_step"]
    out["speedup_vs_fp64_pipe"] = fp64_ms / out["rqrcp"]["ms_per_step"]
    out["note"] = ("28 BF16 slice products per FP64 multiply-add, exact per-diagonal FP32 sums, "
                   "double-FP32 running sums; parity vs the FP64 oracle in tests")
    h.close()
    del A
    return out


def rsrqrcp_leg(args, dev, A0, fp64_ms, emul_ms, stream):
    """Alg. 5 (RSRQRCP: a fresh sample of the trailing matrix every block
    instead of the sample update of Eq. 3) on the same matrix and (b, p):
    the cost of repeated sampling, with the FP64 pipe and with the
    FP64-emulated products."""
    import torch
    import paper_1509_06820_gb300 as rq
    n, b, p = args.n, args.b, args.p
    A = rq.empty_colmajor(n, n, dev)
    out = {"workload": f"rsrqrcp_graded_{n}x{n}_b{b}_p{p}"}
    for emul in (False, True):
        h = rq.Handle(dev)
        h.set_resample(True)
        h.set_fp64_emulation(emul)
        h.reserve("R", n, n, n, b, p)

        def step():
            A.copy_(A0)
            rq.rqrcp_factor(A, b, p, 1, handle=h)
        step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        ref = emul_ms if emul else fp64_ms
        out["emulated" if emul else "fp64"] = {
            "ms_per_step": ms, "over_rqrcp_time": ms / ref if ref else None,
            "device_info": h.sync_info()}
        h.close()
    out["paper_ratio_16k"] = 43.84 / 24.03
    del A
    return out


def qrcp_leg(args, dev, A0, fp64_ms, stream):
    """Deterministic QRCP with level-3 reflection blocking (the paper's
    comparison method) on the same matrix: what the sample saves.  The
    block kernels (one pass over the trailing matrix per pivot) and the
    delayed block updates are timed separately with the handle's events."""
    import torch
    import paper_1509_06820_gb300 as rq
    n, b = args.n, args.b
    A = rq.empty_colmajor(n, n, dev)
    h = rq.Handle(dev)
    h.reserve("P", n, n, n, b, 0)
    # warm-up on a small leading block (kernel attributes, handle scratch)
    Aw = rq.colmajor(A0[:1024, :1024].clone())
    rq.qrcp_factor(Aw, b, handle=h)
    del Aw
    A.copy_(A0)
    torch.cuda.synchronize(dev)
    h.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rq.qrcp_factor(A, b, handle=h)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    prof = h.profile_read()
    h.profile(False)
    # level-2 pass: column j reads rows j.. of the n - i0 - 1 other columns of
    # its block and trailing matrix; summed as 8 (n - j)^2 bytes per pivot
    l2_bytes = sum(8.0 * (n - j) * (n - j) for j in range(n))
    blk_ms = prof["panel"][0]
    out = {
        "workload": f"qrcp_graded_{n}x{n}_b{b}",
        "ms_per_step": ms, "gflops": 4.0 / 3.0 * n ** 3 / ms / 1e6,
        "over_rqrcp_time": ms / fp64_ms if fp64_ms else None,
        "block_kernels_ms": blk_ms, "block_launches": prof["panel"][2],
        "level2_pass_gbs": l2_bytes / (blk_ms * 1e-3) / 1e9 if blk_ms else None,
        "trailing_update_ms": prof["trailing_update"][0],
        "device_info": h.sync_info(),
        "paper_ratio_16k": 176.2 / 24.03,
    }
    h.close()
    del A
    return out


def _quality_matrices(n, dev):
    """Two seeded n x n test matrices for the error-vs-rank curves, with their
    singular values: 'graded' (singular values 10^(-12 (i-1)/(n-1)), Haar
    factors) and 'collinear_block' (n/2 columns of norm ~1 drawn from a 5-dim
    subspace plus 1e-8 noise, then n/2 columns of a rank-n/2 matrix with
    singular values 0.3 / i: presorting by norm takes every collinear column
    first, which is where unpivoted QR fails to reveal rank)."""
    import torch
    import synth
    g = torch.Generator(device="cpu").manual_seed(21)
    out = {}
    A = torch.from_numpy(synth.graded(n)).to(dev)
    out["graded"] = A
    h = n // 2
    C = torch.randn(n, 5, generator=g, dtype=torch.float64) @ torch.randn(5, h, generator=g,
                                                                          dtype=torch.float64)
    C = C / C.norm(dim=0, keepdim=True) + 1e-8 * torch.randn(n, h, generator=g,
                                                               dtype=torch.float64)
    U = torch.linalg.qr(torch.randn(n, h, generator=g, dtype=torch.float64))[0]
    V = torch.linalg.qr(torch.randn(h, h, generator=g, dtype=torch.float64))[0]
    D = (U * (0.3 / torch.arange(1, h + 1, dtype=torch.float64))) @ V.T
    out["collinear_block"] = torch.cat([C, D], dim=1).to(dev)
    return out


def quality_leg(args, dev):
    """Error-vs-rank curves (relative Frobenius error of the rank-k
    approximation) for QR after presorting the columns by norm, RQRCP,
    RSRQRCP, deterministic QRCP, TUXV and the SVD, on synthetic stand-ins for
    the paper's test matrices, plus the expected norm of the sample-selected
    column (Fig. selectExpect) measured over seeds against its exact value."""
    import numpy as np
    import torch
    import paper_1509_06820_gb300 as rq
    n, b, p = 2000, 32, 8
    ranks = [10, 50, 100, 200, 400, 800]
    res = {"n": n, "b": b, "p": p, "ranks": ranks}

    def tail_err(R, nrm):
        r2 = (torch.triu(R[: min(R.shape)]) ** 2).sum(dim=1)
        suf = torch.flip(torch.cumsum(torch.flip(r2, [0]), 0), [0])
        return [float(torch.sqrt(suf[k]) / nrm) if k < len(suf) else 0.0 for k in ranks]

    for name, A in _quality_matrices(n, dev).items():
        nrm = torch.linalg.norm(A)
        curves = {}
        order = torch.argsort(A.norm(dim=0), descending=True)
        F = rq.colmajor(A[:, order].clone())
        rq.qr_factor(F, b)
        curves["qr_presorted"] = tail_err(F, nrm)
        for label, resample in (("rqrcp", False), ("rsrqrcp", True)):
            h = rq.Handle(dev)
            h.set_resample(resample)
            F = rq.colmajor(A.clone())
            rq.rqrcp_factor(F, b, p, 1, handle=h)
            curves[label] = tail_err(F, nrm)
            h.close()
        F = rq.colmajor(A.clone())
        rq.qrcp_factor(F, b)
        curves["qrcp"] = tail_err(F, nrm)
        tux = []
        for k in ranks:
            U, X, V = rq.tuxv(rq.colmajor(A.clone()), k, b, p, 1)
            tux.append(float(torch.linalg.norm(A - U @ X @ V.T) / nrm))
        curves["tuxv"] = tux
        s = torch.linalg.svdvals(A)
        suf = torch.sqrt(torch.flip(torch.cumsum(torch.flip(s ** 2, [0]), 0), [0]))
        curves["svd"] = [float(suf[k] / nrm) for k in ranks]
        res[name] = curves
    # Fig. selectExpect: first sample pivot over seeds, orthogonal columns phi^j;
    # exact values stored by tests/golden/gen_select_expectation.py
    with open(os.path.join(ROOT, "tests", "golden", "select_expectation.json")) as f:
        exact = {(c["phi"], c["ell"], c["n"]): c["exact"] for c in json.load(f)["cases"]}
    sel = []
    m, nc, trials = 96, 32, 2000
    g = torch.Generator().manual_seed(17)
    Q = torch.linalg.qr(torch.randn((m, nc), generator=g, dtype=torch.float64))[0]
    for phi, ell in ((0.9, 8), (0.95, 8), (0.9, 16), (0.95, 16)):
        A = rq.colmajor((Q * phi ** torch.arange(nc, dtype=torch.float64)).to(dev))
        picks = [rq.sample_qrcp(rq.sketch(A, ell, seed), 1)[:1] for seed in range(1, trials + 1)]
        vals = phi ** torch.cat(picks).double().cpu().numpy()
        sel.append({"phi": phi, "ell": ell, "n": nc, "trials": trials,
                    "measured": float(vals.mean()),
                    "stderr": float(vals.std() / np.sqrt(trials)),
                    "exact": exact[(phi, ell, nc)]})
    res["select_expectation"] = sel
    return res


def truncated_leg(args, dev, fp64_peak):
    """TRQRCP and TUXV (FP64) at rank 512 on a 50000 x 20000 matrix
    U_r diag(i^-2) V_r^T (rank 2048) + N(0, 1e-8^2), b = 64, p = 8; FP64
    fractions against `fp64_peak` (TFLOP/s), the headline's unit-count peak."""
    import torch
    import paper_1509_06820_gb300 as rq
    import synth
    m, n, k, b, p = 50000, 20000, 512, 64, 8
    A = rq.colmajor(synth.decaying_lowrank_device(m, n, dev, rank=2048, noise=1e-8))
    h = rq.Handle(dev)
    h.reserve("U", m, n, k, b, p)
    ell = b + p
    out = {}
    for name, fn, extra in (("trqrcp", lambda: rq.trqrcp(A, k, b, p, 1, handle=h), 0.0),
                            ("tuxv", lambda: rq.tuxv(A, k, b, p, 1, handle=h), 2.0 * m * n * k)):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        steps = max(1, min(args.steps, 2))
        for _ in range(steps):
            res = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        fl = 2.0 * m * n * k + 2.0 * ell * m * n + extra
        # fewest HBM bytes: A read once by the sketch, once per block by
        # Y2^T A (k / b blocks), and once more by Z1 = A V1 for TUXV
        passes = 1 + k // b + (1 if extra else 0)
        hbm_bytes = passes * 8.0 * m * n
        peaks = measured_peaks()
        out[name] = {"ms": ms, "gflops": fl / (ms / 1e3) / 1e9, "flop_count": "2mnk + 2lmn (+2mnk)",
                     "roofline": {"fp64_frac": fl / (ms / 1e3) / 1e12 / fp64_peak,
                                  "hbm_frac": hbm_bytes / (ms / 1e3) / 1e9
                                  / (peaks.get("hbm_gbs") or 6800.0),
                                  "hbm_min_bytes": hbm_bytes,
                                  "peaks": f"FP64 = unit-count peak {fp64_peak:.4f} TFLOP/s "
                                           "(probes x sampled clock, as the headline); "
                                           "HBM measured copy"}}
    info = h.sync_info()
    U, X, V = res
    # ||A - U X V^T||_F^2 = ||A||^2 - 2 <U^T A V, X> + ||X||^2 (U, V orthonormal)
    a2 = (A.double() ** 2).sum().item()
    UtAV = (U.t() @ A) @ V
    err2 = a2 - 2.0 * (UtAV * X).sum().item() + (X ** 2).sum().item()
    sig = torch.arange(1, 2049, dtype=torch.float64) ** -2.0
    tail = float((sig[k:] ** 2).sum() + (1e-8) ** 2 * m * n)
    out["tuxv_rel_err"] = (max(err2, 0.0) / a2) ** 0.5
    out["optimum_rel_err_approx"] = (tail / a2) ** 0.5
    out["orth_U"] = (U.t() @ U - torch.eye(k, device=dev, dtype=torch.float64)).abs().max().item()
    out["device_info"] = info
    out["workload"] = f"trqrcp_tuxv_{m}x{n}_k{k}_b{b}_p{p}_decay2_noise1e-8"
    del A, U, X, V, UtAV
    h.close()
    torch.cuda.empty_cache()
    return out


SERVE_BUCKETS = [(1024, 1024, 64), (2048, 2048, 96), (4096, 4096, 128), (2048, 4096, 32),
                 (512, 512, 32)]


def tune_serving(dev, teams=(8, 16), reserve_sms=16, nprob=48):
    """Autotuning of the persistent kernel for the served workload: for each
    team size (CTAs per team, the launch's tile shape) the (b, p) table per
    size bucket, then the team size whose teams serve a batch of served-size
    problems fastest with the SMs a server leaves free for inputs."""
    import torch
    from paper_1509_06820_gb300.autotune import Tuner
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    best, tried = None, {}
    for team in teams:
        cands = [(16, 8), (32, 8), (64, 8)] if team >= 16 else [(16, 8), (32, 8)]
        tuner = Tuner.tune_batched(SERVE_BUCKETS, device=dev, team=team, candidates=cands)
        nteams = max(1, (nsm - reserve_sms) // team)
        res = batched_leg(dev, tuner, nprob=nprob, reps=3, seed=11, team=team, teams=nteams)
        tried[team] = round(res["problems_per_s"], 1)
        if best is None or res["problems_per_s"] > best[2]:
            best = (team, tuner, res["problems_per_s"])
    return best[0], best[1], tried


def ring_serving(args, dev, team=None, tuner=None):
    """The served TRQRCP workload on the persistent kernel's request ring:
    Poisson arrivals at --serve-rate, then a rate below saturation."""
    from paper_1509_06820_gb300.serve import RingServer
    from paper_1509_06820_gb300.autotune import Tuner
    t0 = time.perf_counter()
    tried = None
    if team is None:
        team, tuner, tried = tune_serving(dev)
    elif tuner is None:
        cands = [(16, 8), (32, 8), (64, 8)] if team >= 16 else [(16, 8), (32, 8)]
        tuner = Tuner.tune_batched(SERVE_BUCKETS, device=dev, team=team, candidates=cands)
    tune_s = time.perf_counter() - t0
    bmax = max(v["b"] for v in tuner.table.values())
    pmax = max(v["p"] for v in tuner.table.values())
    srv = RingServer(dev, team=team, tuner=tuner, max_b=bmax, max_p=pmax, capacity=1024)
    try:
        stats = srv.run_poisson(rate=args.serve_rate, duration=args.serve_seconds, warmup=2.0,
                                seed=7)
        low = srv.run_poisson(rate=args.serve_rate / 5, duration=min(5.0, args.serve_seconds),
                              warmup=0.5, seed=8)
    finally:
        srv.close()
    stats = {"mode": "persistent kernel, mapped request ring", "team_ctas": team,
             "teams": srv.nslots, **stats}
    if tried is not None:
        stats["autotune_team_problems_per_s"] = tried
    stats["below_saturation"] = {k: low[k] for k in ("offered_rate", "requests", "throughput_rps",
                                                     "p50_ms", "p99_ms", "gflops")}
    stats["autotune_s"] = tune_s
    stats["autotune_table"] = tuner.table
    return stats


def serving_leg(args, dev):
    """Served TRQRCP: Poisson arrivals, m, n ~ U{256..4096}, k ~ U{16..128},
    A = X Y^T (FP32).  Primary: the persistent kernel fed through the mapped
    request ring (teams of 8 CTAs, SMs left free for the inputs), autotuned
    b/p.  Beside it: the stream-slot server (16 slots, eager trqrcp_mixed
    launches per request, each capped at a quarter of the SMs) on the same
    stream, and one static batch through trqrcp_batched."""
    from paper_1509_06820_gb300.serve import Server
    from paper_1509_06820_gb300.autotune import Tuner
    stats = ring_serving(args, dev)
    t0 = time.perf_counter()
    tuner = Tuner.tune(SERVE_BUCKETS[:4], device=dev)
    tune_s = time.perf_counter() - t0
    srv = Server.on_gpu(dev, slots=16, tuner=tuner, use_graphs=False)
    sl = srv.run_poisson(rate=args.serve_rate, duration=args.serve_seconds, warmup=1.0, seed=7)
    stats["stream_slots"] = {"mode": "16 stream slots, eager trqrcp_mixed per request",
                             "autotune_s": tune_s,
                             **{k: sl[k] for k in ("offered_rate", "requests", "throughput_rps",
                                                   "p50_ms", "p99_ms", "gflops")}}
    del srv
    stats["batched"] = batched_leg(dev, Tuner(stats["autotune_table"]), team=stats["team_ctas"])
    return stats


def batched_specs(tuner, nprob, seed):
    """Served-size problems: m, n ~ U{256..4096}, k ~ U{16..128}, autotuned b/p."""
    import numpy as np
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(nprob):
        m, n = int(rng.integers(256, 4097)), int(rng.integers(256, 4097))
        k = int(min(rng.integers(16, 129), m, n))
        b, p = tuner.choose(m, n, k)
        specs.append((m, n, k, min(b, k), p))
    return specs


class FixedBP:
    """(b, p) for every problem (the kernel case's stand-in for the autotuner)."""

    def __init__(self, b, p):
        self.b, self.p = b, p

    def choose(self, m, n, k):
        return self.b, self.p


def batched_leg(dev, tuner, nprob=64, reps=5, seed=9, team=16, teams=0):
    """One static batch of served-size problems (m, n ~ U{256..4096},
    k ~ U{16..128}, A = X Y^T in FP32, autotuned b/p) through trqrcp_batched:
    one persistent launch (teams of CTAs claim the problems longest-first),
    captured as one CUDA graph and replayed."""
    import torch
    import paper_1509_06820_gb300 as rq
    from paper_1509_06820_gb300.serve import request_flops
    specs = batched_specs(tuner, nprob, seed)
    g = torch.Generator(device=dev)
    probs = []
    for i, (m, n, k, b, p) in enumerate(specs):
        g.manual_seed(1000 + i)
        X = torch.randn((m, k), generator=g, device=dev)
        Yf = torch.randn((n, k), generator=g, device=dev)
        probs.append((rq.colmajor(X @ Yf.t()), k, b, p, 1000 + i))
    h = rq.Handle(dev)
    h.set_batch_team(team)
    h.reserve_batched(0, max(s[0] for s in specs), max(s[1] for s in specs),
                      max(s[2] for s in specs), max(s[3] for s in specs),
                      max(s[4] for s in specs))
    outs = rq.trqrcp_batched(probs, teams=teams, handle=h)
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rq.trqrcp_batched(probs, teams=teams, handle=h, outs=outs)
    graph.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    # one eager launch with the kernel's phase timers on (team-milliseconds)
    h.profile(True)
    rq.trqrcp_batched(probs, teams=teams, handle=h, outs=outs)
    team_ms = {k: round(v, 2) for k, v in h.batched_profile().items() if v > 0}
    h.profile(False)
    flops = sum(request_flops(m, n, k, b + p) for (m, n, k, b, p) in specs)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    return {"problems": nprob, "team_ctas": team, "teams": teams or nsm // team, "ms_per_batch": ms,
            "phase_team_ms": team_ms,
            "problems_per_s": nprob / (ms / 1e3), "gflops": flops / (ms / 1e3) / 1e9,
            "launch": "one persistent cooperative launch per batch, captured in a CUDA graph",
            "device_info": h.sync_info()}


# ------------------------------------------------------------------ kernel cases
def run_case(args):
    """One small kernel case for profiling (prints one JSON line):
      panel       qr_factor of an m x 4b N(0,1) matrix (four b-column panels)
      gemm_bf16x  C = -op(A) op(B) + C, split-BF16 x3 (FP32 operands)
      gemm_f64x   the same in FP64 on the tensor cores (exact slices)
      qrcp        qrcp_factor of an n x n N(0,1) matrix, block b
      sample      the sample QRCP kernel alone: b pivots on a (b + p) x n
                  N(0,1) sample
      mixed       rqrcp_factor_mixed of the n x n spiked FP32 matrix (the
                  mixed-precision configuration), block b, oversampling p
      batched     one persistent trqrcp_batched launch over 64 served-size
                  problems (--reps sets the count, --b/--p the block and
                  oversampling), graph-replayed, with its phase timers
      fp64peak    the arithmetic-peak probes (FP64 FMA, FP64 DMMA m8n8k4 and
                  m16n8k16, FP32 FMA) with the SM clock sampled meanwhile
    Two untimed runs precede the timed ones."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1509_06820_gb300 as rq
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.case == "serve":
        # the ring server alone at --serve-rate for --serve-seconds
        team = args.team if args.team > 0 else None
        print(json.dumps({"case": "serve", **ring_serving(args, dev, team)}), flush=True)
        return
    if args.case == "batched":
        # one persistent batched launch over served-size problems (b = 64, p = 8)
        res = batched_leg(dev, FixedBP(args.b, args.p), nprob=args.reps if args.reps > 1 else 64,
                          team=args.team)
        res.update({"b": args.b, "p": args.p})
        print(json.dumps({"case": "batched", **res}), flush=True)
        return
    if args.case == "fp64peak":
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        res = probe_peaks(dev, kinds=("fp64_fma", "fp64_fma_outer", "fp64_dmma_m8n8k4",
                                      "fp64_dmma_m16n8k16", "fp32_fma"), target_ms=200.0, reps=5)
        clk = clocks.stop()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clk.get("sm_mhz") or 2070.0
        for v in res.values():
            v["flop_per_clk_per_sm"] = v["tflops"] * 1e12 / (sms * mhz * 1e6)
        print(json.dumps({"case": "fp64peak", "sms": sms, "probes": res, "clocks": clk}),
              flush=True)
        return
    g = torch.Generator(device=dev).manual_seed(1)
    h = rq.Handle(dev)
    if args.max_sms:
        h.set_max_sms(args.max_sms)
    out = {"case": args.case, "max_sms": args.max_sms}
    if args.case == "mixed":
        import synth
        n = args.n
        A0 = rq.colmajor(synth.spiked_device(n, n, dev).float())
        A = rq.empty_colmajor(n, n, dev, torch.float32)

        def call():
            A.t().copy_(A0.t())
            rq.rqrcp_factor_mixed(A, args.b, args.p, 1, handle=h)
        out.update({"n": n, "b": args.b, "p": args.p})
    elif args.case in ("rqrcp", "qr"):
        import synth
        n = args.n
        if args.emulated:
            h.set_fp64_emulation(True)
        A0 = synth.graded_device(n, dev)
        A = rq.empty_colmajor(n, n, dev)

        def call():
            A.t().copy_(A0.t())
            if args.case == "rqrcp":
                rq.rqrcp_factor(A, args.b, args.p, 1, handle=h)
            else:
                rq.qr_factor(A, args.b, handle=h)
        out.update({"n": n, "b": args.b, "p": args.p, "emulated": args.emulated})
    elif args.case == "sample":
        ell, n = args.b + args.p, args.n
        B0 = rq.colmajor(torch.randn((ell, n), generator=g, device=dev, dtype=torch.float64))
        B = rq.empty_colmajor(ell, n, dev)

        def call():
            B.copy_(B0)
            rq.sample_qrcp(B, args.b, handle=h)
        out.update({"ell": ell, "n": n, "steps": args.b})
    elif args.case in ("panel", "qrcp"):
        if args.case == "panel":
            m, n = args.m, 4 * args.b
        else:
            m = n = args.n
        A0 = rq.colmajor(torch.randn((m, n), generator=g, device=dev, dtype=torch.float64))
        A = rq.empty_colmajor(m, n, dev)

        def call():
            A.copy_(A0)
            if args.case == "panel":
                rq.qr_factor(A, args.b, handle=h)
            else:
                rq.qrcp_factor(A, args.b, handle=h)
        out.update({"m": m, "n": n, "b": args.b})
    else:
        ta, tb, M, N, K = args.shape.split(",")
        M, N, K = int(M), int(N), int(K)
        dt = torch.float32 if args.case == "gemm_bf16x" else torch.float64

        def colm(r, c):
            return rq.colmajor(torch.randn((r, c), generator=g, device=dev, dtype=dt))
        Am = colm(M, K) if ta == "N" else colm(K, M)
        Bm = colm(K, N) if tb == "N" else colm(N, K)
        C = colm(M, N)
        fn = rq.gemm_bf16x if args.case == "gemm_bf16x" else rq.gemm_f64x

        def call():
            fn(Am, Bm, ta, tb, alpha=-1.0, beta=1.0, C=C, handle=h)
        out.update({"transA": ta, "transB": tb, "M": M, "N": N, "K": K})
    for _ in range(2):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.profile(True)
    e0.record()
    for _ in range(args.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    out["ms_per_call"] = e0.elapsed_time(e1) / args.reps
    prof = h.profile_read()
    out["phases_ms"] = {k: round(v[0] / args.reps, 4) for k, v in prof.items() if v[2]}
    out["launches_per_call"] = sum(v[2] for v in prof.values()) // args.reps
    h.profile(False)
    out["device_info"] = h.sync_info()
    print(json.dumps(out), flush=True)


def summary_of(line, extras):
    """The metric's own comparisons in a few numbers (the last key of the line)."""
    def r(x, nd=4):
        return None if x is None else round(x, nd)
    out = {"rqrcp_ms": r(line["ms_per_step"], 1), "rqrcp_gflops": r(line["value"], 1),
           "qr_ms": r(extras.get("qr_ms_per_step"), 1),
           "rqrcp_over_qr_time": r(extras.get("rqrcp_over_qr_time"))}
    em = extras.get("fp64_emulated") or {}
    if em:
        out["fp64_emulated"] = {"rqrcp_ms": r(em.get("rqrcp", {}).get("ms_per_step"), 1),
                                "qr_ms": r(em.get("qr", {}).get("ms_per_step"), 1),
                                "rqrcp_over_qr_time": r(em.get("rqrcp_over_qr_time")),
                                "speedup_vs_fp64": r(em.get("speedup_vs_fp64_pipe"), 2)}
    mx = extras.get("mixed") or {}
    if mx:
        out["mixed"] = {"ms": r(mx.get("ms_per_step"), 1),
                        "speedup_vs_fp64": r(mx.get("speedup_vs_f64"), 2),
                        "recon_err": mx.get("recon_err_sampled_cols")}
    sv = extras.get("serving") or {}
    if sv:
        out["serving"] = {"offered_rps": sv.get("offered_rate"),
                          "rps": r(sv.get("throughput_rps"), 1), "p50_ms": r(sv.get("p50_ms"), 2),
                          "p99_ms": r(sv.get("p99_ms"), 2)}
    e2e = extras.get("e2e") or {}
    if e2e:
        out["e2e_gflops"] = r(e2e.get("value"), 1)
    return out


# ------------------------------------------------------------------ replicas
def max_over_ranks(x, world, device):
    """The largest of the ranks' values of x: the job's time is its slowest
    replica's (no collective touches the data path; this one reduces a
    timing)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(flops_per_rank, ms, world):
    """Whole-job GFLOP/s: every replica factors its own matrix in the job's
    time `ms` (the max over ranks)."""
    return world * flops_per_rank / (ms / 1e3) / 1e9


# ------------------------------------------------------------------ GPU leg
def main():
    args = parse()
    if args.case is not None:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1509_06820_gb300 as rq
    import synth

    n, b, p = args.n, args.b, args.p
    m = n
    A0 = synth.graded_device(n, dev)                 # column-major, resident
    A = rq.empty_colmajor(m, n, dev)
    h = rq.Handle(dev)
    stream = torch.cuda.current_stream(dev)
    h.reserve("R", m, n, n, b, p)
    h.reserve("Q", m, n, n, b, 0)

    def barrier():
        if world > 1:
            dist.barrier()

    def step():
        A.copy_(A0)
        rq.rqrcp_factor(A, b, p, 1, handle=h)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    info_warm = h.sync_info()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    h.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof = h.profile_read()
    h.profile(False)
    info = h.sync_info()
    ms = max_over_ranks(ms, world, dev)
    fl = flops_geqrf(m, n)
    value = job_rate(fl, ms, world)
    gpu_launches = sum(v[2] for v in prof.values())

    peaks = measured_peaks()
    # the FP64 rate of this GPU, measured now by the library's peak probes:
    # FMA chains on the CUDA cores and DMMA (mma.sync) on the tensor cores;
    # the roofline peak is the faster of the two
    probes = probe_peaks(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    tr_ms, tr_fl, tr_launch = prof["trailing_update"]
    achieved = tr_fl / (tr_ms / 1e3) / 1e12 if tr_ms > 0 else None
    # DRAM traffic of the trailing update: its algorithmic bytes (A2 read by
    # Z = Y^T A2, read and written by A2 -= Y W) times the ratio of measured to
    # algorithmic DRAM bytes of the same three kernels in an ncu capture on a
    # 6144^2 factorization (837.8 MB / 890.2 MB); traffic grows with m_J n2 as
    # the algorithmic bytes do.  Per launch, like `achieved`.
    alg_bytes = 0.0
    j0 = 0
    while j0 < min(m, n):
        bJ = min(b, min(m, n) - j0)
        alg_bytes += 24.0 * (m - j0) * (n - j0 - bJ)
        j0 += bJ
    traffic = 0.941 * alg_bytes / max(tr_launch, 1)
    best_kind = max(probes, key=lambda k: probes[k]["tflops"])
    best = probes[best_kind]["tflops"]
    # the FP64 unit count of an SM: the best probe (FMA chains, a GEMM's
    # outer-product pattern, DMMA m8n8k4 and m16n8k16, all within a few % of
    # one another) divided by SMs x clock x 2 flop, rounded to whole units;
    # peak = units x 2 flop x SMs x the SM clock sampled during the timed steps
    mhz = clk.get("sm_mhz") or 2070.0
    units = max(1, round(best * 1e12 / (2.0 * sms * mhz * 1e6)))
    peak = 2.0 * units * sms * mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": "trailing update (gemm_kernel FP64 FFMA)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch",
                "traffic_source": "algorithmic bytes x 0.941 (ncu DRAM bytes / algorithmic bytes, "
                                  "same kernels, 6144^2 factorization)",
                "peak_source": f"FP64 unit count x clock: {units} FP64 FMA/clk/SM (from the "
                               f"best of this run's probes, {best_kind} {best:.3f} TFLOP/s) x 2 "
                               f"flop x {sms} SMs x {mhz:.0f} MHz (sampled)",
                "peak_probes_tflops": {k: round(v["tflops"], 4) for k, v in probes.items()},
                "frac_of_best_probe": achieved / best if achieved else None,
                "peak_nominal": 1.25,
                "launch_ms_avg": tr_ms / max(tr_launch, 1)}
    phases = {k: {"ms": v[0], "gflop": v[1] / 1e9, "launches": v[2]} for k, v in prof.items()}

    extras = {}
    if "qr" in args.legs:
        # the project's own unpivoted blocked QR on the same matrix
        def qstep():
            A.copy_(A0)
            rq.qr_factor(A, b, handle=h)
        qstep()
        torch.cuda.synchronize(dev)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.steps):
            qstep()
        q1.record(stream)
        torch.cuda.synchronize(dev)
        qr_ms = q0.elapsed_time(q1) / args.steps
        extras["qr_ms_per_step"] = qr_ms
        extras["qr_gflops"] = fl / (qr_ms / 1e3) / 1e9
        extras["rqrcp_over_qr_time"] = ms / qr_ms

    if "e2e" in args.legs:
        # end to end through the public call with host buffers
        Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        Ah.copy_(A0)
        Ah_out = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        jh = torch.empty(n, dtype=torch.int64, pin_memory=True)
        th = torch.empty(min(m, n), dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize(dev)

        def estep():
            # the public host-buffer call: uploads in column chunks overlapped
            # with the sketch, downloads finished columns behind the blocks
            rq.rqrcp_factor_host(Ah, b, p, 1, dA=A, out=(Ah_out, jh, th), handle=h)
        estep()
        torch.cuda.synchronize(dev)
        barrier()
        x0 = torch.cuda.Event(enable_timing=True)
        x1 = torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        for _ in range(args.steps):
            estep()
        x1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = x0.elapsed_time(x1) / args.steps
        e2e_ms = max_over_ranks(e2e_ms, world, dev)
        extras["e2e"] = {"value": job_rate(fl, e2e_ms, world), "unit": UNIT,
                         "ms_per_step": e2e_ms, "h2d_bytes_per_step": m * n * 8,
                         "d2h_bytes_per_step": m * n * 8 + n * 8 + min(m, n) * 8}
        del Ah, Ah_out

    if "cpu" in args.legs and rank == 0:
        import numpy as np
        A_host = np.asfortranarray(A0.cpu().numpy())
        rate, dt = cpu_sample(A_host, b, p, args.cpu_blocks)
        extras["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"first {args.cpu_blocks} blocks (b={b}) of the same {n}x{n} "
                       f"factorization, {dt:.1f} s, rate from their algorithmic flops"),
            "threads": "numpy BLAS default (all host cores)"}

    if "emulated" in args.legs:
        extras["fp64_emulated"] = emulated_leg(args, dev, A0, ms, extras.get("qr_ms_per_step"),
                                               stream)
    if "rsrqrcp" in args.legs:
        em = extras.get("fp64_emulated", {}).get("rqrcp", {}).get("ms_per_step")
        extras["rsrqrcp"] = rsrqrcp_leg(args, dev, A0, ms, em, stream)
    if "qrcp" in args.legs:
        extras["qrcp"] = qrcp_leg(args, dev, A0, ms, stream)
    if "mixed" in args.legs:
        extras["mixed"] = mixed_leg(args, dev, ms, stream)
    if "quality" in args.legs and rank == 0:
        extras["quality"] = quality_leg(args, dev)
    if "truncated" in args.legs:
        extras["truncated"] = truncated_leg(args, dev, peak)
    if "serving" in args.legs and rank == 0:
        extras["serving"] = serving_leg(args, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n, b, p, world),
            "gpu_launches": gpu_launches,
            "device_info": info | info_warm,
            "phases": phases,
        }
        # the long per-leg records first; the headline figures close the line
        for k in ("truncated", "serving", "quality", "qrcp", "rsrqrcp", "fp64_emulated",
                  "mixed"):
            if k in extras:
                line[k] = extras[k]
        line["e2e"] = extras.get("e2e")
        line["cpu_baseline"] = extras.get("cpu_baseline")
        line["clocks"] = clk
        line["roofline"] = roofline
        line["summary"] = summary_of(line, extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
