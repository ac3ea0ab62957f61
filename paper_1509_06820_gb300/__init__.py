"""Python binding of librqrcp (randomized QR with column pivoting on GB300).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``csrc/`` behind the C ABI of ``include/rqrcp.h``.  PyTorch supplies device
memory and the current stream.  There is no CPU fallback: if the library
cannot be loaded the calls raise.

Matrices are column-major float64 CUDA tensors, i.e. tensors with
``stride(0) == 1`` (the transpose of a contiguous tensor); ``colmajor``
converts, ``empty_colmajor`` allocates.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librqrcp.so")

RQRCP_OK = 0
RQRCP_ERR_CUDA = 1000
RQRCP_ERR_ALLOC = 1001
RQRCP_ERR_UNSUPPORTED = 1002
RQRCP_ERR_BATCH = 1003
RQRCP_ERR_BUSY = 1004
OPT_FP64_EMULATION = 1
OPT_RESAMPLE = 2
OPT_MAX_SMS = 3
OPT_TEST_BARRIER_TIMEOUT = 4
OPT_BATCH_TEAM = 5
INFO_NONFINITE = 1
INFO_RESAMPLED = 2
INFO_TIMEOUT = 4
INFO_NOCONV = 8

# (name, restype, argtypes) of every symbol declared in include/rqrcp.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_U64 = ctypes.c_uint64


class Problem(ctypes.Structure):
    """struct rqrcp_problem (include/rqrcp.h): one trqrcp_batched problem."""
    _fields_ = [("m", _I64), ("n", _I64), ("k", _I64), ("b", _I), ("p", _I), ("seed", _U64),
                ("dA", _P), ("lda", _I64), ("d_jpvt", _P), ("d_tau", _P), ("dY", _P),
                ("ldy", _I64), ("dR", _P), ("ldr", _I64), ("d_rdiag", _P)]


SIGNATURES = [
    ("rqrcp_create", _I, [ctypes.POINTER(_P), _P]),
    ("rqrcp_destroy", _I, [_P]),
    ("rqrcp_set_stream", _I, [_P, _P]),
    ("rqrcp_workspace_bytes", ctypes.c_size_t, [ctypes.c_char, _I64, _I64, _I64, _I, _I]),
    ("rqrcp_reserve", _I, [_P, ctypes.c_char, _I64, _I64, _I64, _I, _I]),
    ("rqrcp_set_option", _I, [_P, _I, _I]),
    ("rqrcp_sync_info", _I, [_P, ctypes.POINTER(_I)]),
    ("rqrcp_last_error", ctypes.c_char_p, [_P]),
    ("rqrcp_status_string", ctypes.c_char_p, [_I]),
    ("rqrcp_factor", _I, [_P, _I64, _I64, _P, _I64, _I, _I, _U64, _P, _P]),
    ("qr_factor", _I, [_P, _I64, _I64, _P, _I64, _I, _P]),
    ("rqrcp_factor_mixed", _I, [_P, _I64, _I64, _P, _I64, _I, _I, _U64, _P, _P, _P]),
    ("trqrcp", _I, [_P, _I64, _I64, _P, _I64, _I64, _I, _I, _U64, _P, _P, _P, _I64, _P, _I64]),
    ("trqrcp_mixed", _I, [_P, _I64, _I64, _P, _I64, _I64, _I, _I, _U64, _P, _P, _P, _I64, _P, _I64,
                          _P]),
    ("trqrcp_batched", _I, [_P, _I, ctypes.POINTER(Problem), _I]),
    ("rqrcp_reserve_batched", _I, [_P, _I, _I64, _I64, _I64, _I, _I]),
    ("tuxv", _I, [_P, _I64, _I64, _P, _I64, _I64, _I, _I, _U64, _P, _I64, _P, _I64, _P, _I64]),
    ("tuxv_iter", _I, [_P, _I64, _I64, _P, _I64, _I64, _I, _I, _U64, _I, _P, _I64, _P, _I64, _P,
                       _I64]),
    ("rqrcp_factor_host", _I, [_P, _I64, _I64, _P, _I64, _P, _I64, _I, _I, _U64, _P, _I64, _P,
                               _P]),
    ("qrcp_factor", _I, [_P, _I64, _I64, _P, _I64, _I, _P, _P]),
    ("tuxv_svd", _I, [_P, _I64, _I64, _P, _I64, _I64, _I, _I, _U64, _I, _P, _I64, _P, _P, _I64]),
    ("rqrcp_gaussian", _I, [_P, _U64, ctypes.c_uint32, _I64, _I64, _P, _I64]),
    ("rqrcp_sketch", _I, [_P, _I64, _I64, _P, _I64, _I, _U64, _P, _I64]),
    ("rqrcp_gemm_bf16x", _I, [_P, ctypes.c_char, ctypes.c_char, _I64, _I64, _I64, ctypes.c_float,
                          _P, _I64, _P, _I64, ctypes.c_float, _P, _I64, _I]),
    ("rqrcp_gemm_f64x", _I, [_P, ctypes.c_char, ctypes.c_char, _I64, _I64, _I64, ctypes.c_double,
                         _P, _I64, _P, _I64, ctypes.c_double, _P, _I64]),
    ("rqrcp_sample_qrcp", _I, [_P, _I, _I64, _I, _P, _I64, _P]),
    ("rqrcp_sample_qrcp_noalloc", _I, [_I, _I64, _I, _P, _I64, _P, _P, _P]),
    ("rqrcp_server_start", _I, [_P, _I, _I, _I64, _I64, _I64, _I, _I]),
    ("rqrcp_server_submit", _I, [_P, ctypes.POINTER(Problem), ctypes.POINTER(_I64)]),
    ("rqrcp_server_poll", _I, [_P, _I64, ctypes.POINTER(_I)]),
    ("rqrcp_server_stop", _I, [_P]),
    ("rqrcp_peak_probe", _I, [_I, _I64, _I, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    ("rqrcp_profile", _I, [_P, _I]),
    ("rqrcp_batched_profile", _I, [_P, _I, _P]),
    ("rqrcp_profile_read", _I, [_P, _I, _P, _P, _P]),
]

PHASES = ["sketch", "sample_qrcp", "permute", "panel", "trailing_update", "sample_update",
          "trqrcp_products", "other"]

_lib = None


class RqrcpError(RuntimeError):
    pass


def load(path=None):
    """Load librqrcp.so (building it first is the job of ``build.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RqrcpError(f"librqrcp.so not found at {path}; run paper_1509_06820_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Handle:
    """Owns an rqrcp handle (scratch memory, status word) on one device."""

    def __init__(self, device=None):
        lib = load()
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            h = _P()
            _check(lib.rqrcp_create(ctypes.byref(h), None), None)
        self.h = h

    def bind(self, stream=None):
        stream = stream or torch.cuda.current_stream(self.device)
        load().rqrcp_set_stream(self.h, _P(stream.cuda_stream))
        return self.h

    def sync_info(self):
        info = _I(0)
        _check(load().rqrcp_sync_info(self.bind(), ctypes.byref(info)), self.h)
        return info.value

    def reserve(self, op, m, n, k, b, p):
        _check(load().rqrcp_reserve(self.bind(), op.encode(), m, n, k, b, p), self.h)

    def reserve_batched(self, teams, m, n, k, b, p):
        """Scratch of `teams` teams (0 = as many as the SM budget holds) of the
        persistent batched kernel for problems up to m x n, rank k, block b,
        oversampling p."""
        _check(load().rqrcp_reserve_batched(self.h, teams, m, n, k, b, p), self.h)

    def set_batch_team(self, ctas):
        """CTAs per team of the persistent batched kernel (8, 16 or 32)."""
        _check(load().rqrcp_set_option(self.h, OPT_BATCH_TEAM, ctas), self.h)

    def set_test_barrier_timeout(self, on=True):
        """Test of the failure path only: rqrcp_sample_qrcp on this handle runs
        with a grid barrier that cannot complete and gives up after a few ms."""
        _check(load().rqrcp_set_option(self.h, OPT_TEST_BARRIER_TIMEOUT, 1 if on else 0), self.h)

    def set_fp64_emulation(self, on=True):
        """Run the FP64 trailing update on the BF16 tensor cores (exact slicing)."""
        _check(load().rqrcp_set_option(self.h, OPT_FP64_EMULATION, 1 if on else 0), self.h)

    def set_max_sms(self, n):
        """Cap the CTAs per wave of this handle's launches at n SMs (0: all)."""
        _check(load().rqrcp_set_option(self.h, OPT_MAX_SMS, int(n)), self.h)

    def set_resample(self, on=True):
        """rqrcp_factor runs Alg. 5 (a fresh sample every block) instead of Eq. (3)."""
        _check(load().rqrcp_set_option(self.h, OPT_RESAMPLE, 1 if on else 0), self.h)

    def profile(self, enable=True):
        _check(load().rqrcp_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        """{phase: (ms, flops, launches)} since the last profile(True)."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        fl = (ctypes.c_double * n)()
        ln = (ctypes.c_int64 * n)()
        self.bind()
        _check(load().rqrcp_profile_read(self.h, n, ctypes.cast(ms, _P), ctypes.cast(fl, _P),
                                         ctypes.cast(ln, _P)), self.h)
        return {p: (ms[i], fl[i], ln[i]) for i, p in enumerate(PHASES)}

    def batched_profile(self):
        """Team-milliseconds per phase of the persistent batched kernel since
        profiling was enabled (summed over teams)."""
        ms = (ctypes.c_double * len(PHASES))()
        _check(load().rqrcp_batched_profile(self.h, len(PHASES), ms), self.h)
        return {name: ms[i] for i, name in enumerate(PHASES)}

    def close(self):
        if getattr(self, "h", None):
            load().rqrcp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles = {}


def default_handle(device=None):
    dev = torch.device(device or "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    if dev not in _handles:
        _handles[dev] = Handle(dev)
    return _handles[dev]


def _check(code, h):
    if code == RQRCP_OK:
        return
    lib = load()
    msg = lib.rqrcp_status_string(code).decode()
    if h is not None and code in (RQRCP_ERR_CUDA, RQRCP_ERR_ALLOC, RQRCP_ERR_BATCH):
        msg += ": " + lib.rqrcp_last_error(h).decode()
    if code < 0:
        msg = f"argument {-code} invalid"
    raise RqrcpError(f"rqrcp call failed ({code}): {msg}")


def _is_colmajor(x):
    if x.dim() != 2:
        return False
    rows, cols = x.shape
    ok_rows = rows <= 1 or x.stride(0) == 1
    ok_cols = cols <= 1 or x.stride(1) >= max(1, rows)
    return ok_rows and ok_cols


def _ld(x):
    rows, cols = x.shape
    return x.stride(1) if cols > 1 else max(1, rows)


def colmajor(x):
    """x itself if it is column-major, else a column-major copy."""
    if _is_colmajor(x):
        return x
    out = empty_colmajor(x.shape[0], x.shape[1], x.device, x.dtype)
    out.copy_(x)
    return out


def empty_colmajor(rows, cols, device, dtype=torch.float64):
    return torch.empty((cols, rows), device=device, dtype=dtype).t()


def _cm(x, name):
    if x.device.type != "cuda" or x.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if not _is_colmajor(x):
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return x.data_ptr(), _ld(x)


def _ptr(x):
    return _P(x.data_ptr())


def rqrcp_factor(A, b, p, seed, handle=None):
    """Alg. 4 in place on column-major A; returns (jpvt, tau)."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    jpvt = torch.empty(n, dtype=torch.int64, device=A.device)
    tau = torch.empty(min(m, n), dtype=torch.float64, device=A.device)
    _check(load().rqrcp_factor(h.bind(), m, n, _P(pa), lda, b, p, seed, _ptr(jpvt), _ptr(tau)), h.h)
    return jpvt, tau


def rqrcp_factor_mixed(A, b, p, seed, handle=None):
    """Mixed-precision Alg. 4 in place on a column-major float32 A;
    returns (jpvt, tau (float64), rdiag (float64))."""
    h = handle or default_handle(A.device)
    if A.device.type != "cuda" or A.dtype != torch.float32 or not _is_colmajor(A):
        raise ValueError("A must be a column-major float32 CUDA tensor")
    m, n = A.shape
    k = min(m, n)
    jpvt = torch.empty(n, dtype=torch.int64, device=A.device)
    tau = torch.empty(k, dtype=torch.float64, device=A.device)
    rdiag = torch.empty(k, dtype=torch.float64, device=A.device)
    _check(load().rqrcp_factor_mixed(h.bind(), m, n, _ptr(A), _ld(A), b, p, seed, _ptr(jpvt),
                                     _ptr(tau), _ptr(rdiag)), h.h)
    return jpvt, tau, rdiag


def qr_factor(A, b, handle=None):
    """Unpivoted blocked QR in place; returns tau."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    tau = torch.empty(min(m, n), dtype=torch.float64, device=A.device)
    _check(load().qr_factor(h.bind(), m, n, _P(pa), lda, b, _ptr(tau)), h.h)
    return tau


def rqrcp_factor_host(hA, b, p, seed, dA=None, out=None, handle=None):
    """rqrcp_factor of a column-major float64 matrix in (preferably pinned)
    host memory, copies overlapped with the factorization.  dA: device work
    matrix (allocated if None).  out: (F_host, jpvt_host, tau_host) buffers
    (allocated pinned if None; F may be hA).  Enqueued on the current stream;
    returns (F, jpvt, tau, dA), valid once that stream is synchronised."""
    if hA.device.type != "cpu" or hA.dtype != torch.float64 or not _is_colmajor(hA):
        raise ValueError("hA must be a column-major float64 host tensor")
    m, n = hA.shape
    dev = torch.device("cuda", torch.cuda.current_device())
    h = handle or default_handle(dev)
    if dA is None:
        dA = empty_colmajor(m, n, dev)
    pd, lda = _cm(dA, "dA")
    if out is None:
        F = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        jp = torch.empty(n, dtype=torch.int64, pin_memory=True)
        tau = torch.empty(min(m, n), dtype=torch.float64, pin_memory=True)
    else:
        F, jp, tau = out
    if F.device.type != "cpu" or not _is_colmajor(F) or jp.device.type != "cpu" \
            or tau.device.type != "cpu":
        raise ValueError("outputs must be host tensors (F column-major)")
    _check(load().rqrcp_factor_host(h.bind(), m, n, _P(hA.data_ptr()), _ld(hA), _P(pd), lda, b, p,
                                    seed, _P(F.data_ptr()), _ld(F), _P(jp.data_ptr()),
                                    _P(tau.data_ptr())), h.h)
    return F, jp, tau, dA


def qrcp_factor(A, b=64, handle=None):
    """Deterministic QRCP (level-3 reflection blocking) in place; returns
    (jpvt, tau).  Waits for the device once per block."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    jpvt = torch.empty(n, dtype=torch.int64, device=A.device)
    tau = torch.empty(min(m, n), dtype=torch.float64, device=A.device)
    _check(load().qrcp_factor(h.bind(), m, n, _P(pa), lda, b, _ptr(jpvt), _ptr(tau)), h.h)
    return jpvt, tau


def trqrcp(A, k, b, p, seed, handle=None):
    """Alg. 6; returns (jpvt, tau, Y (m x k), R (k x n, permuted order))."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    jpvt = torch.empty(n, dtype=torch.int64, device=A.device)
    tau = torch.empty(k, dtype=torch.float64, device=A.device)
    Y = empty_colmajor(m, k, A.device)
    R = empty_colmajor(k, n, A.device)
    _check(load().trqrcp(h.bind(), m, n, _P(pa), lda, k, b, p, seed, _ptr(jpvt), _ptr(tau),
                         _ptr(Y), _ld(Y), _ptr(R), _ld(R)), h.h)
    return jpvt, tau, Y, R


def trqrcp_mixed(A, k, b, p, seed, handle=None, out=None):
    """Mixed-precision Alg. 6 on a column-major float32 A; returns
    (jpvt, tau (f64), Y (f32, m x k), R (f32, k x n), rdiag (f64))."""
    h = handle or default_handle(A.device)
    if A.device.type != "cuda" or A.dtype != torch.float32 or not _is_colmajor(A):
        raise ValueError("A must be a column-major float32 CUDA tensor")
    m, n = A.shape
    if out is None:
        out = (torch.empty(n, dtype=torch.int64, device=A.device),
               torch.empty(k, dtype=torch.float64, device=A.device),
               empty_colmajor(m, k, A.device, torch.float32),
               empty_colmajor(k, n, A.device, torch.float32),
               torch.empty(k, dtype=torch.float64, device=A.device))
    jpvt, tau, Y, R, rdiag = out
    _check(load().trqrcp_mixed(h.bind(), m, n, _ptr(A), _ld(A), k, b, p, seed, _ptr(jpvt),
                               _ptr(tau), _ptr(Y), _ld(Y), _ptr(R), _ld(R), _ptr(rdiag)), h.h)
    return jpvt, tau, Y, R, rdiag


def problem_struct(A, k, b, p, seed, out):
    """The rqrcp_problem of one TRQRCP request: A (column-major float32 CUDA
    tensor), its rank, block, oversampling and seed, and its output tensors
    (jpvt, tau, Y, R, rdiag) laid out as trqrcp_mixed's."""
    m, n = A.shape
    jpvt, tau, Y, R, rdiag = out
    return Problem(m, n, k, b, p, seed, _ptr(A), _ld(A), _ptr(jpvt), _ptr(tau), _ptr(Y), _ld(Y),
                   _ptr(R), _ld(R), _ptr(rdiag))


def trqrcp_outputs(m, n, k, device):
    """Output tensors (jpvt, tau, Y, R, rdiag) of a rank-k TRQRCP request."""
    return (torch.empty(n, dtype=torch.int64, device=device),
            torch.empty(k, dtype=torch.float64, device=device),
            empty_colmajor(m, k, device, torch.float32),
            empty_colmajor(k, n, device, torch.float32),
            torch.empty(k, dtype=torch.float64, device=device))


def trqrcp_batched(problems, teams=0, handle=None, outs=None):
    """Alg. 6 in mixed precision on many matrices in one persistent launch.
    `problems` is a list of (A, k, b, p, seed) with A a column-major float32
    CUDA tensor; returns one (jpvt, tau, Y, R, rdiag) tuple per problem, laid
    out as trqrcp_mixed's.  teams: concurrent problems (0 = as many as fit)."""
    if not problems:
        return []
    dev = problems[0][0].device
    h = handle or default_handle(dev)
    arr = (Problem * len(problems))()
    results = []
    for i, (A, k, b, p, seed) in enumerate(problems):
        if A.device.type != "cuda" or A.dtype != torch.float32 or not _is_colmajor(A):
            raise ValueError("A must be a column-major float32 CUDA tensor")
        m, n = A.shape
        out = outs[i] if outs is not None else trqrcp_outputs(m, n, k, A.device)
        arr[i] = problem_struct(A, k, b, p, seed, out)
        results.append(out)
    _check(load().trqrcp_batched(h.bind(), len(problems), arr, teams), h.h)
    return results


def tuxv(A, k, b, p, seed, handle=None, jmax=1):
    """Alg. 7 with j_max iterations; returns (U (m x k), X (k x k), V (n x k)),
    X upper triangular for odd j_max and lower for even j_max."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    U = empty_colmajor(m, k, A.device)
    X = empty_colmajor(k, k, A.device)
    V = empty_colmajor(n, k, A.device)
    if jmax == 1:
        _check(load().tuxv(h.bind(), m, n, _P(pa), lda, k, b, p, seed, _ptr(U), _ld(U),
                           _ptr(X), _ld(X), _ptr(V), _ld(V)), h.h)
    else:
        _check(load().tuxv_iter(h.bind(), m, n, _P(pa), lda, k, b, p, seed, jmax, _ptr(U),
                                _ld(U), _ptr(X), _ld(X), _ptr(V), _ld(V)), h.h)
    return U, X, V


def tuxv_svd(A, k, b, p, seed, handle=None, jmax=1):
    """Alg. 7 with j_max iterations and the SVD of X; returns (U (m x k),
    sigma (k, descending), V (n x k)) with A ~= U diag(sigma) V^T."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    U = empty_colmajor(m, k, A.device)
    sigma = torch.empty(k, dtype=torch.float64, device=A.device)
    V = empty_colmajor(n, k, A.device)
    _check(load().tuxv_svd(h.bind(), m, n, _P(pa), lda, k, b, p, seed, jmax, _ptr(U), _ld(U),
                           _ptr(sigma), _ptr(V), _ld(V)), h.h)
    return U, sigma, V


def gaussian(seed, stream_id, rows, cols, device="cuda", handle=None):
    """The rows x cols seeded GIID block (stream 1 = Omega)."""
    h = handle or default_handle(device)
    out = empty_colmajor(rows, cols, device)
    _check(load().rqrcp_gaussian(h.bind(), seed, stream_id, rows, cols, _ptr(out), _ld(out)),
           h.h)
    return out


def sketch(A, ell, seed, handle=None):
    """B = Omega A with the seeded l x m Omega."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    m, n = A.shape
    B = empty_colmajor(ell, n, A.device)
    _check(load().rqrcp_sketch(h.bind(), m, n, _P(pa), lda, ell, seed, _ptr(B), _ld(B)), h.h)
    return B


def gemm_bf16x(A, B, transA="N", transB="N", alpha=1.0, beta=0.0, C=None, slices=3, handle=None):
    """C = alpha op(A) op(B) + beta C on the tensor cores (FP32, column-major)."""
    h = handle or default_handle(A.device)
    for x, nm in ((A, "A"), (B, "B")):
        if x.dtype != torch.float32 or not _is_colmajor(x):
            raise ValueError(f"{nm} must be a column-major float32 CUDA tensor")
    m = A.shape[0] if transA == "N" else A.shape[1]
    k = A.shape[1] if transA == "N" else A.shape[0]
    n = B.shape[1] if transB == "N" else B.shape[0]
    if C is None:
        C = empty_colmajor(m, n, A.device, torch.float32)
        beta = 0.0
    _check(load().rqrcp_gemm_bf16x(h.bind(), transA.encode(), transB.encode(), m, n, k, alpha,
                                   _ptr(A), _ld(A), _ptr(B), _ld(B), beta, _ptr(C), _ld(C),
                                   slices), h.h)
    return C


def sample_qrcp(B, steps, handle=None):
    """Partial QRCP of the column-major float64 sample B in place; returns swaps."""
    h = handle or default_handle(B.device)
    pb, ldb = _cm(B, "B")
    ell, nc = B.shape
    swaps = torch.empty(steps, dtype=torch.int64, device=B.device)
    _check(load().rqrcp_sample_qrcp(h.bind(), ell, nc, steps, _P(pb), ldb, _ptr(swaps)), h.h)
    return swaps


def gemm_f64x(A, B, transA="N", transB="N", alpha=1.0, beta=0.0, C=None, handle=None):
    """C = alpha op(A) op(B) + beta C in FP64 on the tensor cores (exact slicing)."""
    h = handle or default_handle(A.device)
    pa, lda = _cm(A, "A")
    pb, ldb = _cm(B, "B")
    m = A.shape[0] if transA == "N" else A.shape[1]
    k = A.shape[1] if transA == "N" else A.shape[0]
    n = B.shape[1] if transB == "N" else B.shape[0]
    if C is None:
        C = empty_colmajor(m, n, A.device)
        beta = 0.0
    pc, ldc = _cm(C, "C")
    _check(load().rqrcp_gemm_f64x(h.bind(), transA.encode(), transB.encode(), m, n, k, alpha,
                                  _P(pa), lda, _P(pb), ldb, beta, _P(pc), ldc), h.h)
    return C


def sync_info(device=None):
    return default_handle(device).sync_info()


PEAK_KINDS = {"fp64_fma": 0, "fp64_dmma_m8n8k4": 1, "fp64_dmma_m16n8k16": 2, "fp32_fma": 3,
              "fp64_fma_outer": 4}


def peak_probe(kind, iters, grid, device="cuda"):
    """One launch of the arithmetic-peak probe `kind` (see PEAK_KINDS) on the
    current stream; returns (CUDA-event milliseconds, flops of the launch)."""
    dev = torch.device(device)
    dt = torch.float32 if kind == "fp32_fma" else torch.float64
    sink = torch.empty(grid * 256, dtype=dt, device=dev)
    stream = torch.cuda.current_stream(dev)
    fl = ctypes.c_double(0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = load().rqrcp_peak_probe(PEAK_KINDS[kind], iters, grid, _ptr(sink), _P(stream.cuda_stream),
                                 ctypes.byref(fl))
    e1.record(stream)
    if rc != RQRCP_OK:
        raise RqrcpError(f"rqrcp_peak_probe: {rc}")
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1), fl.value
