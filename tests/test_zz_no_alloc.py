"""The allocation-free sample-QRCP entry point (rqrcp_sample_qrcp_noalloc).

It exists for callers that cannot allocate device memory (stream capture,
allocator-free loops, pool-owned memory): it runs the same kernel as
rqrcp_sample_qrcp with its scratch in a fixed device array of the library.
These tests call it through the C ABI and compare it with the handle-based
entry point on the same inputs, for two calls in a row (the array keeps the
previous call's contents, so the second call checks that each call clears
what it needs).  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sample(ell, nc, seed):
    r = np.random.default_rng(seed)
    B = r.standard_normal((ell, nc)) * np.exp(r.standard_normal(nc))[None, :]
    return torch.from_numpy(B.T.copy()).cuda().t()  # column-major ell x nc


def _noalloc(lib, B, steps):
    raw = lib.load()
    ell, nc = B.shape
    swaps = torch.empty(steps, dtype=torch.int64, device=B.device)
    info = torch.zeros(1, dtype=torch.int32, device=B.device)
    stream = torch.cuda.current_stream(B.device)
    rc = raw.rqrcp_sample_qrcp_noalloc(ell, nc, steps, ctypes.c_void_p(B.data_ptr()), B.stride(1),
                                       ctypes.c_void_p(swaps.data_ptr()),
                                       ctypes.c_void_p(info.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, raw.rqrcp_status_string(rc)
    torch.cuda.synchronize(B.device)
    return swaps, int(info.item())


def test_noalloc_matches_handle_entry_point(lib):
    # two calls in a row; the second is larger than the first
    for call, (ell, nc, steps) in enumerate([(40, 700, 32), (72, 5000, 64)]):
        B = _sample(ell, nc, 100 + call)
        B_ref, B_new = B.clone(), B.clone()
        swaps_ref = lib.sample_qrcp(B_ref, steps)
        assert lib.sync_info() == 0
        swaps_new, info = _noalloc(lib, B_new, steps)
        assert info == 0
        np.testing.assert_array_equal(swaps_new.cpu().numpy(), swaps_ref.cpu().numpy())
        scale = B.abs().max().item()
        assert (B_new - B_ref).abs().max().item() <= 1e-12 * scale


def test_noalloc_matches_oracle(lib):
    """One direct comparison with the oracle's Alg. 1 halted after `steps`
    pivots (replaying the device's pivots through exact ties): the same swap
    sequence and the same S = Q_b^T B P."""
    from oracle.rqrcp import sample_qrcp
    ell, nc, steps = 24, 300, 16
    B = _sample(ell, nc, 7)
    B_host = B.cpu().numpy().copy()
    B_new = B.clone()
    swaps, info = _noalloc(lib, B_new, steps)
    assert info == 0
    sw = swaps.cpu().numpy()
    ids = np.arange(nc)
    for i, s in enumerate(sw):
        ids[[i, s]] = ids[[s, i]]
    S = B_host.copy()
    sw_o, _, _ = sample_qrcp(S, steps, ids=np.arange(nc), forced_ids=ids[:steps])
    np.testing.assert_array_equal(sw, sw_o)
    assert np.abs(B_new.cpu().numpy() - S).max() <= 1e-12 * np.abs(B_host).max()


def test_noalloc_reports_nonfinite(lib):
    """A NaN in the sample is reported through the caller's status word."""
    B = _sample(16, 64, 3)
    B[5, 17] = float("nan")
    _, info = _noalloc(lib, B, 8)
    assert info & lib.INFO_NONFINITE


def test_noalloc_requires_info_word(lib):
    raw = lib.load()
    B = _sample(8, 16, 1)
    swaps = torch.empty(8, dtype=torch.int64, device=B.device)
    p = ctypes.c_void_p
    assert raw.rqrcp_sample_qrcp_noalloc(8, 16, 8, p(B.data_ptr()), 8, p(swaps.data_ptr()),
                                         None, None) == -7


def test_noalloc_rejects_out_of_range(lib):
    raw = lib.load()
    B = _sample(8, 16, 1)
    swaps = torch.empty(8, dtype=torch.int64, device=B.device)
    p = ctypes.c_void_p
    # ell above the array's 192-row capacity
    assert raw.rqrcp_sample_qrcp_noalloc(193, 16, 8, p(B.data_ptr()), 193, p(swaps.data_ptr()),
                                         None, None) == -1
    # more steps than sample rows
    assert raw.rqrcp_sample_qrcp_noalloc(8, 16, 9, p(B.data_ptr()), 8, p(swaps.data_ptr()),
                                         None, None) == -3
