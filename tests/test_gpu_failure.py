"""Failure detection on the device, without a GPU fault.

Every device-side wait of the library (the software grid barrier of the
cooperative kernels, the mbarrier waits of the tensor-core GEMMs) is bounded:
when it runs out the kernel ORs RQRCP_INFO_TIMEOUT into the handle's status
word and returns, and the context stays usable.  This test makes one such
wait run out on purpose through the test-only handle option
RQRCP_OPT_TEST_BARRIER_TIMEOUT: the sample-QRCP kernel's grid barrier then
waits for one CTA that does not exist (a count that nothing completes) and
gives up after a few milliseconds.  Nothing traps, faults or waits forever.
"""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sample(ell, nc, seed):
    r = np.random.default_rng(seed)
    B = r.standard_normal((ell, nc)) * np.exp(r.standard_normal(nc))[None, :]
    return torch.from_numpy(B.T.copy()).cuda().t()  # column-major ell x nc


def test_grid_barrier_timeout_is_reported_and_handle_recovers(lib):
    ell, nc, steps = 72, 5000, 64
    B0 = _sample(ell, nc, 11)
    h = lib.Handle()

    # a wait that cannot complete: bounded, reported, no partial result
    B = B0.clone()
    h.set_test_barrier_timeout(True)
    t0 = time.perf_counter()
    swaps = lib.sample_qrcp(B, steps, handle=h)
    info = h.sync_info()
    elapsed = time.perf_counter() - t0
    assert info & lib.INFO_TIMEOUT, info
    assert elapsed < 5.0, elapsed
    assert torch.equal(B, B0)                      # the sample is left as it was
    assert torch.equal(swaps.cpu(), torch.arange(steps))  # no-exchange partners
    assert h.sync_info() == 0                      # reading the word cleared it

    # the same handle, option off: a normal call, identical to a fresh handle's
    h.set_test_barrier_timeout(False)
    B1 = B0.clone()
    swaps1 = lib.sample_qrcp(B1, steps, handle=h)
    assert h.sync_info() == 0
    B2 = B0.clone()
    h2 = lib.Handle()
    swaps2 = lib.sample_qrcp(B2, steps, handle=h2)
    assert h2.sync_info() == 0
    assert torch.equal(swaps1, swaps2)
    assert torch.equal(B1, B2)
