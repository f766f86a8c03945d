"""Failure detection on the device without a GPU fault.

Every device-side wait of the library (the mbarrier that a TMA bulk copy completes) polls a bounded
number of times; when it gives up the kernel records an error flag and returns, and the call
reports QMMM_ERR_TIMEOUT.  The self-test makes such a wait run out on a barrier that nothing
completes; the CUDA context must stay usable afterwards, which the same process then shows by
evaluating a small system to full parity with the oracle."""
import time

import numpy as np
import pytest

import oracle
import workloads
from _gpuutil import TOL_FP64, gpu_all, rel_fro

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    torch.cuda.init()
    t0 = time.perf_counter()
    rc = q.qmmm_selftest_bounded_wait(torch.cuda.current_stream())
    dt = time.perf_counter() - t0
    assert rc == -4, (rc, q.qmmm_last_error())
    assert dt < 10.0
    # the context still runs kernels correctly
    s = workloads.small_system(5, n_atoms=3, lmax=2)
    g = gpu_all(s, precision=0)
    assert rel_fro(g["V"], oracle.vpot(s)) < TOL_FP64
    assert torch.cuda.is_available() and float(torch.ones(4, device="cuda").sum().item()) == 4.0


def test_bounded_wait_repeatable():
    torch = pytest.importorskip("torch")
    import paper_2408_03273_gb300 as q
    for _ in range(2):
        assert q.qmmm_selftest_bounded_wait(None) == -4
    torch.cuda.synchronize()
