"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes gives
up within its limit, reports LBM_ETIMEOUT to the host, and leaves the context usable; the step
kernels' copies use the same wait.  (Failures on the host side, invalid inputs, unstable states and
failing server jobs, are covered by the ABI, parity and server tests.)"""
import time

import pytest

from paper_2408_15654_gb300 import lbm
from paper_2408_15654_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    t0 = time.time()
    rc = lbm.lbm_selftest_wait(word.data_ptr(), stream.cuda_stream)
    dt = time.time() - t0
    assert rc == lbm.LBM_ETIMEOUT, lbm.lbm_last_error()
    assert int(word.item()) != 0          # the kernel recorded the timeout
    assert dt < 5.0                       # the wait is bounded (about one second)
    # the context still runs the fused step
    p, f = W.stationary_drop(32, 32, R=8)
    g = lbm.Lattice(p)
    g.init(**f)
    g.step(10)
    assert g.status == lbm.LBM_OK
    g.close()
