"""Bounded device waits: a wait that nothing completes gives up, the device
flag reports TC_ERR_TIMEOUT once, and the context stays usable."""
import numpy as np
import pytest

import oracle
import tcsynth as ts
from gpu_util import compare, run

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_context_survives():
    import torch
    from paper_1307_2100_gb300 import tc
    s = torch.cuda.current_stream().cuda_stream
    assert tc.tc_device_status(s) == tc.TC_OK
    tc.tc_selftest_wait_timeout(50_000_000, s)     # 50 ms
    torch.cuda.synchronize()
    assert tc.tc_device_status(s) == tc.TC_ERR_TIMEOUT
    assert tc.tc_device_status(s) == tc.TC_OK      # read-and-clear
    p = ts.fused_permute_48(n=9)
    assert compare(run(p), oracle.contract_problem(p), p.C) <= 1e-12
