"""The workspace-free scalar contraction (tc_contract_dot_noalloc).

Callers that cannot allocate device memory while they contract (runtimes
that own all device memory, plug-ins given only input and output pointers)
use this entry point; it keeps the partial sums of the scalar reduction in a
scratch array built into the library.  The test compares it, through the C
ABI, with the regular tc_contract (which takes a workspace) and with the CPU
oracle, on two calls in a row, for FP64 and FP32 data, within the FP64 parity
tolerance of the other tests.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import tcsynth as ts

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _plan(p, dtype, math):
    from paper_1307_2100_gb300 import tc
    return tc.tc_plan((p.A.labels, p.A.extents, p.A.strides),
                      (p.B.labels, p.B.extents, p.B.strides),
                      (p.C.labels, p.C.extents, p.C.strides), dtype, math)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_scalar_matches_tc_contract_twice(dt):
    import torch
    from paper_1307_2100_gb300 import tc
    npdt = np.float64 if dt == "f64" else np.float32
    tdt = torch.float64 if dt == "f64" else torch.float32
    dev = torch.device("cuda:0")
    s = torch.cuda.current_stream().cuda_stream
    handle = _plan(ts.problem("k1", "ijk", "kji", "", dict(i=37, j=41, k=53), 7),
                   tc.TC_F64 if dt == "f64" else tc.TC_F32,
                   tc.MATH["fp64"] if dt == "f64" else tc.MATH["fp32"])
    try:
        info = tc.tc_plan_get_info(handle)
        assert info.cls == 1 and info.workspace > 0
        ws = torch.empty(int(info.workspace), dtype=torch.uint8, device=dev)
        for call, (seed, alpha, beta) in enumerate([(8, 1.0, 0.0), (9, -0.5, 2.0)]):
            p = ts.problem("k1", "ijk", "kji", "", dict(i=37, j=41, k=53), seed, dtype=npdt)
            A = torch.from_numpy(p.A.data).to(dev)
            B = torch.from_numpy(p.B.data).to(dev)
            c0 = torch.full((1,), 0.75, dtype=tdt, device=dev)
            ref = c0.clone()
            got = c0.clone()
            tc.tc_contract(handle, alpha, A.data_ptr(), B.data_ptr(), beta, ref.data_ptr(),
                           ws.data_ptr(), ws.numel(), s)
            tc.tc_contract_dot_noalloc(handle, alpha, A.data_ptr(), B.data_ptr(), beta,
                                       got.data_ptr(), s)
            torch.cuda.synchronize()
            r, g = float(ref.item()), float(got.item())
            assert abs(g - r) <= TOL * max(abs(r), 1e-300), (call, g, r)
            # and against the oracle, from the same (storage-precision) inputs;
            # an FP32 result is also rounded once to FP32 (half an ulp, 2^-24)
            o = oracle.contract(p.A, p.B, p.C, alpha, beta,
                                c_init=np.full(1, float(c0.item())))
            tol = TOL + (2.0 ** -24 if dt == "f32" else 0.0)
            assert abs(g - o[0]) <= tol * max(abs(o[0]), 1e-300), (call, g, o[0])
    finally:
        tc.tc_plan_destroy(handle)


def test_noalloc_rejects_plans_that_are_not_a_scalar_dot():
    from paper_1307_2100_gb300 import tc
    p = ts.fused_permute_48(n=5)
    handle = _plan(p, tc.TC_F64, tc.MATH["fp64"])
    try:
        with pytest.raises(tc.TcError) as e:
            tc.tc_contract_dot_noalloc(handle, 1.0, 16, 16, 0.0, 16, 0)
        assert e.value.status == 5
    finally:
        tc.tc_plan_destroy(handle)
