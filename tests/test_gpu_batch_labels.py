"""GPU parity of contractions with batch (Hadamard) labels -- labels in A, B
and C, beyond the paper's definition: one contraction per value, through the
GEMM view's batch group, on every kernel family that takes it."""
import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import TOL_FP64, compare, magnitude, run, tc_bounds, within

pytestmark = pytest.mark.gpu


def cases():
    return [
        ts.problem("bgemm", "aiz", "ibz", "abz", dict(a=70, i=90, b=40, z=5), 101),
        ts.problem("bgemm2", "zajb", "jcz", "abcz", dict(z=3, a=20, j=33, b=6, c=25), 102),
        ts.problem("bgemv", "aiz", "iz", "az", dict(a=300, i=200, z=6), 103),
        ts.problem("bdot", "iz", "iz", "z", dict(i=5000, z=9), 104),
        ts.problem("hadamard", "ab", "ab", "ab", dict(a=130, b=70), 105),
    ]


@pytest.mark.parametrize("k", range(5))
def test_batch_labels_fp64_every_mapping(k):
    p = cases()[k]
    ref = oracle.contract_problem(p)
    for mapping in ("auto", "fused_gemm", "slice_gemm", "gemv", "dot", "ger"):
        try:
            got = run(p, "fp64", mapping)
        except Exception as e:  # a mapping that cannot take the contraction
            assert "UNSUPPORTED" in str(e), (p.name, mapping, e)
            continue
        assert compare(got, ref, p.C) <= TOL_FP64, (p.name, mapping)


@pytest.mark.parametrize("form", ["bf16x6", "fp32"])
def test_batch_labels_fp32_storage(form):
    for p in cases()[:2]:
        for t in (p.A, p.B, p.C):
            t.data = t.data.astype(np.float32)
        got = run(p, form, "fused_gemm")
        mag = magnitude(p)
        if form == "bf16x6":
            acc, _ = tc_bounds(p, form)
            ok, d = within(got, op.contract_form(p, form), mag, p.C, acc)
        else:
            K = int(np.prod([e for l, e in zip(p.A.labels, p.A.extents)
                             if l in p.B.labels and l not in p.C.labels]))
            ok, d = within(got, oracle.contract_problem(p), mag, p.C, (K + 2) * 2.0 ** -23)
        assert ok, (p.name, form, d)
