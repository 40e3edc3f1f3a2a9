"""GPU parity of the GER mapping (rank-K update for tiny contracted ranges).

FP64 storage: against the FP64 oracle within 1e-12 relative Frobenius.
FP32 storage: each output is a K-term FP32 sum (K <= 32) of exact products,
so it is within (K + 2) * 2^-24 of sum |a||b| of the FP64 oracle, whatever
the math form the plan names."""
import numpy as np
import pytest

import oracle
import tcsynth as ts
from gpu_util import TOL_FP64, compare, magnitude, run, within

pytestmark = pytest.mark.gpu


def cases():
    return [
        # GR-shaped (Sec. 4.2): the two contracted indices of extent 4
        ts.problem("gr", "iajb", "icjd", "abcd", dict(i=4, j=4, a=37, b=23, c=41, d=19), 81),
        ts.problem("outer", "ai", "ib", "ab", dict(a=1000, i=1, b=333), 82),
        ts.problem("k3", "aib", "ic", "abc", dict(a=300, i=3, b=7, c=129), 83),
        ts.problem("k32", "ia", "bi", "ab", dict(i=32, a=257, b=65), 84),
        ts.problem("cperm", "aijb", "ijcd", "abcd", dict(a=20, i=2, j=5, b=17, c=33, d=6), 85,
                   order_c=[2, 0, 3, 1]),          # C stored c fastest, then a, d, b
    ]


@pytest.mark.parametrize("k", range(5))
def test_ger_fp64(k):
    p = cases()[k]
    info = []
    got = run(p, "fp64", "ger", plan_out=info)
    assert info[0]["kernel_name"] == "ger"
    assert compare(got, oracle.contract_problem(p), p.C) <= TOL_FP64


def test_ger_fp64_alpha_beta():
    p = cases()[0]
    p.C.data = np.linspace(-1, 1, p.C.data.size)
    p.alpha, p.beta = 0.75, -2.0
    got = run(p, "fp64", "ger")
    assert compare(got, oracle.contract_problem(p), p.C) <= TOL_FP64


@pytest.mark.parametrize("form", ["fp32", "bf16x6"])
def test_ger_fp32_storage(form):
    for p in cases():
        for t in (p.A, p.B, p.C):
            t.data = t.data.astype(np.float32)
        K = int(np.prod([e for l, e in zip(p.A.labels, p.A.extents) if l in p.B.labels]))
        got = run(p, form, "ger")
        ok, d = within(got, oracle.contract_problem(p), magnitude(p), p.C, (K + 2) * 2.0 ** -24)
        assert ok, (p.name, form, d)
