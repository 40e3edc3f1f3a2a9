"""Free-index sharding on the GPU: every shard of a contraction planned and run
through the C ABI one after another on one device (standing in for one
device per rank), each writing its slab of C; the assembled C against the
oracle (FP64 within 1e-12, integers bit for bit; BF16x6 within its bound)."""
import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import TOL_FP64, compare, magnitude, tc_bounds, within

pytestmark = pytest.mark.gpu


def _run_shards(p, n, dtype, math):
    import torch
    from paper_1307_2100_gb300.shard import ShardedContraction
    dev = torch.device("cuda:0")
    descs = [(t.labels, t.extents, t.strides) for t in (p.A, p.B, p.C)]
    A = torch.from_numpy(np.ascontiguousarray(p.A.data)).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(p.B.data)).to(dev)
    C = torch.full((max(p.C.data.size, 1),), float("nan"), dtype=A.dtype, device=dev)
    spans = []
    for r in range(n):
        sc = ShardedContraction(*descs, dtype, math, rank=r, world=n)
        sc(A, B, C)
        spans.append((sc.shard.begin, sc.shard.end))
    torch.cuda.synchronize()
    return C.cpu().numpy().astype(np.float64)[: p.C.data.size], spans


@pytest.mark.parametrize("n", [2, 3, 7])
def test_fp64_shards_against_the_oracle(n):
    for p in [ts.direct_gemm_64(n=19), ts.fused_permute_48(n=13),
              ts.problem("gemv", "aib", "i", "ab", dict(a=300, i=211, b=7), 53),
              ts.problem("c_rowmajor", "ai", "ib", "ab", dict(a=130, i=40, b=129), 57,
                         order_c=[1, 0])]:
        got, spans = _run_shards(p, n, "f64", "fp64")
        assert compare(got, oracle.contract_problem(p), p.C) <= TOL_FP64, (p.name, n)


def test_integer_shards_bitwise():
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=2), 41,
                   dist="int", lo=-4, hi=4)
    got, spans = _run_shards(p, 4, "f64", "fp64")
    np.testing.assert_array_equal(got, oracle.contract_problem(p))
    assert spans == [(0, 17), (17, 35), (35, 52), (52, 70)]   # a (70) is the largest index


def test_bf16x6_shards_within_the_form_bound():
    p = ts.direct_gemm_64(n=23)
    for t in (p.A, p.B, p.C):
        t.data = t.data.astype(np.float32)
    got, _ = _run_shards(p, 3, "f32", "bf16x6")
    acc, _ = tc_bounds(p, "bf16x6")
    ok, d = within(got, op.contract_form(p, "bf16x6"), magnitude(p), p.C, acc)
    assert ok, d
