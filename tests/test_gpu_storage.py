"""GPU parity of BF16 and FP16 storage and of the FP16 tensor-core form.

Inputs are made 2-byte by rounding FP32 values to the storage type; the oracle
then contracts the stored values (read exactly, widened to FP64).  Bounds,
as multiples of sum |a||b| (the worst-case scale of rounding errors):
  * accumulation in FP32: at most one unit of the running sum per 16-product
    tensor-core block, (K/16 + 1) 2^-23; on the CUDA cores K 2^-24 per output;
  * the result rounded once to the storage type: 2^-9 (BF16), 2^-12 (FP16);
  * the FP16 form from FP32 storage rounds both operands to binary16 first:
    against the oracle's FP16 form (oracle.precision.contract_f16, the same
    rounded products summed exactly) only accumulation remains, against the
    FP64 oracle on the FP32 values 2 * 2^-11 more.
Small integers are exact in both 2-byte types, and with them every partial
sum is exact in FP32: those results must equal the oracle's bit for bit."""
import copy

import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import addressed_index, magnitude, within

pytestmark = pytest.mark.gpu

OUT_ROUND = {"bf16": 2.0 ** -9, "f16": 2.0 ** -12}


def _torch_dtype(dt):
    import torch
    return {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32}[dt]


def stored(p, dt):
    """Problem p with its A and B rounded to storage type dt (to nearest, by
    torch on the host); the data arrays hold the stored values widened."""
    import torch
    q = copy.deepcopy(p)
    for t in (q.A, q.B, q.C):
        x = torch.from_numpy(np.asarray(t.data, np.float32)).to(_torch_dtype(dt))
        t.data = x.to(torch.float64).numpy()
    return q


def run_storage(q, dt, math, mapping="auto", tile=-1, alpha=1.0, beta=0.0):
    """Run q (values already representable in dt) with A, B, C stored as dt;
    returns C's buffer widened to FP64 and the plan's info."""
    import torch
    from paper_1307_2100_gb300 import Contraction
    dev = torch.device("cuda:0")
    tdt = _torch_dtype(dt)
    plan = Contraction((q.A.labels, q.A.extents, q.A.strides),
                       (q.B.labels, q.B.extents, q.B.strides),
                       (q.C.labels, q.C.extents, q.C.strides), dt, math, mapping, tile)
    mk = lambda t: torch.from_numpy(np.asarray(t.data, np.float64)).to(dev).to(tdt) \
        if t.data.size else torch.zeros(1, dtype=tdt, device=dev)
    A, B, C = mk(q.A), mk(q.B), mk(q.C)
    plan(A, B, C, alpha, beta)
    torch.cuda.synchronize()
    return C.to(torch.float64).cpu().numpy()[: q.C.data.size], plan.info


def k_of(p):
    K = 1
    for l, e in zip(p.A.labels, p.A.extents):
        if l in p.B.labels:
            K *= int(e)
    return K


def shapes():
    return [
        ts.direct_gemm_64(n=21),                                      # Class 3.2
        ts.fused_permute_48(n=15),                                    # Class 3.1
        ts.problem("cfromb", "ai", "ib", "ba", dict(a=140, i=77, b=260), 52),
        ts.problem("gemv", "aib", "i", "ab", dict(a=300, i=211, b=7), 53),   # Class 2
        ts.problem("dot", "ijk", "kji", "", dict(i=37, j=41, k=23), 54),     # Class 1
        ts.problem("ger", "ai", "ib", "ab", dict(a=333, i=5, b=97), 55),     # tiny K
    ]


CASES = [("bf16", "fp32"), ("bf16", "bf16"), ("f16", "fp32"), ("f16", "fp16")]
MAPS = ["auto", "fused_gemm", "slice_gemm", "copy_gemm", "gemv", "dot", "ger"]


def _feasible(p, mapping):
    from oracle import classify as ocl
    cls = ocl.classify(p.A, p.B, p.C).cls
    if mapping in ("slice_gemm", "copy_gemm", "fused_gemm") and cls not in (31, 32):
        return False
    if mapping == "ger" and k_of(p) > 32:
        return False
    return True


@pytest.mark.parametrize("dt,math", CASES)
def test_integer_inputs_bitwise_every_mapping(dt, math):
    # entries in [-2, 2], K = 16: |C| <= 64, so every result is a BF16 and
    # an FP16 value and every partial sum is exact in FP32
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=4, a=70, j=4, b=3, c=65, d=2), 61,
                   dist="int", lo=-2, hi=2, dtype=np.float32)
    q = stored(p, dt)
    ref = oracle.contract_problem(q)
    for mapping in MAPS:
        if not _feasible(q, mapping):
            continue
        got, info = run_storage(q, dt, math, mapping)
        np.testing.assert_array_equal(got, ref, err_msg=f"{dt} {math} {mapping}")


@pytest.mark.parametrize("dt,math", CASES)
def test_shapes_against_the_fp64_oracle(dt, math):
    for p in shapes():
        q = stored(p, dt)
        ref = oracle.contract_problem(q)
        got, info = run_storage(q, dt, math)
        K = k_of(q)
        acc = (K / 16 + 1) * 2.0 ** -23 if info.kernel == 2 else K * 2.0 ** -24
        ok, d = within(got, ref, magnitude(q), q.C, acc + OUT_ROUND[dt])
        assert ok, (p.name, dt, math, info.kernel, d)


@pytest.mark.parametrize("dt,math", CASES)
def test_alpha_beta_read_and_write_the_storage_type(dt, math):
    p = ts.problem("ab", "iajb", "jcid", "abcd", dict(i=3, a=40, j=5, b=2, c=33, d=3), 71,
                   dist="int", lo=-2, hi=2, dtype=np.float32)
    q = stored(p, dt)
    rng = np.random.default_rng(5)
    q.C.data = rng.integers(-8, 9, q.C.data.size).astype(np.float64)
    ref = oracle.contract(q.A, q.B, q.C, 0.5, -2.0)
    got, _ = run_storage(q, dt, math, alpha=0.5, beta=-2.0)
    np.testing.assert_array_equal(got, ref)


def test_fp16_form_from_fp32_storage():
    """The FP16 form of FP32 data: packed tensor-core GEMM on binary16-rounded
    operands; integers exact, general values within the accumulation bound of
    the oracle's FP16 form and within 2 * 2^-11 more of the FP64 oracle."""
    from gpu_util import run
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=2), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    np.testing.assert_array_equal(run(p, "fp16", "fused_gemm"), oracle.contract_problem(p))
    for q in [ts.direct_gemm_64(n=19), ts.fused_permute_48(n=13),
              ts.problem("long_k", "ai", "ib", "ab", dict(a=130, i=3000, b=140), 56)]:
        for t in (q.A, q.B, q.C):
            t.data = t.data.astype(np.float32)
        got = run(q, "fp16", "auto")
        K = k_of(q)
        acc = (K / 16 + 1) * 2.0 ** -23
        mag = magnitude(q)
        ok, d = within(got, op.contract_f16(q), mag, q.C, acc)
        assert ok, (q.name, "form", d)
        ok, d = within(got, oracle.contract_problem(q), mag, q.C, acc + 2 * 2.0 ** -11)
        assert ok, (q.name, "fp64", d)


def test_fp16_form_overflow_to_infinity():
    """binary16 overflows from 65520 on: a product involving such an input is
    infinite on the tensor cores, as the oracle's rounding says."""
    from gpu_util import run
    p = ts.problem("ov", "ai", "ib", "ab", dict(a=130, i=40, b=129), 57, dtype=np.float32)
    p.A.data[5] = 70000.0            # row 5 of A, first k
    got = run(p, "fp16", "fused_gemm")
    ref = op.contract_f16(p)
    assert np.all(np.isinf(got[np.isinf(ref)])) and np.isinf(ref).any()
    fin = np.isfinite(ref)
    assert np.all(np.isfinite(got[fin]))


def test_bf16_storage_with_batch_labels_runs_on_the_cuda_cores():
    """A batch (Hadamard) label gives a batch of GEMMs; for BF16 data with the
    BF16 form they run on the CUDA cores in FP32, bitwise equal on integers."""
    p = ts.problem("bat", "aib", "icb", "acb", dict(a=40, i=9, c=37, b=5), 81,
                   dist="int", lo=-2, hi=2, dtype=np.float32)
    q = stored(p, "bf16")
    got, info = run_storage(q, "bf16", "bf16")
    assert info.kernel == 1
    np.testing.assert_array_equal(got, oracle.contract_problem(q))


@pytest.mark.parametrize("tile", [4, 5])
@pytest.mark.parametrize("dt,math", [("bf16", "bf16"), ("f16", "fp16"), ("f32", "fp16")])
def test_tensor_core_forms_on_wide_tiles(dt, math, tile):
    """The 128 x 256 tiles and the 256 x 256 pair tiles with each operand type."""
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=4, a=70, j=4, b=3, c=65, d=5), 61,
                   dist="int", lo=-2, hi=2, dtype=np.float32)
    q = stored(p, dt)
    got, info = run_storage(q, dt, math, "fused_gemm", tile)
    assert info.tile == tile
    np.testing.assert_array_equal(got, oracle.contract_problem(q))
    for p in shapes()[:3]:
        q = stored(p, dt)
        got, info = run_storage(q, dt, math, "fused_gemm", tile)
        K = k_of(q)
        acc = (K / 16 + 1) * 2.0 ** -23
        rnd = OUT_ROUND.get(dt, 0.0) + (2 * 2.0 ** -11 if dt == "f32" else 0.0)
        ok, d = within(got, oracle.contract_problem(q), magnitude(q), q.C, acc + rnd)
        assert ok, (p.name, dt, math, d)

