"""GPU parity of the tensor-core path (FP32 storage; BF16, BF16x3, BF16x6 math).

Two references, each with a worst-case bound proportional to sum |a||b|
(gpu_util.tc_bounds derives them from the arithmetic):
  * the split-form oracle (oracle.precision.contract_form): the same BF16 term
    products summed exactly in FP64; the kernel differs only by its FP32
    accumulation;
  * the FP64 oracle on the FP32 inputs: the form's split error on top.
The FP32-class claim is checked as stated: BF16x6 on the precision workload
is within 1e-6 relative Frobenius of the FP64 oracle.
Integer inputs in [-4, 4] are BF16 values and all partial sums are exact in
FP32, so every form must then match the FP64 oracle bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import (SPLIT_ERR, compare, gather, magnitude, random_output_indices, run,
                      sample_outputs, sample_outputs_form, tc_bounds, within)

pytestmark = pytest.mark.gpu

FORMS = ["bf16", "bf16x3", "bf16x6"]
FP32_CLASS = 1e-6


def f32(p):
    for t in (p.A, p.B, p.C):
        t.data = t.data.astype(np.float32)
    return p


def shapes():
    return [
        f32(ts.direct_gemm_64(n=23)),                                  # Class 3.2, ragged tiles
        f32(ts.fused_permute_48(n=17)),                                # Class 3.1, fused permute
        f32(ts.problem("m1", "ai", "ib", "ab", dict(a=300, i=200, b=130), 51)),
        f32(ts.problem("cfromb", "ai", "ib", "ba", dict(a=140, i=77, b=260), 52)),
        f32(ts.slice_gemm_48()),
    ]


# tile 0: operands gathered and split inside the GEMM; tile 3: packed operands
# (a pack pass splits them once, the GEMM moves the terms with bulk copies)
TILES = [0, 3]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("form", FORMS)
def test_integer_inputs_exact(form, tile):
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=2), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    got = run(p, form, "fused_gemm", tile)
    np.testing.assert_array_equal(got, oracle.contract_problem(p))


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("form", FORMS)
def test_forms_against_method_and_fp64_oracles(form, tile):
    for p in shapes():
        got = run(p, form, "fused_gemm", tile)
        mag = magnitude(p)
        acc, tot = tc_bounds(p, form)
        ok, d = within(got, op.contract_form(p, form), mag, p.C, acc)
        assert ok, (p.name, form, "method", d)
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, tot)
        assert ok, (p.name, form, "fp64", d)


@pytest.mark.parametrize("mapping", ["fused_gemm", "slice_gemm", "copy_gemm"])
def test_bf16x6_mappings(mapping):
    p = f32(ts.fused_permute_48(n=19))
    got = run(p, "bf16x6", mapping)
    acc, _ = tc_bounds(p, "bf16x6")
    assert within(got, op.contract_form(p, "bf16x6"), magnitude(p), p.C, acc)[0]


@pytest.mark.parametrize("tile", [0, 1, 2])
def test_chunk_configurations(tile):
    p = f32(ts.problem("longk", "aijb", "ijc", "abc", dict(a=130, i=40, j=60, b=2, c=129), 53))
    mag = magnitude(p)
    for form in ("bf16x3", "bf16x6"):
        got = run(p, form, "fused_gemm", tile)
        acc, _ = tc_bounds(p, form, chunk_k={0: 256, 1: 64, 2: 1024}[tile])
        assert within(got, op.contract_form(p, form), mag, p.C, acc)[0], (tile, form)


@pytest.mark.parametrize("tile", TILES)
def test_alpha_beta_tc(tile):
    p = f32(ts.direct_gemm_64(n=21))
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    got = run(p, "bf16x6", "fused_gemm", tile)
    acc, _ = tc_bounds(p, "bf16x6")
    mag = magnitude(p) + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
    assert within(got, op.contract_form(p, "bf16x6"), mag, p.C, acc)[0]


def test_packed_ragged_and_long_k():
    """Packed operands: K not a multiple of 32 or 128, one-row tiles, K spanning
    many chunks, every form."""
    cases = [f32(ts.problem("r1", "ai", "ib", "ab", dict(a=129, i=45, b=131), 81)),
             f32(ts.problem("r2", "aijb", "ijc", "abc", dict(a=3, i=7, j=5, b=70, c=200), 82)),
             f32(ts.problem("r3", "ai", "ib", "ab", dict(a=200, i=3000, b=150), 83))]
    for p in cases:
        for form in FORMS:
            got = run(p, form, "fused_gemm", 3)
            acc, _ = tc_bounds(p, form)
            ok, d = within(got, op.contract_form(p, form), magnitude(p), p.C, acc)
            assert ok, (p.name, form, d)


def test_precision_workload_full_size_sampled():
    """C[a,b,i,j] = sum_{e,f} A[a,b,e,f] B[e,f,i,j], a=b=e=f=128, i=j=32 (FP32
    storage) at full size, sampled outputs against both oracles."""
    p = ts.precision_ccd()
    s = random_output_indices(p, 96, seed=3)
    ref64 = sample_outputs(p, s)
    import copy
    pm = copy.copy(p)
    pm.A = copy.copy(p.A)
    pm.B = copy.copy(p.B)
    pm.A.data = np.abs(p.A.data)
    pm.B.data = np.abs(p.B.data)
    mag = sample_outputs(pm, s)
    for form, tile in [(f, t) for f in FORMS for t in TILES]:
        got = run(p, form, "fused_gemm", tile)
        g = gather(got, p.C, s)
        acc, tot = tc_bounds(p, form)
        assert np.linalg.norm(g - sample_outputs_form(p, s, form)) <= acc * np.linalg.norm(mag), form
        assert np.linalg.norm(g - ref64) <= tot * np.linalg.norm(mag), form
        assert np.all(np.isfinite(got))
        if form == "bf16x6":   # the FP32-class claim
            assert oracle.rel_fro(g, ref64) <= FP32_CLASS


def test_gathering_kernel_multi_label_k_groups():
    """Single launches of the gathering kernel (tiles 0-2) on operands whose K
    group keeps two labels (not linear in B): the K offsets come from a shared
    table rewritten for every block, including the prefetch prologue."""
    items = ts.batching_items(512)
    for j in (1, 104):
        p = items[j]
        mag = magnitude(p)
        for tile in (0, 1, 2):
            got = run(p, "bf16x6", "fused_gemm", tile)
            acc, _ = tc_bounds(p, "bf16x6", chunk_k={0: 256, 1: 64, 2: 1024}[tile])
            ok, d = within(got, op.contract_form(p, "bf16x6"), mag, p.C, acc)
            assert ok, (j, tile, d)


def test_packed_split_k():
    """Few output tiles and a long K (the CCD shape of Sec. 4.2 with short free
    extents): the packed GEMM shares K out among CTAs and adds their FP64
    partial sums in order; every form within its bound."""
    p = f32(ts.problem("splitk", "iajb", "icjd", "abcd",
                       dict(i=60, j=55, a=30, b=8, c=30, d=9), 121))
    plans = []
    for form in FORMS:
        got = run(p, form, "fused_gemm", 3, plan_out=plans)
        acc, _ = tc_bounds(p, form)
        ok, d = within(got, op.contract_form(p, form), magnitude(p), p.C, acc)
        assert ok, (form, d)
    # 2 x 3 tiles of 128 x 128 and 104 K blocks: split-K workspace in the plan
    info = plans[-1]
    tiles = -(-info["M"] // 128) * -(-info["N"] // 128)
    assert tiles < 152 and info["workspace"] > 0


# tile 4: packed operands on 128 x 256 tiles, one FP32 accumulator per chunk;
# tile 5: the same arithmetic on 256 x 256 tiles shared by a pair of SMs
WIDE_FORMS = ["bf16", "bf16x3"]
WIDE_TILES = [4, 5]


@pytest.mark.parametrize("tile", WIDE_TILES)
@pytest.mark.parametrize("form", WIDE_FORMS)
def test_wide_tiles_integer_inputs_exact(form, tile):
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=5), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    got = run(p, form, "fused_gemm", tile)
    np.testing.assert_array_equal(got, oracle.contract_problem(p))


@pytest.mark.parametrize("tile", WIDE_TILES)
@pytest.mark.parametrize("form", WIDE_FORMS)
def test_wide_tiles_against_method_and_fp64_oracles(form, tile):
    """Shapes of every kind, an odd number of 128-column tiles (the second
    half of the last wide tile missing), ragged K, a long K and a split-K
    shape (few tiles): within the one-accumulator bound of the form's oracle."""
    cases = shapes() + [
        f32(ts.problem("odd_n", "ai", "ib", "ab", dict(a=129, i=45, b=260), 84)),
        f32(ts.problem("one_n", "ai", "ib", "ab", dict(a=300, i=70, b=60), 85)),
        f32(ts.problem("one_m", "ai", "ib", "ab", dict(a=100, i=70, b=390), 86)),
        f32(ts.problem("longk", "ai", "ib", "ab", dict(a=200, i=3000, b=150), 83)),
        f32(ts.problem("splitk", "iajb", "icjd", "abcd",
                       dict(i=60, j=55, a=30, b=8, c=30, d=9), 121)),
    ]
    for p in cases:
        plans = []
        got = run(p, form, "fused_gemm", tile, plan_out=plans)
        assert plans[-1]["tile"] == tile
        mag = magnitude(p)
        acc, _ = tc_bounds(p, form, single=True)
        ok, d = within(got, op.contract_form(p, form), mag, p.C, acc)
        assert ok, (p.name, form, "method", d)
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, acc + SPLIT_ERR[form])
        assert ok, (p.name, form, "fp64", d)


@pytest.mark.parametrize("tile", WIDE_TILES)
def test_wide_tiles_alpha_beta(tile):
    p = f32(ts.direct_gemm_64(n=21))
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    got = run(p, "bf16x3", "fused_gemm", tile)
    acc, _ = tc_bounds(p, "bf16x3", single=True)
    mag = magnitude(p) + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
    assert within(got, op.contract_form(p, "bf16x3"), mag, p.C, acc)[0]


def test_wide_tiles_refuse_the_fp32_class_form_pairs_take_it():
    from paper_1307_2100_gb300 import tc
    p = f32(ts.direct_gemm_64(n=9))
    d = ((p.A.labels, p.A.extents, p.A.strides), (p.B.labels, p.B.extents, p.B.strides),
         (p.C.labels, p.C.extents, p.C.strides))
    # tile 4 keeps one accumulator per chunk; the pairs (tile 5) run BF16x6
    # with the compensated sums of the 128 x 128 kernel
    assert tc.tc_plan_status(*d, tc.TC_F32, tc.MATH["bf16x6"], tc.MAPPING["fused_gemm"], 4) == 5
    assert tc.tc_plan_status(*d, tc.TC_F32, tc.MATH["bf16x6"], tc.MAPPING["fused_gemm"], 5) == 0


@pytest.mark.parametrize("tile", WIDE_TILES)
@pytest.mark.parametrize("form", WIDE_FORMS)
def test_wide_tiles_precision_workload_full_size_sampled(form, tile):
    p = ts.precision_ccd()
    s = random_output_indices(p, 96, seed=3)
    ref64 = sample_outputs(p, s)
    import copy
    pm = copy.copy(p)
    pm.A = copy.copy(p.A)
    pm.B = copy.copy(p.B)
    pm.A.data = np.abs(p.A.data)
    pm.B.data = np.abs(p.B.data)
    mag = sample_outputs(pm, s)
    got = run(p, form, "fused_gemm", tile)
    g = gather(got, p.C, s)
    acc, _ = tc_bounds(p, form, single=True)
    assert np.linalg.norm(g - sample_outputs_form(p, s, form)) <= acc * np.linalg.norm(mag)
    assert np.linalg.norm(g - ref64) <= (acc + SPLIT_ERR[form]) * np.linalg.norm(mag)



# BF16x6 on CTA pairs (tile 5): 256 x 128 tiles, the 128 x 128 kernel's
# compensated chunk sums and separate correction accumulator
def test_bf16x6_pairs_integer_inputs_exact():
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=5), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    plans = []
    got = run(p, "bf16x6", "fused_gemm", 5, plan_out=plans)
    assert plans[-1]["tile"] == 5
    np.testing.assert_array_equal(got, oracle.contract_problem(p))


def test_bf16x6_pairs_against_method_and_fp64_oracles():
    """Every shape kind, an odd number of 128-row tiles (the second CTA of the
    last pair holding no rows of C), one row tile, long K and split-K."""
    cases = shapes() + [
        f32(ts.problem("odd_m", "ai", "ib", "ab", dict(a=390, i=45, b=260), 87)),
        f32(ts.problem("one_m", "ai", "ib", "ab", dict(a=100, i=70, b=390), 86)),
        f32(ts.problem("longk", "ai", "ib", "ab", dict(a=200, i=3000, b=150), 83)),
        f32(ts.problem("splitk", "iajb", "icjd", "abcd",
                       dict(i=60, j=55, a=30, b=8, c=30, d=9), 121)),
    ]
    for p in cases:
        got = run(p, "bf16x6", "fused_gemm", 5)
        mag = magnitude(p)
        acc, tot = tc_bounds(p, "bf16x6")
        ok, d = within(got, op.contract_form(p, "bf16x6"), mag, p.C, acc)
        assert ok, (p.name, "method", d)
        ok, d = within(got, oracle.contract_problem(p), mag, p.C, tot)
        assert ok, (p.name, "fp64", d)


def test_bf16x6_pairs_alpha_beta():
    p = f32(ts.direct_gemm_64(n=21))
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    got = run(p, "bf16x6", "fused_gemm", 5)
    acc, _ = tc_bounds(p, "bf16x6")
    mag = magnitude(p) + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
    assert within(got, op.contract_form(p, "bf16x6"), mag, p.C, acc)[0]


def test_bf16x6_pairs_precision_workload_full_size_fp32_class():
    p = ts.precision_ccd()
    s = random_output_indices(p, 96, seed=3)
    ref64 = sample_outputs(p, s)
    got = run(p, "bf16x6", "fused_gemm", 5)
    g = gather(got, p.C, s)
    assert np.all(np.isfinite(got))
    assert oracle.rel_fro(g, ref64) <= FP32_CLASS


@pytest.mark.parametrize("form", ["bf16", "bf16x3"])
def test_pairs_tail_split(form):
    """80 pair tiles of 256 x 256 on 76 pairs: 76 whole tiles write C, the 4
    tiles of the last round split K in two and a reduction adds their partial
    sums (aligned and ragged shapes); integer inputs stay exact."""
    for dims in (dict(a=2560, i=1024, b=2048), dict(a=2500, i=1100, b=2000)):
        p = f32(ts.problem("tail", "ai", "ib", "ab", dims, 71))
        plans = []
        got = run(p, form, "fused_gemm", 5, plan_out=plans)
        assert plans[0]["tile"] == 5
        acc, _ = tc_bounds(p, form, single=True)
        ok, d = within(got, op.contract_form(p, form), magnitude(p), p.C, acc)
        assert ok, (dims, form, d)
    q = ts.problem("int", "ai", "ib", "ab", dict(a=2500, i=1100, b=2000), 72, dist="int",
                   dtype=np.float32, lo=-2, hi=2)
    np.testing.assert_array_equal(run(q, form, "fused_gemm", 5), oracle.contract_problem(q))
