"""GPU parity of the FP8-E4M3 form (per-128-K block power-of-two scales).

Reference: the FP8 oracle (oracle.precision.contract_fp8), which rounds the
same blocks to E4M3 with the same scales (a decision taken on exact FP32
values in both programs, so the E4M3 codes agree bit for bit) and sums the
dequantised products exactly in FP64.  The kernel differs from it only by the
tensor cores' FP32 accumulation (gpu_util.fp8_bound).  A wrong block membership, a wrong
scale or a dropped block changes the result by about 2^-5 relative, far above
that bound, and the block-order case below checks that the test can see it.
Integer inputs in [-4, 4] are exact in every step, so the kernel must then
match the FP64 oracle bit for bit."""
import copy

import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts
from gpu_util import (fp8_bound, gather, magnitude, random_output_indices, run, sample_outputs,
                      sample_outputs_fp8, within)

pytestmark = pytest.mark.gpu

QUANT = 0.13   # FP8 form against the FP64 oracle: E4M3 rounding, <= 2^-4 per factor


def f32(p):
    for t in (p.A, p.B, p.C):
        t.data = t.data.astype(np.float32)
    return p


def shapes():
    return [
        f32(ts.direct_gemm_64(n=23)),                                  # Class 3.2, ragged tiles
        f32(ts.fused_permute_48(n=17)),                                # Class 3.1, gathered K
        f32(ts.problem("m1", "ai", "ib", "ab", dict(a=300, i=200, b=130), 51)),
        f32(ts.problem("cfromb", "ai", "ib", "ba", dict(a=140, i=77, b=260), 52)),
        f32(ts.problem("longk", "aijb", "ijc", "abc", dict(a=130, i=40, j=60, b=2, c=129), 53)),
        f32(ts.precision_ccd(v=24, o=20)),
    ]


def test_fp8_integer_inputs_exact():
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=29, a=70, j=11, b=3, c=65, d=2), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    got = run(p, "fp8", "auto")
    np.testing.assert_array_equal(got, oracle.contract_problem(p))


@pytest.mark.parametrize("k", range(6))
def test_fp8_against_fp8_oracle(k):
    p = shapes()[k]
    got = run(p, "fp8", "auto")
    mag = magnitude(p)
    ok, d = within(got, op.contract_fp8(p), mag, p.C, fp8_bound(p))
    assert ok, (p.name, d)
    ok, d = within(got, oracle.contract_problem(p), mag, p.C, QUANT)
    assert ok, (p.name, d)


def test_fp8_alpha_beta():
    p = f32(ts.direct_gemm_64(n=21))
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    got = run(p, "fp8", "auto")
    mag = magnitude(p) + abs(p.beta) * np.abs(p.C.data.astype(np.float64))
    assert within(got, op.contract_fp8(p), mag, p.C, fp8_bound(p))[0]


def test_fp8_block_order_follows_a():
    """The kernel's first operand is B here (C's stride-1 index is B's), and A
    is stored in two layouts whose stride order of the contracted i, j
    differs: each run matches the oracle of its own layout, and the two
    oracles differ by far more than the bound (so the order is observable)."""
    base = f32(ts.problem("kord", "aij", "jib", "ba", dict(a=150, i=20, j=30, b=140), 71))
    # A is 2^20 larger (B 2^-30 smaller) at j = 0: a block holding such an
    # element rounds its other elements (2^-12 of its scale) to zero.  With i
    # fastest those elements fill part of one block, with j fastest one in 30
    # elements of every block.
    Av = base.A.data.reshape(150, 20, 30, order="F").copy()
    Av[:, :, 0] *= np.float32(2.0 ** 20)
    base.A.data = Av.reshape(-1, order="F")
    Bv = base.B.data.reshape(30, 20, 140, order="F").copy()
    Bv[0] *= np.float32(2.0 ** -30)
    base.B.data = Bv.reshape(-1, order="F")
    # the same A values stored with j varying faster than i
    alt = copy.deepcopy(base)
    ext = dict(zip(base.A.labels, base.A.extents))
    a, i, j = base.A.labels
    st = {a: 1, j: ext[a], i: ext[a] * ext[j]}
    alt.A.strides = [st[l] for l in base.A.labels]
    ia, ii, jj = np.meshgrid(np.arange(ext[a]), np.arange(ext[i]), np.arange(ext[j]),
                             indexing="ij")
    sa0, si0, sj0 = base.A.strides
    vals = np.zeros(ts.span(alt.A.extents, alt.A.strides), np.float32)
    vals[ia * st[a] + ii * st[i] + jj * st[j]] = base.A.data[ia * sa0 + ii * si0 + jj * sj0]
    alt.A.data = vals
    assert op.k_order(base) != op.k_order(alt)
    mag = magnitude(base)
    r_base, r_alt = op.contract_fp8(base), op.contract_fp8(alt)
    assert not within(r_base, r_alt, mag, base.C, 10 * fp8_bound(base))[0]
    for p, ref in ((base, r_base), (alt, r_alt)):
        info = []
        got = run(p, "fp8", "auto", plan_out=info)
        assert info[0]["swapped"] == 1
        ok, d = within(got, ref, mag, p.C, fp8_bound(p))
        assert ok, (op.k_order(p), d)


def test_fp8_wide_dynamic_range():
    """Block exponents from about -60 to +60, blocks of zeros, and values that
    round to E4M3 subnormals within their block."""
    p = f32(ts.problem("range", "aijb", "ijc", "abc", dict(a=130, i=64, j=6, b=2, c=129), 73))
    rng = np.random.default_rng(5)
    A = p.A.data.astype(np.float64).reshape(p.A.extents, order="F")
    A *= np.exp2(rng.integers(-60, 60, size=(1, 1, 6, 1)))          # per K block (64*2 = 128)
    A[:7] = 0.0                                                     # zero rows
    A[:, :, :, 1] *= np.where(rng.random((130, 64, 6)) < 0.2, 2.0 ** -12, 1.0)
    p.A.data = A.reshape(-1, order="F").astype(np.float32)
    got = run(p, "fp8", "auto")
    ok, d = within(got, op.contract_fp8(p), magnitude(p), p.C, fp8_bound(p))
    assert ok, d


def test_fp8_empty_and_degenerate():
    # K = 1 (one ragged block), M = 3 (one ragged tile)
    for p in (f32(ts.problem("k1", "ai", "ib", "ab", dict(a=200, i=1, b=150), 74)),
              f32(ts.problem("m3", "ai", "ib", "ab", dict(a=3, i=300, b=150), 75))):
        got = run(p, "fp8", "fused_gemm")
        assert within(got, op.contract_fp8(p), magnitude(p), p.C, fp8_bound(p))[0], p.name
    # M = 1 makes it Class 2, which has no FP8 form
    from paper_1307_2100_gb300 import tc
    with pytest.raises(tc.TcError) as e:
        run(f32(ts.problem("m1", "ai", "ib", "ab", dict(a=1, i=300, b=150), 75)), "fp8")
    assert e.value.status == 5
    # K = 0: C = beta * C
    p = f32(ts.problem("k0", "ai", "ib", "ab", dict(a=20, i=0, b=15), 76))
    p.C.data = np.ones(p.C.data.size, np.float32)
    p.beta = 2.0
    np.testing.assert_array_equal(run(p, "fp8", "auto"), 2.0 * np.ones(p.C.data.size))


def test_fp8_precision_workload_full_size_sampled():
    """C[a,b,i,j] = sum_{e,f} A[a,b,e,f] B[e,f,i,j], a=b=e=f=128, i=j=32 (FP32
    storage; the bench's precision workload) at full size: sampled outputs
    against the FP8 oracle and the FP64 oracle."""
    p = ts.precision_ccd()
    s = random_output_indices(p, 96, seed=4)
    ref64 = sample_outputs(p, s)
    pm = copy.copy(p)
    pm.A = copy.copy(p.A)
    pm.B = copy.copy(p.B)
    pm.A.data = np.abs(p.A.data)
    pm.B.data = np.abs(p.B.data)
    mag = sample_outputs(pm, s)
    got = run(p, "fp8", "auto")
    assert np.all(np.isfinite(got))
    g = gather(got, p.C, s)
    assert np.linalg.norm(g - sample_outputs_fp8(p, s)) <= fp8_bound(p) * np.linalg.norm(mag)
    assert np.linalg.norm(g - ref64) <= QUANT * np.linalg.norm(mag)


# Tile configuration 1: the first operand packed inside the GEMM launch.  Its
# pack warps produce the same E4M3 codes and scale bytes as the packing pass
# and the MMAs run in the same order, so C must equal tile 0's bit for bit.
def fusable(k):
    return [
        lambda: f32(ts.problem("m1", "ai", "ib", "ab", dict(a=300, i=200, b=130), 51)),
        lambda: f32(ts.precision_ccd(v=24, o=20)),                     # merged M and K labels
        lambda: f32(ts.problem("longk", "ai", "ib", "ab", dict(a=132, i=3000, b=140), 56)),
        lambda: f32(ts.problem("wide_n", "ai", "ib", "ab", dict(a=260, i=130, b=2100), 57)),
    ][k]()


@pytest.mark.parametrize("k", range(4))
def test_fp8_in_kernel_packing_matches_the_packing_pass(k):
    p = fusable(k)
    info = []
    got1 = run(p, "fp8", "fused_gemm", tile=1, plan_out=info)
    assert info[0]["tile"] == 1
    np.testing.assert_array_equal(got1, run(p, "fp8", "fused_gemm", tile=0))
    ok, d = within(got1, op.contract_fp8(p), magnitude(p), p.C, fp8_bound(p))
    assert ok, (p.name, d)


def test_fp8_in_kernel_packing_alpha_beta_and_integers():
    p = fusable(0)
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    np.testing.assert_array_equal(run(p, "fp8", "fused_gemm", tile=1),
                                  run(p, "fp8", "fused_gemm", tile=0))
    q = ts.problem("int", "ai", "ib", "ab", dict(a=300, i=200, b=130), 62, dist="int",
                   dtype=np.float32, lo=-4, hi=4)
    np.testing.assert_array_equal(run(q, "fp8", "fused_gemm", tile=1), oracle.contract_problem(q))


def test_fp8_in_kernel_packing_over_several_groups():
    """200 row tiles of A and one pair of column tiles: 200 GEMM tiles on at
    most 152 CTAs, so the pack units come in two groups and the second wave
    of tiles waits on the second group."""
    p = f32(ts.problem("groups", "ai", "ib", "ab", dict(a=25600, i=264, b=200), 58))
    np.testing.assert_array_equal(run(p, "fp8", "fused_gemm", tile=1),
                                  run(p, "fp8", "fused_gemm", tile=0))


# Tile configuration 2: CTA pairs over 256 x 256 tiles.  The same E4M3 codes
# and scale bytes, and for each output the same block-scaled MMAs in the same
# K order, so C must equal the 128 x 256 tiles' (tile 0) bit for bit.
def pair_shapes(k):
    return [
        lambda: f32(ts.problem("m1", "ai", "ib", "ab", dict(a=300, i=200, b=130), 51)),  # odd pair row
        lambda: f32(ts.problem("wide_n", "ai", "ib", "ab", dict(a=260, i=130, b=2100), 57)),  # 17 col tiles
        lambda: f32(ts.direct_gemm_64(n=23)),                                # gathered groups
        lambda: f32(ts.problem("cfromb", "ai", "ib", "ba", dict(a=140, i=77, b=260), 52)),
        lambda: f32(ts.problem("longk", "aijb", "ijc", "abc", dict(a=130, i=40, j=60, b=2, c=129), 53)),
    ][k]()


@pytest.mark.parametrize("k", range(5))
def test_fp8_pairs_match_the_one_cta_tiles(k):
    p = pair_shapes(k)
    info = []
    got2 = run(p, "fp8", "fused_gemm", tile=2, plan_out=info)
    assert info[0]["tile"] == 2
    np.testing.assert_array_equal(got2, run(p, "fp8", "fused_gemm", tile=0))
    ok, d = within(got2, op.contract_fp8(p), magnitude(p), p.C, fp8_bound(p))
    assert ok, (p.name, d)


def test_fp8_pairs_alpha_beta_and_integers():
    p = pair_shapes(0)
    p.C.data = np.linspace(-2, 2, p.C.data.size).astype(np.float32)
    p.alpha, p.beta = -1.5, 0.25
    np.testing.assert_array_equal(run(p, "fp8", "fused_gemm", tile=2),
                                  run(p, "fp8", "fused_gemm", tile=0))
    q = ts.problem("int", "iajb", "jcid", "abcd", dict(i=29, a=70, j=11, b=3, c=65, d=2), 61,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    np.testing.assert_array_equal(run(q, "fp8", "fused_gemm", tile=2), oracle.contract_problem(q))
