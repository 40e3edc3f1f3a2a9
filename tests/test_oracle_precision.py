"""Pins of the reduced-precision oracle (BF16 rounding and split terms, E4M3)."""
import copy

import numpy as np
import pytest

import oracle
from oracle import precision as op
import tcsynth as ts


def f32(x):
    return np.asarray(x, dtype=np.float32)


def test_bf16_rounding_ties_to_even_hand_values():
    one = 1.0
    ulp = 2.0 ** -7                     # BF16 spacing just above 1
    cases = {
        one + ulp / 2: one,             # halfway, 1.0 has even significand
        one + 3 * ulp / 2: one + 2 * ulp,   # halfway, rounds to the even neighbour
        one + ulp / 2 + 2.0 ** -20: one + ulp,  # just above halfway
        one + ulp / 2 - 2.0 ** -20: one,        # just below halfway
        -(one + 3 * ulp / 2): -(one + 2 * ulp),
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert float(op.bf16_rne(f32([x]))[0]) == want, x


def test_bf16_values_have_zero_low_bits_and_are_nearest():
    rng = np.random.default_rng(1)
    x = f32(rng.standard_normal(20000) * np.exp2(rng.integers(-20, 20, 20000)))
    r = op.bf16_rne(x)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    # nearest: no BF16 value (the two neighbours of r) is strictly closer
    rb = r.view(np.uint32)
    up = (rb + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    dn = (rb - np.uint32(0x10000)).view(np.float32).astype(np.float64)
    d = np.abs(x.astype(np.float64) - r)
    assert np.all(d <= np.abs(x - up)) and np.all(d <= np.abs(x - dn))
    assert np.all(d <= np.abs(x.astype(np.float64)) * 2.0 ** -8)


def test_three_bf16_terms_reconstruct_fp32_exactly():
    rng = np.random.default_rng(2)
    x = f32(rng.standard_normal(50000) * np.exp2(rng.integers(-30, 30, 50000)))
    t0, t1, t2 = op.split_bf16(x, 3)
    s = t0.astype(np.float64) + t1.astype(np.float64) + t2.astype(np.float64)
    np.testing.assert_array_equal(s, x.astype(np.float64))
    # each residual is at most half an ulp of the previous term
    assert np.all(np.abs(t1) <= np.abs(t0) * 2.0 ** -8)
    assert np.all(np.abs(t2) <= np.abs(t1) * 2.0 ** -8)


def test_two_term_split_error_bound():
    rng = np.random.default_rng(3)
    x = f32(rng.uniform(-1, 1, 10000))
    t0, t1 = op.split_bf16(x, 2)
    err = np.abs(x.astype(np.float64) - t0 - t1.astype(np.float64))
    assert np.all(err <= np.abs(x) * 2.0 ** -16)


def test_forms_error_ordering_on_small_contraction():
    p = ts.precision_ccd(v=16, o=8)
    ref = oracle.contract_problem(p)
    errs = {f: oracle.rel_fro(op.contract_form(p, f), ref) for f in ("bf16", "bf16x3", "bf16x6")}
    assert 1e-4 < errs["bf16"] < 1e-2
    assert errs["bf16x3"] < 1e-4
    assert errs["bf16x6"] < 1e-6
    assert errs["bf16x6"] < errs["bf16x3"] < errs["bf16"]


def test_bf16_form_on_bf16_integers_is_exact():
    # integers in [-4, 4] are BF16 values: every form equals the exact result
    p = ts.problem("t", "aijb", "ijcd", "abcd", dict(a=3, b=4, c=5, d=2, i=6, j=7), 3,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    ref = oracle.contract_problem(p)
    for f in ("bf16", "bf16x3", "bf16x6"):
        np.testing.assert_array_equal(op.contract_form(p, f), ref)


def test_e4m3_table():
    vals, codes = op.e4m3_values()
    assert len(vals) == 127
    assert vals.max() == 448.0
    assert vals[1] == 2.0 ** -9          # smallest subnormal
    assert 2.0 ** -6 in set(vals)        # smallest normal
    assert np.all(np.diff(vals) > 0)


def test_e4m3_rounding_hand_values():
    q = op.e4m3_rne
    assert q(1.0 + 1 / 16)[()] == 1.0          # halfway between 1 and 1.125: even code
    assert q(1.0 + 3 / 16)[()] == 1.25         # halfway between 1.125 and 1.25: even
    assert q(500.0)[()] == 448.0               # saturation
    assert q(-1e9)[()] == -448.0
    assert q(2.0 ** -10)[()] == 0.0            # half of smallest subnormal ties to 0
    assert q(3 * 2.0 ** -10)[()] == 2.0 ** -8  # 1.5 subnormal ulps ties to the even code 2


def test_pow2_scale_exponent():
    for amax in (448.0, 449.0, 1.0, 0.001, 1e5, 896.0, 2.0 ** -100, 3.4e38):
        e = int(op.pow2_scale_exponent(amax))
        assert amax / 2.0 ** e <= 448.0 < amax / 2.0 ** (e - 1)
    # the floor: zero and tiny maxima
    assert int(op.pow2_scale_exponent(0.0)) == -126
    assert int(op.pow2_scale_exponent(2.0 ** -140)) == -126
    assert int(op.pow2_scale_exponent(448 * 2.0 ** -126)) == -126
    assert int(op.pow2_scale_exponent(449 * 2.0 ** -126)) == -125


def test_block_quantisation_error():
    rng = np.random.default_rng(4)
    m = rng.standard_normal((8, 300))
    dq, e = op.quantize_rows_e4m3(m)
    assert e.shape == (8, 3)
    assert np.max(np.abs(dq - m) / np.maximum(np.abs(m), 2.0 ** -6 * np.exp2(e.max()))) < 0.07


def test_gemm_view_reproduces_the_contraction():
    p = ts.problem("v", "iajb", "jcid", "abcd", dict(i=5, a=3, j=4, b=2, c=3, d=2), 9)
    Am, Bm, fa, fb, kl = op.gemm_view(p)
    assert kl == ts.lab("ij")                      # ascending stride in A
    ref = oracle.contract_problem(p)
    Cm = Am @ Bm
    # C is column-major over (a,b,c,d) = (free A, free B): same flattening
    np.testing.assert_allclose(Cm.reshape(-1, order="F"), ref, rtol=1e-13)


def test_fp8_form_is_exact_on_small_integers():
    # |x| <= 4 integers: the block scale is 2^-6 and 64 * x is an E4M3 value
    p = ts.problem("i8", "aijb", "ijc", "abc", dict(a=7, i=40, j=9, b=3, c=11), 10,
                   dist="int", dtype=np.float32, lo=-4, hi=4)
    np.testing.assert_array_equal(op.contract_fp8(p), oracle.contract_problem(p))


def test_fp8_form_scale_equivariance_and_error():
    p = ts.precision_ccd(v=16, o=8)
    base = op.contract_fp8(p)
    q = copy.deepcopy(p)
    q.A.data = (p.A.data * np.float32(2.0 ** 5)).astype(np.float32)
    np.testing.assert_array_equal(op.contract_fp8(q), base * 2.0 ** 5)
    err = oracle.rel_fro(base, oracle.contract_problem(p))
    assert 1e-4 < err < 6e-2


# ----------------------------------------------------------- binary16 (FP16)

def test_f16_value_table_edges():
    vals, codes = op.f16_values()
    assert len(vals) == 0x7C00 == 31744            # every finite non-negative code
    assert np.all(np.diff(vals) > 0)                # codes increase with value
    assert vals[1] == 2.0 ** -24                    # smallest subnormal
    assert vals[0x3FF] == 1023 / 1024 * 2.0 ** -14  # largest subnormal
    assert vals[0x400] == 2.0 ** -14                # smallest normal
    assert vals[0x3C00] == 1.0 and vals[0x3C01] == 1.0 + 2.0 ** -10
    assert vals[-1] == op.F16_MAX == 65504.0


def test_f16_rounding_ties_to_even_hand_values():
    cases = {
        1.0 + 2.0 ** -11: 1.0,                    # halfway: 1.0 has the even code
        1.0 + 3 * 2.0 ** -11: 1.0 + 2.0 ** -9,    # halfway: up to the even code
        1.0 + 2.0 ** -11 + 2.0 ** -20: 1.0 + 2.0 ** -10,
        2049.0: 2048.0,                           # spacing 2 above 2048
        2051.0: 2052.0,
        2.0 ** -25: 0.0,                          # halfway between 0 and 2^-24
        3 * 2.0 ** -25: 2.0 ** -23,               # halfway between codes 1 and 2
        65519.0: 65504.0,                         # below the overflow midpoint
        65520.0: np.inf,                          # the midpoint itself: to infinity
        -70000.0: -np.inf,
        -(1.0 + 3 * 2.0 ** -11): -(1.0 + 2.0 ** -9),
    }
    for x, want in cases.items():
        assert float(op.f16_rne([x])[0]) == want, x


def test_f16_rounding_matches_numpy_float16_conversion():
    """numpy's float32 -> float16 cast is IEEE round-to-nearest-even: an
    independent implementation to compare with, across the subnormal range,
    the normal range and overflow."""
    rng = np.random.default_rng(16)
    x = f32(rng.standard_normal(100000) * np.exp2(rng.uniform(-30, 17.5, 100000)))
    ref = x.astype(np.float16).astype(np.float64)
    got = op.f16_rne(x)
    np.testing.assert_array_equal(got, ref)


def test_f16_form_exact_on_f16_integers_and_rounds_otherwise():
    # integers up to 2048 are binary16 values: the form equals the contraction
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=5, a=7, j=3, b=2, c=6, d=3), 61,
                   dist="int", lo=-8, hi=8, dtype=np.float32)
    np.testing.assert_array_equal(op.contract_f16(p), oracle.contract_problem(p))
    # general FP32 data: the result is the contraction of the rounded values,
    # within the binary16 input rounding (2^-11 relative per operand) of it
    q = ts.problem("u", "aik", "kib", "ab", dict(a=9, i=11, k=7, b=8), 62, dtype=np.float32)
    exact = oracle.contract_problem(q)
    form = op.contract_f16(q)
    err = oracle.rel_fro(form, exact)
    assert 0 < err <= 2 * 2.0 ** -11
