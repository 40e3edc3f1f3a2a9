"""GPU parity of the FP64 path against the oracle (through the C ABI).

Tolerance: relative Frobenius error <= 1e-12 (the FP64 bound of the plain
path); integer-valued inputs must agree bit for bit, since every partial sum
is then exact in any order."""
import numpy as np
import pytest

import oracle
import tcsynth as ts
from gpu_util import (TOL_FP64, compare, gather, random_output_indices, run,
                      sample_outputs)

pytestmark = pytest.mark.gpu

GEMM_MAPS = ["auto", "fused_gemm", "slice_gemm", "copy_gemm", "gemv", "dot"]


def small_workloads():
    # the workloads' shapes at sizes spanning several tiles with ragged tails
    return [
        ts.slice_gemm_48(),                                   # config 1 at full size
        ts.direct_gemm_64(n=19),
        ts.fused_permute_48(n=13),
        ts.problem("xy_b_skew", "iajb", "jcid", "abcd",
                   dict(i=33, a=7, j=21, b=3, c=9, d=5), 31),
        ts.problem("gemm_c_from_b", "ai", "ib", "ba", dict(a=70, i=45, b=67), 32),
        ts.problem("tenscase_vi", "ibc", "si", "bcs", dict(i=37, b=11, c=6, s=29), 33),
    ]


@pytest.mark.parametrize("mapping", GEMM_MAPS)
def test_fp64_small_workloads_all_mappings(mapping):
    for p in small_workloads():
        ref = oracle.contract_problem(p)
        got = run(p, "fp64", mapping)
        err = compare(got, ref, p.C)
        assert err <= TOL_FP64, (p.name, mapping, err)


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_fp64_gemm_tiles(tile):
    p = ts.fused_permute_48(n=17)
    ref = oracle.contract_problem(p)
    assert compare(run(p, "fp64", "fused_gemm", tile), ref, p.C) <= TOL_FP64


@pytest.mark.parametrize("mapping", GEMM_MAPS)
def test_fp64_integer_inputs_bitwise(mapping):
    p = ts.problem("int", "iajb", "jcid", "abcd", dict(i=9, a=70, j=11, b=3, c=65, d=2), 41,
                   dist="int", lo=-4, hi=4)
    ref = oracle.contract_problem(p)
    got = run(p, "fp64", mapping)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("seed", range(10))
def test_fp64_random_descriptors(seed):
    rng = np.random.Generator(np.random.PCG64(7000 + seed))
    for _ in range(12):
        p = ts.random_problem(rng, max_order=5, max_ext=6, min_ext=1, max_p=3)
        ref = oracle.contract_problem(p)
        got = run(p, "fp64", "auto")
        assert compare(got, ref, p.C) <= TOL_FP64, (p.A.labels, p.B.labels, p.C.labels)


def test_fp64_alpha_beta_and_nan_output_not_read():
    p = ts.fused_permute_48(n=11)
    base = oracle.contract_problem(p)
    got = run(p, "fp64", "auto", alpha=-0.75, beta=0.0)      # C is NaN-filled
    assert compare(got, -0.75 * base, p.C) <= TOL_FP64
    p.C.data[:] = np.linspace(-1, 1, p.C.data.size)
    p.alpha, p.beta = 0.5, 2.0
    ref = oracle.contract_problem(p)
    for mapping in GEMM_MAPS:
        assert compare(run(p, "fp64", mapping), ref, p.C) <= TOL_FP64, mapping


def test_fp64_edge_cases():
    # empty contracted range: C = beta * C, and zeros for beta == 0
    p = ts.problem("emptyk", "ai", "ib", "ab", dict(a=5, i=0, b=4), 1)
    p.C.data[:] = 3.0
    p.beta = 0.5
    np.testing.assert_array_equal(run(p), np.full(20, 1.5))
    p.beta = 0.0
    np.testing.assert_array_equal(run(p), np.zeros(20))
    # empty output: nothing to do
    q = ts.problem("emptyc", "ai", "ib", "ab", dict(a=0, i=3, b=4), 1)
    assert run(q).size == 0
    # Class 1: scalar result (single-output DOT with a workspace reduction)
    r = ts.problem("class1", "ijk", "kji", "", dict(i=37, j=41, k=53), 2)
    assert compare(run(r), oracle.contract_problem(r), r.C) <= TOL_FP64
    # outer product: no contracted index
    o = ts.problem("outer", "a", "b", "ab", dict(a=77, b=65), 3)
    np.testing.assert_array_equal(run(o), oracle.contract_problem(o))
    # extent-1 indices everywhere
    e = ts.problem("ones", "xaiy", "ziyb", "axbz", dict(x=1, a=20, i=31, y=1, z=1, b=9), 4)
    assert compare(run(e), oracle.contract_problem(e), e.C) <= TOL_FP64
    # maximum order: 12 indices per operand
    la = "abcdefijklmn"
    lb = "ijklmnopqrst"
    lc = "abcdefopqrst"
    m = ts.problem("maxorder", la, lb, lc, {c: 2 for c in set(la + lb)}, 5)
    assert compare(run(m), oracle.contract_problem(m), m.C) <= TOL_FP64


def test_fp64_strided_output_with_gaps():
    p = ts.problem("gaps", "iaj", "jbi", "ab", dict(i=13, a=50, j=7, b=40), 6)
    p.C = ts.Tensor(p.C.labels, p.C.extents, [2, 137], np.full(2 + 49 * 2 + 39 * 137, 9.0))
    ref = oracle.contract_problem(p)
    got = run(p)
    assert compare(got, ref, p.C) <= TOL_FP64
    # the gaps between addressed elements are untouched
    mask = np.ones(got.size, bool)
    from gpu_util import addressed_index
    mask[addressed_index(p.C)] = False
    assert np.all(got[mask] == 9.0)


def test_fp64_full_size_class3_sampled():
    """(i) direct GEMM 64^6 and (ii) fused permute 48^6 at full size, in the
    launch configuration the benchmark times (AUTO mapping, default tile)."""
    for p in (ts.direct_gemm_64(), ts.fused_permute_48()):
        got = run(p, "fp64", "auto")
        s = random_output_indices(p, 64, seed=1)
        ref = sample_outputs(p, s)
        assert oracle.rel_fro(gather(got, p.C, s), ref) <= TOL_FP64, p.name
        assert np.all(np.isfinite(got))


def test_fp64_full_size_gemv_sampled():
    p = ts.gemv_1024_full()
    got = run(p, "fp64", "auto")
    s = random_output_indices(p, 256, seed=2)
    ref = sample_outputs(p, s)
    assert oracle.rel_fro(gather(got, p.C, s), ref) <= TOL_FP64
    assert np.all(np.isfinite(got))


def test_fp64_split_k_long_k():
    """Few output tiles and a long K: the 64 x 64 tiles split K into ranges
    whose partial tiles are summed in order (ragged M, N and K, several
    contracted labels, alpha/beta, the copying mapping)."""
    cases = [ts.problem("sk_ragged", "ai", "ib", "ab", dict(a=130, i=5003, b=70), 61),
             ts.problem("sk_multik", "aijb", "ijc", "abc", dict(a=3, i=41, j=37, b=40, c=67), 62),
             ts.problem("sk_perm", "iajb", "jcid", "abcd",
                        dict(i=45, a=9, j=47, b=7, c=5, d=11), 63)]
    for p in cases:
        info = []
        ref = oracle.contract_problem(p)
        got = run(p, "fp64", "auto", plan_out=info)
        assert info[0]["kernel_name"] == "gemm_simt" and info[0]["workspace"] > 0, info[0]
        assert compare(got, ref, p.C) <= TOL_FP64, p.name
    p = cases[0]
    p.C.data = np.linspace(-3, 3, p.C.data.size)
    p.alpha, p.beta = 0.75, -1.25
    assert compare(run(p, "fp64", "fused_gemm"), oracle.contract_problem(p), p.C) <= TOL_FP64
    p = cases[2]
    assert compare(run(p, "fp64", "copy_gemm"), oracle.contract_problem(p), p.C) <= TOL_FP64


def test_fp64_split_k_at_the_range_cap():
    """One ragged tile and K long enough for the cap of 64 K ranges (K not a
    multiple of the 16-wide K block nor of the range count)."""
    p = ts.problem("sk_cap", "ai", "ib", "ab", dict(a=37, i=40003, b=50), 65)
    info = []
    ref = oracle.contract_problem(p)
    got = run(p, "fp64", "auto", plan_out=info)
    assert info[0]["workspace"] == 64 * 64 * 64 * 8, info[0]
    assert compare(got, ref, p.C) <= TOL_FP64


def test_fp64_split_k_integer_bitwise():
    p = ts.problem("sk_int", "ai", "ib", "ab", dict(a=65, i=4099, b=64), 64,
                   dist="int", lo=-4, hi=4)
    np.testing.assert_array_equal(run(p, "fp64", "fused_gemm"), oracle.contract_problem(p))


def test_16x16_tiles_bitwise_on_integers():
    """Tile configuration 3 (16 x 16, a candidate of the FP64 selector) on
    config 1's shape: bitwise exact on integers."""
    p = ts.slice_gemm_48(dist="int")
    plans = []
    got = run(p, "fp64", "fused_gemm", 3, plan_out=plans)
    assert plans[-1]["kernel"] == 1 and plans[-1]["tile"] == 3
    np.testing.assert_array_equal(got, oracle.contract_problem(p))

