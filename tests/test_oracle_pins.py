"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each pin is independent of the oracle's code: naive loops written here,
integer arithmetic that is exact in any order, closed forms, the invariances
the paper states, and a brute-force expansion of the sum with itertools.
"""
import copy
import itertools

import numpy as np
import pytest

import oracle
import tcsynth as ts
from tcsynth import lab


def _prob(la, lb, lc, ext, seed=1, dist="uniform", order_a=None, order_b=None, order_c=None,
          lo=-1.0, hi=1.0):
    return ts.problem("t", la, lb, lc, ext, seed, dist, order_a=order_a, order_b=order_b,
                      order_c=order_c, lo=lo, hi=hi)


def _dense(t):
    """Logical dense array (axes in label order) of a tcsynth.Tensor."""
    if t.order == 0:
        return np.array(t.data[0])
    idx = np.zeros(t.extents, dtype=np.int64)
    for ax, (e, s) in enumerate(zip(t.extents, t.strides)):
        shape = [1] * t.order
        shape[ax] = e
        idx = idx + (np.arange(e) * s).reshape(shape)
    return t.data[idx]


def _oracle_dense(p, **kw):
    c = oracle.contract_problem(p, **kw)
    C = copy.copy(p.C)
    C.data = c
    return _dense(C)


def brute_force(p):
    """Expand C[c] = sum_k A*B with itertools over every label value."""
    A, B, C = p.A, p.B, p.C
    ext = {}
    for t in (A, B, C):
        for l, e in zip(t.labels, t.extents):
            ext[l] = e
    con = [l for l in A.labels if l in B.labels]
    out = np.zeros([ext[l] for l in C.labels]) if C.order else np.zeros(())
    Ad, Bd = _dense(A), _dense(B)
    for cidx in itertools.product(*[range(ext[l]) for l in C.labels]):
        val = dict(zip(C.labels, cidx))
        s = 0.0
        for kidx in itertools.product(*[range(ext[l]) for l in con]):
            v = dict(val)
            v.update(zip(con, kidx))
            s += Ad[tuple(v[l] for l in A.labels)] * Bd[tuple(v[l] for l in B.labels)]
        out[cidx] = s
    return out


# --------------------------------------------------------------- naive loops

def test_matrix_product_naive_triple_loop():
    # C[a,b] = sum_i A[a,i] B[i,b] (Sec. 2.2, c_ij = sum_h a_ih b_hj)
    p = _prob("ai", "ib", "ab", dict(a=5, i=7, b=6), seed=3)
    A, B = _dense(p.A), _dense(p.B)
    ref = np.zeros((5, 6))
    for a in range(5):
        for b in range(6):
            s = 0.0
            for i in range(7):
                s += A[a, i] * B[i, b]
            ref[a, b] = s
    np.testing.assert_array_equal(_oracle_dense(p), ref)


def test_matrix_product_four_slicings_agree():
    """Sec. 2.2: GEMVs over rows of A, GEMVs over columns of B, a sum of GERs
    over h, and DOTs over (i, j) all give C = AB."""
    p = _prob("ih", "hj", "ij", dict(i=6, h=9, j=4), seed=4, dist="int", lo=-4, hi=4)
    A, B = _dense(p.A), _dense(p.B)
    m, k = A.shape
    n = B.shape[1]
    s1 = np.stack([A[i, :] @ B for i in range(m)])                  # rows of A
    s2 = np.stack([A @ B[:, j] for j in range(n)], axis=1)          # columns of B
    s3 = sum(np.outer(A[:, h], B[h, :]) for h in range(k))          # GER sum
    s4 = np.array([[A[i, :] @ B[:, j] for j in range(n)] for i in range(m)])  # DOTs
    ref = _oracle_dense(p)
    for s in (s1, s2, s3, s4):
        np.testing.assert_array_equal(s, ref)  # integer data: exact in any order


def test_gemv_and_dot_naive():
    p = _prob("ai", "i", "a", dict(a=9, i=11), seed=5)
    A, x = _dense(p.A), _dense(p.B)
    ref = np.array([sum(A[a, i] * x[i] for i in range(11)) for a in range(9)])
    np.testing.assert_array_equal(_oracle_dense(p), ref)
    q = _prob("i", "i", "", dict(i=13), seed=6)
    u, v = _dense(q.A), _dense(q.B)
    s = 0.0
    for i in range(13):
        s += u[i] * v[i]
    assert _oracle_dense(q) == s


def test_matches_torch_matmul_fp64():
    torch = pytest.importorskip("torch")
    p = _prob("ai", "ib", "ab", dict(a=33, i=17, b=29), seed=7)
    A, B = _dense(p.A), _dense(p.B)
    ref = (torch.from_numpy(A) @ torch.from_numpy(B)).numpy()
    np.testing.assert_allclose(_oracle_dense(p), ref, rtol=1e-13, atol=1e-14)


def test_outer_product_no_contracted_index():
    p = _prob("a", "b", "ab", dict(a=4, b=5), seed=8)
    np.testing.assert_array_equal(_oracle_dense(p), np.outer(_dense(p.A), _dense(p.B)))


# ------------------------------------------------------------ integer exactness

@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny_random_integer_exact(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    p = ts.random_problem(rng, max_order=4, max_ext=3, dist="int")
    p.A.data = np.round(p.A.data * 4)
    p.B.data = np.round(p.B.data * 4)
    got = _oracle_dense(p)
    np.testing.assert_array_equal(got, brute_force(p))


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_tiny_random_float(seed):
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    p = ts.random_problem(rng, max_order=4, max_ext=3)
    np.testing.assert_allclose(_oracle_dense(p), brute_force(p), rtol=1e-13, atol=1e-13)


def test_integer_exact_against_einsum_moderate():
    # entries in {-4..4}: every partial sum is an integer below 2^53, so any
    # summation order gives the same FP64 result
    p = _prob("iajb", "jcid", "abcd", dict(a=5, b=4, c=3, d=6, i=7, j=5), seed=9,
              dist="int", lo=-4, hi=4)
    ref = np.einsum("iajb,jcid->abcd", _dense(p.A), _dense(p.B))
    np.testing.assert_array_equal(_oracle_dense(p), ref)


# ----------------------------------------------------------------- closed forms

def test_all_ones_gives_product_of_contracted_extents():
    p = _prob("aijb", "ijcd", "abcd", dict(a=3, b=2, c=4, d=2, i=5, j=7), dist="ones")
    got = _oracle_dense(p)
    assert np.all(got == 35.0)


def test_rank_one_separable_inputs():
    rng = np.random.Generator(np.random.PCG64(11))
    ext = dict(a=4, i=5, j=3, b=6)
    u = {l: rng.uniform(-1, 1, ext[l]) for l in "aij"}
    v = {l: rng.uniform(-1, 1, ext[l]) for l in "ijb"}
    p = _prob("aij", "jib", "ab", ext)
    Ad = np.einsum("a,i,j->aij", u["a"], u["i"], u["j"])
    Bd = np.einsum("j,i,b->jib", v["j"], v["i"], v["b"])
    p.A.data = Ad.reshape(-1, order="F").copy()
    p.B.data = Bd.reshape(-1, order="F").copy()
    ref = np.outer(u["a"], v["b"]) * (u["i"] @ v["i"]) * (u["j"] @ v["j"])
    np.testing.assert_allclose(_oracle_dense(p), ref, rtol=1e-13, atol=1e-15)


def test_delta_tensor_relabels_the_other_operand_exactly():
    # A[a,i] = delta(a,i): C[a,b,c] = B[a,c,b] relabelled (one nonzero term per sum)
    n = 5
    p = _prob("ai", "icb", "abc", dict(a=n, i=n, b=3, c=4), seed=12)
    p.A.data = np.eye(n).reshape(-1, order="F").copy()
    Bd = _dense(p.B)
    np.testing.assert_array_equal(_oracle_dense(p), np.transpose(Bd, (0, 2, 1)))


# ------------------------------------------------------------------ invariances

def test_operand_order_does_not_matter_bitwise():
    # footnote in Sec. 2.3: once the indices are explicit, T S == S T
    p = _prob("aijb", "jcid", "abdc", dict(a=3, b=4, c=2, d=5, i=6, j=7), seed=13)
    q = copy.copy(p)
    q.A, q.B = p.B, p.A
    np.testing.assert_array_equal(oracle.contract_problem(p), oracle.contract_problem(q))


def test_storage_permutation_is_bitwise_invariant():
    # the same logical tensors stored with different index orders (footnote of
    # Sec. 4.1: transposed storage computes the same R)
    ext = dict(a=3, b=4, c=2, d=5, i=6, j=7)
    p = _prob("iajb", "jcid", "abcd", ext, seed=14)
    q = _prob("iajb", "jcid", "abcd", ext, seed=15, order_a=[2, 0, 3, 1], order_b=[3, 1, 0, 2],
              order_c=[1, 3, 0, 2])
    # copy p's logical values into q's storage
    Ad, Bd = _dense(p.A), _dense(p.B)
    for t, d in ((q.A, Ad), (q.B, Bd)):
        for idx in itertools.product(*[range(e) for e in t.extents]):
            t.data[sum(i * s for i, s in zip(idx, t.strides))] = d[idx]
    np.testing.assert_array_equal(_oracle_dense(p), _oracle_dense(q))


def test_monotone_relabelling_is_bitwise_invariant():
    p = _prob("aijb", "ijcd", "abcd", dict(a=3, b=4, c=2, d=5, i=6, j=7), seed=16)
    q = copy.deepcopy(p)
    remap = lambda ls: [l + 1000 for l in ls]
    q.A.labels, q.B.labels, q.C.labels = remap(p.A.labels), remap(p.B.labels), remap(p.C.labels)
    np.testing.assert_array_equal(oracle.contract_problem(p), oracle.contract_problem(q))


def test_thread_count_does_not_change_result():
    p = _prob("aijb", "ijcd", "abcd", dict(a=6, b=5, c=4, d=3, i=9, j=8), seed=17)
    np.testing.assert_array_equal(oracle.contract_problem(p, nthreads=1),
                                  oracle.contract_problem(p, nthreads=4))


# ------------------------------------------------------------ alpha, beta, edges

def test_alpha_beta_and_beta_zero_never_reads_c():
    p = _prob("ai", "ib", "ab", dict(a=4, i=3, b=5), seed=18)
    base = oracle.contract_problem(p)
    p.C.data[:] = np.nan
    p.alpha, p.beta = 2.0, 0.0
    np.testing.assert_array_equal(oracle.contract_problem(p), 2.0 * base)
    p.C.data[:] = 1.5
    p.beta = -0.5
    np.testing.assert_array_equal(oracle.contract_problem(p), 2.0 * base + (-0.5) * 1.5)


def test_empty_contracted_range_gives_beta_c():
    p = _prob("ai", "ib", "ab", dict(a=3, i=0, b=2), seed=19)
    p.C.data[:] = 7.0
    p.beta = 0.5
    np.testing.assert_array_equal(oracle.contract_problem(p), np.full(6, 3.5))
    p.beta = 0.0
    np.testing.assert_array_equal(oracle.contract_problem(p), np.zeros(6))


def test_empty_output_is_noop_and_scalar_output():
    p = _prob("ai", "ib", "ab", dict(a=0, i=3, b=2), seed=20)
    assert oracle.contract_problem(p).size == 0
    q = _prob("ij", "ji", "", dict(i=3, j=4), seed=21)
    A, B = _dense(q.A), _dense(q.B)
    assert oracle.contract_problem(q)[0] == pytest.approx(float(np.sum(A * B.T)), rel=1e-15)


@pytest.mark.parametrize("la,lb,lc,code", [
    ("aa", "ab", "b", 2),        # repeated label in one tensor
    ("ai", "ib", "a", 2),        # free label of B missing from C
    ("ai", "jb", "ab", 2),       # label in A only, not in C
])
def test_invalid_label_sets_rejected(la, lb, lc, code):
    ext = {l: 3 for l in "abij"}
    with pytest.raises(oracle.OracleError, match=f"status {code}"):
        A = ts.make_tensor(np.random.default_rng(0), la, {ord(k): v for k, v in ext.items()})
        B = ts.make_tensor(np.random.default_rng(0), lb, {ord(k): v for k, v in ext.items()})
        C = ts.empty_output(lc, {ord(k): v for k, v in ext.items()})
        oracle.contract(A, B, C)


def test_extent_mismatch_rejected():
    A = ts.Tensor(lab("ai"), [3, 4], [1, 3], np.zeros(12))
    B = ts.Tensor(lab("ib"), [5, 2], [1, 5], np.zeros(10))
    C = ts.Tensor(lab("ab"), [3, 2], [1, 3], np.zeros(6))
    with pytest.raises(oracle.OracleError, match="status 3"):
        oracle.contract(A, B, C)


def test_batch_labels_are_batched_matrix_products():
    # C[a,b,z] = sum_i A[a,i,z] B[i,b,z]: numpy's batched matmul, slice by slice
    p = _prob("aiz", "ibz", "abz", dict(a=5, i=7, b=4, z=6), seed=31, dist="int", lo=-4, hi=4)
    A = _dense(p.A)
    B = _dense(p.B)
    want = np.einsum("aiz,ibz->abz", A, B)
    got = oracle.contract_problem(p).reshape(p.C.extents, order="F")
    np.testing.assert_array_equal(got, want)
    for z in range(6):
        np.testing.assert_array_equal(got[:, :, z], A[:, :, z] @ B[:, :, z])


def test_hadamard_and_batched_dot():
    p = _prob("ab", "ab", "ab", dict(a=9, b=5), seed=32)   # no contracted label
    np.testing.assert_allclose(oracle.contract_problem(p).reshape(9, 5, order="F"),
                               _dense(p.A) * _dense(p.B), rtol=1e-15)
    q = _prob("iz", "iz", "z", dict(i=50, z=7), seed=33)   # a dot product per z
    np.testing.assert_allclose(oracle.contract_problem(q), np.sum(_dense(q.A) * _dense(q.B), 0),
                               rtol=1e-13)
