"""Host-side tests of libtc.so (no GPU needed): exported symbols, the planner's
classification against the classification oracle, error statuses and the
GEMM views built for the workloads."""
import glob
import json
import os
import re

import numpy as np
import pytest

import tcsynth as ts
from oracle import classify as oc

tc = pytest.importorskip("paper_1307_2100_gb300.tc")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = re.sub(r"#[^\n]*", "", src)
        names |= set(re.findall(r"\b(tc_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_function():
    names = declared_functions()
    assert "tc_plan" in names and "tc_contract" in names
    missing = [n for n in names if not hasattr(tc.lib, n)]
    assert not missing, missing


def _t(t):
    return (t.labels, t.extents, t.strides)


def plan_info(p, math=0, mapping=0, tile=-1, dtype=None):
    dt = tc.TC_F64 if dtype is None else dtype
    h = tc.tc_plan(_t(p.A), _t(p.B), _t(p.C), dt, math, mapping, tile)
    try:
        return tc.tc_plan_get_info(h)
    finally:
        tc.tc_plan_destroy(h)


def bits(v):
    return sum(1 << i for i, x in enumerate(v) if x)


@pytest.mark.parametrize("seed", range(6))
def test_planner_classification_matches_oracle(seed):
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    for _ in range(300):
        p = ts.random_problem(rng, max_order=5, max_ext=4, min_ext=1, max_p=3)
        info = plan_info(p)
        r = oc.classify(p.A, p.B, p.C)
        assert info.cls == r.cls
        assert (info.p, info.delta_a, info.delta_b) == (r.p, r.delta_a, r.delta_b)
        assert info.stride1_a == (r.stride1_a if r.stride1_a is not None else -1)
        assert info.stride1_b == (r.stride1_b if r.stride1_b is not None else -1)
        assert info.slice_a == bits(r.slice_a), (p.A.labels, p.B.labels, p.C.labels)
        assert info.slice_b == bits(r.slice_b)


def test_planner_on_paper_cases():
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "classification_cases.json")))
    names = {}
    for case in gold["cases"]:
        def mk(ls, out=False):
            labels = [names.setdefault(x, len(names) + 1) for x in ls]
            ext = [5] * len(labels)
            data = np.zeros(ts.span(ext, ts.col_major(ext)))
            return ts.Tensor(labels, ext, ts.col_major(ext), data)
        A, B, C = mk(case["A"]), mk(case["B"]), mk(case["C"])
        info = plan_info(ts.Problem(case["name"], A, B, C))
        assert info.cls == case["cls"], case["cite"]
        r = oc.classify(A, B, C)
        assert info.slice_a == bits(r.slice_a) and info.slice_b == bits(r.slice_b)


def test_gemm_views_of_the_workloads():
    i1 = plan_info(ts.slice_gemm_48())
    assert (i1.cls, i1.M, i1.N, i1.K, i1.batch) == (32, 48 * 48, 48, 48, 1)
    s1 = plan_info(ts.slice_gemm_48(), mapping=tc.MAPPING["slice_gemm"])
    assert (s1.M, s1.N, s1.K, s1.batch) == (48, 48, 48, 48)
    d = plan_info(ts.direct_gemm_64())
    assert (d.cls, d.M, d.N, d.K) == (32, 64 * 64, 64 * 64, 64 * 64)
    f = plan_info(ts.fused_permute_48())
    assert (f.cls, f.M, f.N, f.K) == (31, 48 * 48, 48 * 48, 48 * 48)
    c = plan_info(ts.fused_permute_48(), mapping=tc.MAPPING["copy_gemm"])
    assert c.workspace >= 48 ** 4 * 8
    g = plan_info(ts.gemv_1024())
    assert (g.cls, g.kernel, g.M, g.N, g.K) == (2, 3, 1024 * 1024, 1, 2048)
    assert g.flops == 2.0 * 1024 * 1024 * 2048


def test_class1_dot_needs_workspace():
    p = ts.problem("dot", "ij", "ji", "", dict(i=50, j=40), 1)
    info = plan_info(p)
    assert info.cls == 1 and info.kernel == 4 and info.workspace > 0


E = dict(a=3, b=4, i=5, j=6)


def _desc(ls, strides=None):
    labels = ts.lab(ls)
    ext = [E[c] for c in ls]
    return (labels, ext, strides)


@pytest.mark.parametrize("A,B,C,code", [
    (_desc("ai"), _desc("jb"), _desc("ab"), 2),           # label in neither C nor B
    (_desc("ai"), _desc("ib"), _desc("a"), 2),            # free label of B not in C
    (_desc("aa"), _desc("ab"), _desc("b"), 2),            # repeated label
    (_desc("ai", [1, -3]), _desc("ib"), _desc("ab"), 4),  # negative stride
    (_desc("ai", [0, 3]), _desc("ib"), _desc("ab"), 4),   # zero stride, extent > 1
    (_desc("ai"), _desc("ib"), _desc("ab", [1, 1]), 4),   # aliasing output
])
def test_plan_rejects_invalid_descriptors(A, B, C, code):
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0) == code


def test_plan_rejects_extent_mismatch_and_bad_enums():
    A = (ts.lab("ai"), [3, 5], None)
    B = (ts.lab("ib"), [6, 4], None)
    C = (ts.lab("ab"), [3, 4], None)
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0) == 3
    B = (ts.lab("ib"), [5, 4], None)
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0) == 0
    assert tc.tc_plan_status(A, B, C, 7, 0) == 1             # bad dtype
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 9) == 1     # bad math
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 2) == 5     # FP64 storage, BF16 math
    assert tc.tc_plan_status(A, B, C, tc.TC_F32, 0) == 5     # FP32 storage, FP64 math
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0, 42) == 1  # bad mapping
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0, 0, 99) == 5  # bad tile
    x = (ts.lab("i"), [5], None)
    # SLICE_GEMM and COPY_GEMM exist only for Class 3
    assert tc.tc_plan_status(A, x, (ts.lab("a"), [3], None), tc.TC_F64, 0,
                             tc.MAPPING["slice_gemm"]) == 5


def test_order_limit():
    n = tc.MAX_ORDER + 1
    A = (list(range(1, n + 1)), [1] * n, None)
    assert tc.tc_plan_status(A, A, ([], [], None), tc.TC_F64, 0) == 1


def test_contract_host_checks_before_any_launch():
    h = tc.tc_plan(_desc("ij"), (ts.lab("ji"), [6, 5], None), ([], [], None), tc.TC_F64, 0)
    try:
        with pytest.raises(tc.TcError) as e:
            tc.tc_contract(h, 1.0, 16, 16, 0.0, 16, 0, 0, 0)   # no workspace given
        assert e.value.status == 6
        with pytest.raises(tc.TcError) as e:
            tc.tc_contract(0, 1.0, 16, 16, 0.0, 16)
        assert e.value.status == 1
    finally:
        tc.tc_plan_destroy(h)


def test_status_strings():
    assert tc.tc_status_string(0) == "ok"
    assert "timed out" in tc.tc_status_string(8)


def test_fp8_plans():
    p = ts.fused_permute_48(n=40)                       # Class 3.1: M=N=K=1600
    info = plan_info(p, tc.MATH["fp8"], dtype=tc.TC_F32)
    assert tc.KERNEL_NAME[info.kernel] == "gemm_fp8"
    assert tc.MAPPING_NAME[info.mapping] == "fused_gemm"
    tm, tn, nkb = -(-info.M // 128), -(-info.N // 128), -(-info.K // 128)
    ng = -(-nkb // 4)                                   # scale bytes: 512 per 4 blocks
    r = lambda x: -(-x // 256) * 256
    want = r(tm * nkb * 16384) + r(tn * nkb * 16384) + r(tm * ng * 512) + r(tn * ng * 512)
    want += r(16 + tm * nkb * 4)                        # in-kernel packing: claim counter, counts
    assert info.workspace == want
    f8 = tc.MATH["fp8"]
    x = (ts.lab("i"), [5], None)
    A = (ts.lab("ai"), [3, 5], None)
    # one block-scaled GEMM: Class 3 and the fused mapping only; FP32 storage only
    assert tc.tc_plan_status(A, x, (ts.lab("a"), [3], None), tc.TC_F32, f8) == 5
    assert tc.tc_plan_status(x, x, ([], [], None), tc.TC_F32, f8) == 5
    B = (ts.lab("ib"), [5, 4], None)
    C = (ts.lab("ab"), [3, 4], None)
    assert tc.tc_plan_status(A, B, C, tc.TC_F32, f8) == 0
    assert tc.tc_plan_status(A, B, C, tc.TC_F64, f8) == 5
    for m in ("slice_gemm", "copy_gemm", "gemv", "dot"):
        assert tc.tc_plan_status(A, B, C, tc.TC_F32, f8, tc.MAPPING[m]) == 5
    # a workspace that is not 16-byte aligned is refused before any launch
    h = tc.tc_plan(A, B, C, tc.TC_F32, f8)
    try:
        ws = tc.tc_plan_get_info(h).workspace
        with pytest.raises(tc.TcError) as e:
            tc.tc_contract(h, 1.0, 256, 256, 0.0, 256, 4104, ws)
        assert e.value.status == 1
    finally:
        tc.tc_plan_destroy(h)


def test_fp8_k_order_follows_a_whichever_operand_is_first():
    # C's stride-1 index b is B's: the kernel's first operand is B, yet the
    # contracted indices keep A's stride order (i before j) for the scale blocks
    p = ts.problem("kord", "aij", "jib", "ba", dict(a=150, i=20, j=30, b=140), 71)
    info = plan_info(p, tc.MATH["fp8"], dtype=tc.TC_F32)
    assert info.swapped == 1 and info.K == 600


def test_tensor_core_tile_defaults():
    # one GEMM: packed operands on CTA pairs (tile 5: M spans two row tiles)
    # with a workspace; a batch of GEMMs (the slicing mapping): the gathering
    # kernel, no workspace
    p = ts.fused_permute_48(n=40)
    bf = tc.MATH["bf16x6"]
    info = plan_info(p, bf, dtype=tc.TC_F32)
    assert info.tile == 5 and info.batch == 1 and info.M > 128
    tm, tn, nkb = -(-info.M // 128), -(-info.N // 128), -(-info.K // 32)
    r = lambda x: -(-x // 256) * 256
    assert info.workspace == r(tm * nkb * 3 * 8192) + r(tn * nkb * 3 * 8192)
    s = ts.slice_gemm_48()
    info = plan_info(s, bf, tc.MAPPING["slice_gemm"], dtype=tc.TC_F32)
    assert info.batch > 1 and info.tile == 0 and info.workspace == 0
    assert tc.tc_plan_status(_t(s.A), _t(s.B), _t(s.C), tc.TC_F32, bf,
                             tc.MAPPING["slice_gemm"], 3) == 5


def test_fp64_split_k_workspace():
    # FP64 on the CUDA cores with fewer 64 x 64 tiles than SMs and a long K:
    # min(floor(2 * 152 / tiles), K blocks of 16 / 32, 64) ranges, each with
    # FP64 partial tiles in the workspace; other tiles, dtypes, shapes: none
    p = ts.problem("sk", "ai", "ib", "ab", dict(a=130, i=5003, b=70), 61)
    info = plan_info(p)
    tiles = 3 * 2
    ks = min(304 // tiles, (5003 + 15) // 16 // 32, 64)
    assert info.kernel == 1 and info.tile == 0 and ks == 9
    assert info.workspace == ks * tiles * 64 * 64 * 8
    for tile in (1, 2):
        assert plan_info(p, tile=tile).workspace == 0
    assert plan_info(p, tc.MATH["fp32"], dtype=tc.TC_F32).workspace == 0
    short = ts.problem("sk_short", "ai", "ib", "ab", dict(a=130, i=900, b=70), 61)
    assert plan_info(short).workspace == 0          # under 64 K blocks: one range
    wide = ts.problem("sk_wide", "ai", "ib", "ab", dict(a=1100, i=5003, b=1100), 61)
    assert plan_info(wide).workspace == 0           # 18 x 18 tiles fill the GPU
    cap = ts.problem("sk_cap", "ai", "ib", "ab", dict(a=37, i=40003, b=50), 65)
    assert plan_info(cap).workspace == 64 * 1 * 64 * 64 * 8   # at most 64 ranges


def test_batch_routes_are_checked_before_any_allocation():
    bf = tc.MATH["bf16x6"]
    p = ts.fused_permute_48(n=6)
    s = ts.slice_gemm_48()
    h1 = tc.tc_plan(_t(p.A), _t(p.B), _t(p.C), tc.TC_F32, bf)
    h2 = tc.tc_plan(_t(s.A), _t(s.B), _t(s.C), tc.TC_F32, bf, tc.MAPPING["slice_gemm"])
    try:
        for bad in ([4, -1], [-2, 0]):
            with pytest.raises(tc.TcError) as e:
                tc.tc_batch_plan_routes([h1, h2], bad)
            assert e.value.status == 1
        # the slicing mapping's batch group cannot take the tensor-core route
        with pytest.raises(tc.TcError) as e:
            tc.tc_batch_plan_routes([h1, h2], [-1, 1])
        assert e.value.status == 5
    finally:
        tc.tc_plan_destroy(h1)
        tc.tc_plan_destroy(h2)


def test_autotune_buckets():
    from paper_1307_2100_gb300 import autotune
    assert autotune.bucket_of(3201, 520, 300) == (9, 4)
    assert autotune.bucket_of(1, 7, 1) == (0, 0)
    assert autotune.bucket_of(1 << 20, 1 << 20, 1 << 30) == (10, 10)


def test_ger_mapping_limits():
    ger = tc.MAPPING["ger"]
    for K, want in ((32, 0), (33, 5), (1, 0)):
        A = (ts.lab("ai"), [40, K], None)
        B = (ts.lab("ib"), [K, 30], None)
        C = (ts.lab("ab"), [40, 30], None)
        assert tc.tc_plan_status(A, B, C, tc.TC_F64, 0, ger) == want, K
    A = (ts.lab("aij"), [40, 4, 4], None)
    B = (ts.lab("ijb"), [4, 4, 30], None)
    h = tc.tc_plan(A, B, (ts.lab("ab"), [40, 30], None), tc.TC_F32, tc.MATH["bf16x6"], ger)
    try:
        info = tc.tc_plan_get_info(h)
        assert tc.KERNEL_NAME[info.kernel] == "ger" and info.K == 16 and info.workspace == 0
    finally:
        tc.tc_plan_destroy(h)


def _restored(t, order):
    """Tensor t stored column-major in the given order of its index positions."""
    import copy
    u = copy.copy(t)
    u.strides = ts.storage_strides(t.extents, order)
    return u


@pytest.mark.parametrize("seed", range(3))
def test_layout_advice_turns_class_31_into_32(seed):
    rng = np.random.Generator(np.random.PCG64(2000 + seed))
    seen = 0
    for _ in range(6000):
        if seen >= 15:
            break
        p = ts.random_problem(rng, max_order=5, max_ext=4, min_ext=1, max_p=3)
        h = tc.tc_plan(_t(p.A), _t(p.B), _t(p.C), tc.TC_F64, 0)
        try:
            info, adv = tc.tc_plan_get_info(h), tc.tc_plan_layout_advice(h)
        finally:
            tc.tc_plan_destroy(h)
        if info.cls != 31:
            assert adv.operand == 0 and adv.cls_after == info.cls
            continue
        seen += 1
        assert adv.operand in (1, 2) and adv.cls_after == 32
        t = p.A if adv.operand == 1 else p.B
        order = list(adv.storage_order[: adv.order])
        assert sorted(order) == list(range(t.order))
        assert adv.copy_bytes == 2 * 8 * int(np.prod(t.extents))
        A2 = _restored(p.A, order) if adv.operand == 1 else p.A
        B2 = _restored(p.B, order) if adv.operand == 2 else p.B
        assert oc.classify(A2, B2, p.C).cls == 32
    assert seen >= 15


def test_layout_advice_on_the_paper_case():
    # Eq. xy (b): C[a,b,c,d] = sum A[i,a,j,b] B[j,c,i,d], Class 3.1; equal sizes: re-store B
    p = ts.fused_permute_48(n=8)
    h = tc.tc_plan(_t(p.A), _t(p.B), _t(p.C), tc.TC_F64, 0)
    try:
        adv = tc.tc_plan_layout_advice(h)
    finally:
        tc.tc_plan_destroy(h)
    assert adv.operand == 2 and adv.cls_after == 32
    assert ts.lab("jcid")[adv.storage_order[0]] in ts.lab("cd")   # a free index of B first


def test_batch_labels_form_the_batch_group():
    # C[a,b,z] = sum_i A[a,i,z] B[i,b,z]: one GEMM per z
    p = ts.problem("bat", "aiz", "ibz", "abz", dict(a=40, i=30, b=20, z=7), 91)
    info = plan_info(p)
    assert (info.cls, info.M, info.N, info.K, info.batch) == (32, 40, 20, 30, 7)
    assert info.slice_a & 4 and info.slice_b & 4            # z counts as sliced
    # the FP8 form and the COPY baseline take no batch labels
    p32 = f32p = ts.problem("bat", "aiz", "ibz", "abz", dict(a=40, i=30, b=20, z=7), 91,
                            dtype=np.float32)
    assert tc.tc_plan_status(_t(f32p.A), _t(f32p.B), _t(f32p.C), tc.TC_F32,
                             tc.MATH["fp8"]) == 5
    assert tc.tc_plan_status(_t(p.A), _t(p.B), _t(p.C), tc.TC_F64, 0,
                             tc.MAPPING["copy_gemm"]) == 5
    # Hadamard product (nothing contracted): K = 1
    h = ts.problem("had", "ab", "ab", "ab", dict(a=9, b=5), 92)
    hi = plan_info(h)
    assert hi.batch == 45 and hi.K == 1


def test_autotune_passes_repeat_while_changes_are_kept(monkeypatch):
    """The search over route and shape (1 tensor cores, 2 CUDA-core tiles, 3
    CUDA cores per output) repeats its visit of the buckets while a pass keeps
    a change: a bucket whose change pays only after another bucket moved is
    found in the second pass, and each visit keeps the faster of the two
    shapes tried (fake plans and a fake timer, no GPU)."""
    from types import SimpleNamespace
    from paper_1307_2100_gb300 import autotune
    # bucket X (4 items, per output by the rule) and bucket Y (2 items, tiles
    # by the rule; most flops: visited first)
    infos = ([SimpleNamespace(M=8, N=8, K=4, batch=1, flops=10.0)] * 4 +
             [SimpleNamespace(M=32, N=32, K=4, batch=1, flops=100.0)] * 2)
    monkeypatch.setattr(autotune.tc, "tc_plan_get_info", lambda h: infos[h])
    table = {(3, 2): 10.0, (3, 1): 11.0, (3, 3): 12.0, (1, 2): 8.0, (2, 2): 9.5,
             (1, 1): 6.0, (1, 3): 9.0, (2, 1): 7.0, (2, 3): 10.5}

    def fake_time(plans, routes, ptrs, stream, reps):
        return table[(int(routes[0]), int(routes[4]))]

    monkeypatch.setattr(autotune, "time_routes", fake_time)
    routes, rep = autotune.tune_routes(list(range(6)), None, None, passes=3)
    assert list(routes) == [1, 1, 1, 1, 1, 1]
    assert rep["default_ms"] == 10.0 and rep["tuned_ms"] == 6.0
    kept = [(t["pass"], tuple(t["bucket"]), t["route"]) for t in rep["trials"] if t["kept"]]
    assert kept == [(0, autotune.bucket_of(8, 8, 4), 1), (1, autotune.bucket_of(32, 32, 4), 1)]
    routes1, rep1 = autotune.tune_routes(list(range(6)), None, None, passes=1)
    assert list(routes1) == [1, 1, 1, 1, 2, 2] and rep1["tuned_ms"] == 8.0


def test_storage_and_math_combinations_planned_or_refused():
    """BF16 storage takes the FP32 and BF16 forms, FP16 storage the FP32 and
    FP16 forms; FP32 storage also takes the FP16 form."""
    p = ts.fused_permute_48(n=5)
    d = ((p.A.labels, p.A.extents, p.A.strides), (p.B.labels, p.B.extents, p.B.strides),
         (p.C.labels, p.C.extents, p.C.strides))
    ok = {("bf16", "fp32"), ("bf16", "bf16"), ("f16", "fp32"), ("f16", "fp16")}
    for dt in ("bf16", "f16"):
        for m in tc.MATH:
            st = tc.tc_plan_status(*d, tc.DTYPE[dt], tc.MATH[m])
            assert (st == 0) == ((dt, m) in ok), (dt, m, st)
    assert tc.tc_plan_status(*d, tc.TC_F32, tc.MATH["fp16"]) == 0
    assert tc.tc_plan_status(*d, 4, tc.MATH["fp32"]) == 1          # no such storage type


def test_packed_tile_defaults_by_form_and_shape():
    """Packed one-GEMM plans: CTA pairs (tile 5) for BF16 / FP16 / BF16x3 when
    M and N span two 128-row tiles and for BF16x6 when M does; 128 x 256
    tiles (4) for BF16x3 when only N does; 128 x 128 tiles (3) otherwise."""
    big = ts.problem("big", "ai", "ib", "ab", dict(a=300, i=64, b=300), 1)
    skinny_m = ts.problem("sm", "ai", "ib", "ab", dict(a=100, i=64, b=300), 2)
    skinny_n = ts.problem("sn", "ai", "ib", "ab", dict(a=300, i=64, b=100), 3)
    want = {("bf16", "big"): 5, ("bf16x3", "big"): 5, ("bf16x6", "big"): 5, ("fp16", "big"): 5,
            ("bf16", "sm"): 3, ("bf16x3", "sm"): 4, ("bf16x6", "sm"): 3,
            ("bf16", "sn"): 3, ("bf16x3", "sn"): 3, ("bf16x6", "sn"): 5}
    for (m, name), tile in want.items():
        p = {"big": big, "sm": skinny_m, "sn": skinny_n}[name]
        info = plan_info(p, tc.MATH[m], dtype=tc.TC_F32)
        assert info.tile == tile, (m, name, info.tile, info.M, info.N)



def test_fp8_tile_defaults():
    """FP8: CTA pairs over 256 x 256 tiles (tile 2) by default when M and N
    both span two 128-row tiles, else the 128 x 256 tiles (tile 0); the first
    operand packed inside the GEMM launch (tile 1) on request when it is a
    plain matrix with M contiguous and a K stride of a multiple of 16 bytes,
    and tile 1 refused otherwise."""
    fp8 = tc.MATH["fp8"]
    for p in (ts.problem("f", "ai", "ib", "ab", dict(a=300, i=200, b=130), 1),
              ts.precision_ccd(v=24, o=20)):
        assert plan_info(p, fp8, dtype=tc.TC_F32).tile == 2, p.name
        assert plan_info(p, fp8, tile=1, dtype=tc.TC_F32).tile == 1, p.name
    for d, want in ((dict(a=128, i=64, b=300), 0), (dict(a=300, i=64, b=128), 0),
                    (dict(a=129, i=64, b=129), 2)):
        p = ts.problem("edge", "ai", "ib", "ab", d, 4)
        assert plan_info(p, fp8, dtype=tc.TC_F32).tile == want, d
    for p in (ts.problem("odd", "ai", "ib", "ab", dict(a=130, i=200, b=140), 2),   # stride 130
              ts.direct_gemm_64(n=9),                                             # two M labels
              ts.problem("kfast", "ia", "ib", "ab", dict(a=300, i=200, b=130), 3)):  # K fastest
        with pytest.raises(tc.TcError) as e:
            plan_info(p, fp8, tile=1, dtype=tc.TC_F32)
        assert e.value.status == 5


def test_pair_tail_split_workspace():
    """CTA pairs (tile 5) split K over the tiles of a last, partial round:
    the plan's workspace then holds their partial sums on top of the packed
    operands (which tile 4 needs alone): parts x tail tiles x 4 quarters x
    128^2 (s, r) pairs of FP32.  80 pair tiles on 76 pairs: 4 tail tiles in
    2 parts; 76 tiles (a whole number of rounds) and K < 1024 (parts shorter
    than 512 K) split nothing."""
    bf16x3 = tc.MATH["bf16x3"]

    def extra(a, i, b):
        p = ts.problem("tail", "ai", "ib", "ab", dict(a=a, i=i, b=b), 5)
        w5 = plan_info(p, bf16x3, tile=5, dtype=tc.TC_F32).workspace
        w4 = plan_info(p, bf16x3, tile=4, dtype=tc.TC_F32).workspace
        return w5 - w4

    assert extra(2560, 1024, 2048) == 2 * 4 * 4 * 128 * 128 * 8   # 10 x 8 pair tiles
    assert extra(4864, 1024, 1024) == 0                            # 19 x 4 = 76 pair tiles
    assert extra(2560, 992, 2048) == 0                             # 31 K blocks: no 2 parts
