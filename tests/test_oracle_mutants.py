"""The oracle's pins must catch plausible mistakes.  Each mutant below is a
copy of the oracle's C source with one planted mistake, compiled on the CPU;
at least one pin must fail for every mutant."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "tco.c")

MUTANTS = {
    "dropped_last_term": ("for (int64_t k = 0; k < ncon; ++k)",
                          "for (int64_t k = 0; k < ncon - (ncon > 1); ++k)"),
    "wrong_sign": ("s = s + prod;", "s = s - prod;"),
    "transposed_A": ("out.sa[i] = pa >= 0 ? stride_of(A, pa) : 0;",
                     "out.sa[i] = pa >= 0 ? stride_of(A, A->order - 1 - pa) : 0;"),
    "beta_ignored": ("if (beta != 0.0) r = r + beta * c[oc];", ""),
    "alpha_ignored": ("double r = alpha * s;", "double r = s;"),
    "b_contracted_stride_from_a": ("con.sb[i] = stride_of(B, pb);", "con.sb[i] = stride_of(A, pa);"),
}

PINS = [
    pins.test_matrix_product_naive_triple_loop,
    pins.test_matrix_product_four_slicings_agree,
    pins.test_gemv_and_dot_naive,
    pins.test_all_ones_gives_product_of_contracted_extents,
    pins.test_rank_one_separable_inputs,
    pins.test_alpha_beta_and_beta_zero_never_reads_c,
    pins.test_integer_exact_against_einsum_moderate,
] + [lambda s=s: pins.test_brute_force_tiny_random_integer_exact(s) for s in range(6)]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, name
    mdir = tmp_path / name
    mdir.mkdir()
    (mdir / "tco.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(os.path.dirname(SRC), "tco.h"), mdir / "tco.h")
    so = mdir / "libtco_mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                    str(mdir / "tco.c"), "-o", str(so)], check=True, capture_output=True)
    saved = oracle._load()
    oracle._lib = oracle._configure(ctypes.CDLL(str(so)))
    failures = 0
    try:
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failures += 1
    finally:
        oracle._lib = saved
    assert failures >= 1, f"no pin caught mutant {name}"
